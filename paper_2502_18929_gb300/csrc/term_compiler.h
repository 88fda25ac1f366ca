// Host-side term compiler: schedule -> expanded Pauli superoperator terms ->
// per-step column programs (see qmc_types.h for the layout).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qmc.h"

namespace qmc {

struct Schedule {
    int n = 0;
    std::vector<qmc_ham_term> ham;
    std::vector<qmc_lindblad> lind;
    std::vector<qmc_pauli_coef> coefs;
    std::vector<qmc_rate> rates;
    std::vector<qmc_window> windows;
};

// Validate ids and masks; returns QMC_OK or QMC_ERR_INVALID_ARG with a reason.
int validate_schedule(const Schedule& s, std::string* why);

// Column program of dt_eff * L(t) appended to blob (8-byte aligned).
// Returns QMC_OK or QMC_ERR_COEF_RANGE.
int build_program(const Schedule& s, double t, double dt_eff, std::vector<uint8_t>* blob);

// Bound on the spawn probability of any state: dt_eff * sum over expanded
// terms of (|Re c| + |Im c|) |rate|.
double spawn_prob_bound(const Schedule& s, double t, double dt_eff);

// FNV-1a hash of the schedule and configuration (for checkpoints).
uint64_t schedule_hash(const Schedule& s, uint64_t seed, int32_t nseg, int32_t integrator,
                       int64_t n_diag, int64_t init_min);

} // namespace qmc
