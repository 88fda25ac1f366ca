// Host evaluation of the compiled column program: the same program and the
// same evaluator (column_eval.h) the kernels use, callable without a GPU.
#include <vector>

#include "../../include/qmc.h"
#include "column_eval.h"
#include "term_compiler.h"

using namespace qmc;

namespace {

template <class M, class K>
int eval_t(const std::vector<uint8_t>& blob, uint64_t x, uint64_t y, int32_t cap, uint64_t* mask, uint64_t* mask_hi,
           int64_t* vre, int64_t* vim, int64_t* p_out)
{
    const ProgT<M, K> p = prog_at_t<M, K>(blob.data());
    int64_t sre, sim;
    *p_out = column_weight(p, (M)x, (M)y, &sre, &sim);
    if (*p_out > p.h->p_bound) return QMC_ERR_STATE; // the spawn filter bound must hold
    const int ne = p.h->n_entry;
    for (int e = 0; e < ne && e < cap; ++e) {
        int64_t a, b;
        entry_value(p, p.ent[e], (M)x, (M)y, sre, sim, &a, &b);
        mask[e] = (uint64_t)p.ent[e].mask_key;
        if (mask_hi) mask_hi[e] = (uint64_t)((u128)p.ent[e].mask_key >> 64);
        vre[e] = a;
        vim[e] = b;
    }
    return ne;
}

} // namespace

extern "C" int qmc_column_eval(int32_t n_qubits, const qmc_ham_term* ham, int32_t n_ham, const qmc_lindblad* lind,
                               int32_t n_lind, const qmc_pauli_coef* coefs, int32_t n_coefs, const qmc_rate* rates,
                               int32_t n_rates, const qmc_window* windows, int32_t n_windows, double t, double dt_eff,
                               uint64_t x, uint64_t y, int32_t cap, uint64_t* mask, uint64_t* mask_hi, int64_t* vre,
                               int64_t* vim, int64_t* p_out)
{
    if (n_qubits < 1 || n_qubits > QMC_MAX_QUBITS || !p_out) return QMC_ERR_INVALID_ARG;
    Schedule s;
    s.n = n_qubits;
    if (n_ham > 0) s.ham.assign(ham, ham + n_ham);
    if (n_lind > 0) s.lind.assign(lind, lind + n_lind);
    if (n_coefs > 0) s.coefs.assign(coefs, coefs + n_coefs);
    if (n_rates > 0) s.rates.assign(rates, rates + n_rates);
    if (n_windows > 0) s.windows.assign(windows, windows + n_windows);
    if (validate_schedule(s, nullptr) != QMC_OK) return QMC_ERR_INVALID_ARG;
    const uint64_t lim = (1ull << n_qubits) - 1;
    if ((x & ~lim) || (y & ~lim)) return QMC_ERR_INVALID_ARG;
    std::vector<uint8_t> blob;
    int rc = build_program(s, t, dt_eff, &blob);
    if (rc != QMC_OK) return rc;
    if (n_qubits <= 32) return eval_t<uint32_t, uint64_t>(blob, x, y, cap, mask, mask_hi, vre, vim, p_out);
    return eval_t<uint64_t, u128>(blob, x, y, cap, mask, mask_hi, vre, vim, p_out);
}
