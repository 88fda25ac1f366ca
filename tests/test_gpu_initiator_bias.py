"""Initiator bias and its xi -> 0 extrapolation where the exact answer is
known [End Matter, simulation methodology: the initiator truncation error
extrapolates to zero as xi -> 0].

GHZ-8 preparation (800 AB2 steps), 32 vectors of 10^5 walkers for each xi;
the exact reference is the dense AB2 recursion on the same time grid (applied
as operators).  Without the initiator the walker mean is unbiased; with it,
the fidelity's bias at xi = 10^-3 must lie within the error of the linear
xi -> 0 extrapolation of the xi > 0 runs, and that extrapolation must agree
with the exact value.
"""
import math

import numpy as np
import pytest

from oracle import dense as Dn
from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import studies

pytestmark = pytest.mark.gpu


def test_ghz8_initiator_extrapolates_to_exact():
    n = 8
    rows = studies.initiator_study(sizes=(n,), xis=(1e-2, 3e-3, 1e-3, 3e-4, 0.0), nvec=32, n_diag=10**5,
                                   zero_max_n=n)
    prob = P.ghz_circuit(n)
    ref = Dn.evolve_operators(prob, Dn.rho_from_entries(n, P.rho_basis(0)), 0.01, 800, "ab2")
    f_exact = Dn.fidelity(ref, P.ghz_target(n))
    by_xi = {r["xi"]: r for r in rows}
    z0 = by_xi[0.0]
    assert abs(z0["fidelity"] - f_exact) < 3 * z0["fidelity_se"], (z0, f_exact)
    r3 = by_xi[1e-3]
    F0, se0 = r3["extrapolated_F0"], r3["extrapolated_se"]
    assert abs(F0 - f_exact) < 3 * se0, (F0, se0, f_exact)
    assert abs(r3["fidelity"] - f_exact) < 3 * math.hypot(se0, r3["fidelity_se"]), (r3, f_exact)
    # the initiator keeps the walker count smaller
    assert by_xi[1e-2]["records_final"] <= z0["records_final"]
    print({k: (round(v["fidelity"], 5), round(v["fidelity_se"], 5)) for k, v in by_xi.items()}, f_exact)
