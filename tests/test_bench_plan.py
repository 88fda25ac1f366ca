"""Host-side checks of the benchmark's workloads: every workload holds the
standard run of 5 warm-up + 20 timed steps, the population capacity covers the
growth over those steps, and the CPU leg reports its host."""
import pytest

import bench

WORKLOADS = ["spread32", "spread32s", "dd12", "dd12i", "ghz4", "ghz16", "ghz24", "ghz32", "ghz16i", "ghz32i"]


@pytest.mark.parametrize("name", WORKLOADS)
def test_workload_holds_standard_run(name):
    wl = bench.workload(name)
    pl, total, K = bench.plan_steps(wl, 5, 20)
    assert K == 20 and total >= 25
    # the default K also fits after the default warm-up
    _, _, k0 = bench.plan_steps(wl, 3, 0)
    assert k0 >= 1


def test_spread_stays_in_cnot_window():
    """The spread workloads run inside one CNOT pulse (t in [5, 6)), so every
    step of the plan has the same Liouvillian shape and dt."""
    wl = bench.workload("spread32")
    pl, total, _ = bench.plan_steps(wl, 5, 20)
    assert total == 100
    assert len(pl) == 1 and abs(pl[0][0] - 5.0) < 1e-12 and abs(pl[0][1] - 0.01) < 1e-12


def test_too_long_run_is_refused():
    wl = bench.workload("spread32")
    with pytest.raises(SystemExit):
        bench.plan_steps(wl, 5, 100)


def test_capacity_covers_growth():
    wl = bench.workload("spread32")
    base = wl["spread"] * wl["nseg"]
    # measured growth is about 1.3 % of the initial records per step
    for steps in (13, 25, 60):
        assert bench.capacity_hint(wl, steps) >= base * (1.0 + 0.013 * steps) * 1.2
    g = bench.workload("ghz4")   # from one state: one record per walker
    assert bench.capacity_hint(g, 25) >= g["n_diag"] * g["nseg"]


def test_cpu_info_names_host():
    info = bench.cpu_info()
    assert info["nproc"] >= 1 and isinstance(info["cpu_model"], str) and info["cpu_model"]


def test_oracle_vector_runs_whole_steps():
    w, s, n = bench.oracle_vector("ghz4", 0, 0.05)
    assert n >= 1 and w > 0 and s > 0
