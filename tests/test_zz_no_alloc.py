"""qmc_observables_noalloc against qmc_observables.

Some callers cannot call cudaMalloc: code running under an external memory
manager that has already reserved the device memory, and code that must not
risk the implicit synchronisation cudaMalloc and cudaFree can cause.  They hold
the population in their own device memory and call qmc_observables_noalloc,
which accumulates into a static device array owned by the library.  Its
per-vector counts must equal those of qmc_observables exactly, on two calls in
a row (the second call reuses the same accumulators, which must be cleared
first).
"""
import ctypes as C

import numpy as np
import pytest

from paper_2502_18929_gb300 import problems as P
from paper_2502_18929_gb300 import qmc

pytestmark = pytest.mark.gpu

MAX_SEGMENTS = 4096   # QMC_NOALLOC_MAX_SEGMENTS in include/qmc.h


def _device_population(gpu):
    """The context's N(t) copied into caller-owned device memory."""
    import torch
    keys, res, ims, counts = [], [], [], []
    for s in range(gpu.nseg):
        k, r, i = gpu.export(s)
        keys.append(k)
        res.append(r)
        ims.append(i)
        counts.append(len(k))
    rec = np.zeros(sum(counts), dtype=[("key", "<u8"), ("re", "<i4"), ("im", "<i4")])
    rec["key"] = np.concatenate(keys)
    rec["re"] = np.concatenate(res)
    rec["im"] = np.concatenate(ims)
    off = np.zeros(gpu.nseg + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    d_rec = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
    d_off = torch.from_numpy(off).cuda()
    return d_rec, d_off


def test_noalloc_matches_qmc_observables_twice():
    import torch
    torch.cuda.init()
    nseg = 6
    gpu = qmc.QMC(4, nseg, 99, 3000)
    gpu.load_schedule(P.ghz_circuit(4))
    gpu.init_populations(P.rho_basis(0))
    L = qmc.lib()
    stream = torch.cuda.current_stream()
    out = torch.empty((nseg, 4), dtype=torch.int64, device="cuda")
    for call in range(2):
        gpu.step(0.01, 40 + 30 * call)   # a different population on each call
        d_rec, d_off = _device_population(gpu)
        out.fill_(-1)
        rc = L.qmc_observables_noalloc(C.c_void_p(d_rec.data_ptr()), C.c_void_p(d_off.data_ptr()), nseg, 4,
                                       C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == qmc.OK
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), gpu.observables()), f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    torch.cuda.init()
    L = qmc.lib()
    d = torch.zeros(64, dtype=torch.int64, device="cuda")
    out = torch.zeros((8, 4), dtype=torch.int64, device="cuda")
    rc = L.qmc_observables_noalloc(C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()), MAX_SEGMENTS + 1, 4,
                                   C.c_void_p(out.data_ptr()), None)
    assert rc == qmc.ERR_INVALID_ARG
