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


def _call(L, d_rec, d_off, nseg, n, out, stream):
    return L.qmc_observables_noalloc(C.c_void_p(d_rec.data_ptr()), C.c_void_p(d_off.data_ptr()), nseg, n,
                                     C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))


def _host_obs(keys, re, im, off, n):
    """Per-vector K, N_tot, N^diag of back-to-back records (host reference)."""
    nseg = len(off) - 1
    out = np.zeros((nseg, 4), dtype=np.int64)
    ymask = np.uint64((1 << n) - 1)
    diag = (keys >> np.uint64(n)) == (keys & ymask)
    for s in range(nseg):
        a, b = off[s], off[s + 1]
        out[s, 0] = b - a
        out[s, 1] = np.abs(re[a:b].astype(np.int64)).sum() + np.abs(im[a:b].astype(np.int64)).sum()
        out[s, 2] = re[a:b][diag[a:b]].astype(np.int64).sum()
        out[s, 3] = im[a:b][diag[a:b]].astype(np.int64).sum()
    return out


def test_noalloc_empty_vectors_and_32_qubit_keys():
    """Vectors of very different sizes with empty ones in the middle and at
    the end, keys of 32 qubits (x in the high word), records placed after an
    unused head (seg_offsets[0] > 0); checked against a host sum and against
    qmc_observables on the same population, on two calls in a row."""
    import torch
    torch.cuda.init()
    rng = np.random.default_rng(5)
    n = 32
    sizes = [70000, 0, 3, 1, 0, 129, 40000, 0]
    nseg = len(sizes)
    head = 5
    L = qmc.lib()
    stream = torch.cuda.current_stream()
    out = torch.empty((nseg, 4), dtype=torch.int64, device="cuda")
    for call in range(2):
        pops = []
        for s, m in enumerate(sizes):
            x = rng.integers(0, 1 << 32, size=m, dtype=np.uint64)
            y = np.where(rng.random(m) < 0.3, x, rng.integers(0, 1 << 32, size=m, dtype=np.uint64))
            keys = np.unique((x << np.uint64(32)) | y)
            re = rng.integers(-3000, 3000, size=len(keys)).astype(np.int32)
            im = rng.integers(-3000, 3000, size=len(keys)).astype(np.int32)
            re[(re == 0) & (im == 0)] = 1
            pops.append((keys, re, im))
        counts = np.array([len(p[0]) for p in pops], dtype=np.int64)
        off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        keys = np.concatenate([p[0] for p in pops])
        re = np.concatenate([p[1] for p in pops])
        im = np.concatenate([p[2] for p in pops])
        expect = _host_obs(keys, re, im, off, n)
        rec = np.zeros(head + len(keys), dtype=[("key", "<u8"), ("re", "<i4"), ("im", "<i4")])
        rec["key"][:head] = 12345
        rec["re"][:head] = 7777
        rec["key"][head:] = keys
        rec["re"][head:] = re
        rec["im"][head:] = im
        d_rec = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
        d_off = torch.from_numpy(off + head).cuda()
        out.fill_(-1)
        assert _call(L, d_rec, d_off, nseg, n, out, stream) == qmc.OK
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), expect), f"call {call}"
        ctx = qmc.QMC(n, nseg, 1, 1000)
        ctx.load_schedule(P.pure_noise(n, 0.01, 0.0))
        ctx.set_populations(pops)
        assert np.array_equal(ctx.observables(), expect)
        ctx.close()


def test_noalloc_allocates_no_device_memory():
    """After the first call on the device (which looks up the static array's
    address and loads the kernels), further calls leave the free device
    memory unchanged."""
    import torch
    torch.cuda.init()
    nseg = 300
    rng = np.random.default_rng(1)
    counts = rng.integers(0, 2000, size=nseg)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    rec = np.zeros(int(off[-1]), dtype=[("key", "<u8"), ("re", "<i4"), ("im", "<i4")])
    rec["key"] = np.arange(len(rec), dtype=np.uint64)
    rec["re"] = 1
    d_rec = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
    d_off = torch.from_numpy(off).cuda()
    out = torch.empty((nseg, 4), dtype=torch.int64, device="cuda")
    L = qmc.lib()
    stream = torch.cuda.current_stream()
    assert _call(L, d_rec, d_off, nseg, 10, out, stream) == qmc.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        assert _call(L, d_rec, d_off, nseg, 10, out, stream) == qmc.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(out[:, 0].cpu().numpy(), counts)


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    torch.cuda.init()
    L = qmc.lib()
    d = torch.zeros(64, dtype=torch.int64, device="cuda")
    out = torch.zeros((8, 4), dtype=torch.int64, device="cuda")
    rc = L.qmc_observables_noalloc(C.c_void_p(d.data_ptr()), C.c_void_p(d.data_ptr()), MAX_SEGMENTS + 1, 4,
                                   C.c_void_p(out.data_ptr()), None)
    assert rc == qmc.ERR_INVALID_ARG
