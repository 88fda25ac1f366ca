"""Pins of the oracle's Philox4x32-10 (the paper names no generator; the
counter-based stream is reading R3 of the design)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(v, 16) for v in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("row", _kat())
def test_known_answer_vectors(row):
    ctr, key, expect = row
    assert list(O.philox(ctr, key)) == expect


def _torch_include():
    try:
        import torch
    except Exception:  # pragma: no cover
        return None
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        return inc
    return None


def test_matches_torch_philox_engine(tmp_path):
    """Cross-check against an independent implementation: PyTorch's header-only
    at::philox_engine (counter = {offset, subsequence}, key = seed)."""
    inc = _torch_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("torch headers or g++ not available")
    src = tmp_path / "t.cpp"
    src.write_text(r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char** argv) {
  for (int i = 1; i + 2 < argc; i += 3) {
    at::philox_engine e(strtoull(argv[i], 0, 0), strtoull(argv[i + 1], 0, 0),
                        strtoull(argv[i + 2], 0, 0));
    for (int j = 0; j < 4; ++j) printf("%u ", e());
    printf("\n");
  }
}
""")
    exe = tmp_path / "t"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", inc, "-o", str(exe), str(src)], check=True)
    rng = np.random.default_rng(7)
    args, cases = [], []
    for _ in range(64):
        ctr = rng.integers(0, 2**32, size=4, dtype=np.uint64)
        key = rng.integers(0, 2**32, size=2, dtype=np.uint64)
        seed = int(key[0]) | (int(key[1]) << 32)
        sub = int(ctr[2]) | (int(ctr[3]) << 32)
        off = int(ctr[0]) | (int(ctr[1]) << 32)
        args += [str(seed), str(sub), str(off)]
        cases.append((ctr.astype(np.uint32), key.astype(np.uint32)))
    out = subprocess.run([str(exe)] + args, check=True, capture_output=True, text=True).stdout
    lines = out.strip().splitlines()
    assert len(lines) == len(cases)
    for (ctr, key), line in zip(cases, lines):
        expect = [int(v) for v in line.split()]
        assert list(O.philox(ctr, key)) == expect


def test_uniform_words_are_unbiased():
    """The 52-bit words the spawn step compares against P are uniform: their
    mean and the fraction below a threshold match the uniform law."""
    ctrs = np.arange(20000, dtype=np.uint64)
    vals = []
    for c in ctrs[:4000]:
        w = O.philox([int(c), 0, 5, 0], [11, 13])
        vals.append(((int(w[1]) << 32) | int(w[0])) >> 12)
        vals.append(((int(w[3]) << 32) | int(w[2])) >> 12)
    u = np.array(vals, dtype=np.float64) / 2.0**52
    assert abs(u.mean() - 0.5) < 3 * (1 / np.sqrt(12 * len(u)))
    frac = (u < 0.1).mean()
    assert abs(frac - 0.1) < 3 * np.sqrt(0.09 / len(u))


def test_walker_draws_uniform_and_independent():
    """The spawn draws T (52 bits) of the walkers of many parents: the first
    walkers of four consecutive ranks share one Philox call, further walkers
    take four words of their parent's call, and every walker adds its own low
    bits.  T must be uniform on [0, 2^52) (chi-square over 64 bins of the top
    bits and of the low 20 bits) and the draws of neighbouring walkers
    uncorrelated -- the law of the per-walker Bernoulli(p) spawn test needs
    exactly that."""
    from scipy import stats
    kd = [0x9E3779B9, 0x7F4A7C15]
    T, Tn, Tw = [], [], []
    for r in range(6000):
        are = 1 + r % 2      # 1 or 2 real walkers, then 1 imaginary one
        t0 = O.walker_T(kd, r, r & 1, 0, 0, are)
        T.append(t0)
        Tn.append(O.walker_T(kd, r + 1, r & 1, 0, 0, 1))      # first walker of the next rank
        Tw.append(O.walker_T(kd, r, r & 1, 1, 0, are))   # first imaginary walker
    T, Tn, Tw = (np.array(a, dtype=np.float64) for a in (T, Tn, Tw))
    assert T.min() >= 0 and T.max() < 2.0 ** 52
    for vals in (np.floor(T / 2.0 ** 46), np.mod(T, 2.0 ** 20) // 2.0 ** 14):
        counts = np.bincount(vals.astype(np.int64), minlength=64)
        assert stats.chisquare(counts).pvalue > 1e-3
    for other in (Tn, Tw):
        rho = np.corrcoef(T, other)[0, 1]
        assert abs(rho) < 3.0 / np.sqrt(len(T))
