"""Pins for the oracle's random numbers: Philox4x32-10 against an independent
implementation (PyTorch's host philox_engine, compiled from its installed header),
the exact uniform conversion, and uniformity of the stream."""
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

_HELPER = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
int main() {
  unsigned long long seed, sub, off;
  while (std::scanf("%llx %llx %llx", &seed, &sub, &off) == 3) {
    at::philox_engine e(seed, sub, off);
    unsigned w0 = e(); unsigned w1 = e(); unsigned w2 = e(); unsigned w3 = e();
    std::printf("%08x %08x %08x %08x\n", w0, w1, w2, w3);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def torch_philox():
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    d = tempfile.mkdtemp(prefix="philox_xcheck_")
    src, exe = os.path.join(d, "x.cpp"), os.path.join(d, "x")
    with open(src, "w") as f:
        f.write(_HELPER)
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", inc, src, "-o", exe])

    def run(triples):
        inp = "".join(f"{s:x} {b:x} {o:x}\n" for s, b, o in triples)
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True)
        return [[int(v, 16) for v in line.split()] for line in out.stdout.strip().splitlines()]
    return run


def test_philox_matches_torch_engine(oracle, torch_philox):
    # torch's engine: key = seed (lo, hi); counter = (offset lo, offset hi,
    # subsequence lo, subsequence hi); its first four outputs are one Philox block.
    rng = np.random.default_rng(123)
    triples, ours = [], []
    for i in range(300):
        seed = int(rng.integers(0, 2**63)) * 2 + int(i & 1)
        c = [int(v) for v in rng.integers(0, 2**32, size=4, dtype=np.uint64)]
        if i < 4:
            c = [0, 0, 0, 0] if i == 0 else [0xffffffff] * 4 if i == 1 else c
            seed = 0 if i == 0 else (2**64 - 1 if i == 1 else seed)
        sub = c[2] | (c[3] << 32)
        off = c[0] | (c[1] << 32)
        triples.append((seed, sub, off))
        ours.append(oracle.philox(c, [seed & 0xffffffff, seed >> 32]))
    assert torch_philox(triples) == ours


def test_uniform_conversion_exact(oracle):
    # u = (n + 1/2) 2^-52 with n = (w0>>6) 2^26 + (w1>>6), exactly, in (0, 1).
    rng = np.random.default_rng(5)
    cases = [(0, 0), (0xffffffff, 0xffffffff), (0x3f, 0x3f), (0x40, 0)]
    cases += [tuple(int(v) for v in rng.integers(0, 2**32, 2, dtype=np.uint64)) for _ in range(2000)]
    for w0, w1 in cases:
        n = ((w0 >> 6) << 26) | (w1 >> 6)
        assert Fraction(oracle.u01(w0, w1)) == Fraction(2 * n + 1, 2**53)
    assert oracle.u01(0, 0) == 2.0**-53
    assert oracle.u01(0xffffffff, 0xffffffff) == 1.0 - 2.0**-53


def test_uniform_stream_is_uniform(oracle):
    us = []
    for i in range(20000):
        w = oracle.philox([i, 7, 3, 0], [11, 0])
        us.append(oracle.u01(w[0], w[1]))
        us.append(oracle.u01(w[2], w[3]))
    assert stats.kstest(us, "uniform").pvalue > 1e-3
    # words are not correlated across the two halves of one block
    us = np.array(us).reshape(-1, 2)
    assert abs(np.corrcoef(us[:, 0], us[:, 1])[0, 1]) < 0.03
