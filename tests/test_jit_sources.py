"""Model-specialized kernels, host side (no GPU): the generated source of every driver,
precision and register budget compiles with NVRTC for sm_103a, for networks covering
the code paths the tables switch on -- zero-order and first-order reactions only,
a reversible pair in partial equilibrium (the implicit solve), second- and third-order
reactions with their step-size factors, and the padded 8 x 16 variant.  The device
results of these kernels are checked against the oracle by tests/test_gpu_specialized.py.
"""
import os
import subprocess

import numpy as np
import pytest

from paper_1608_07058_gb300 import build as B
from paper_1608_07058_gb300 import workloads as W
from tests.test_gpu_parity import _generic_network

HERE = os.path.dirname(os.path.abspath(__file__))

# (species, reactions) capacities of the thread variants, smallest first
VARIANTS = [(1, 2), (3, 4), (3, 6), (8, 16)]


def _tables(crn):
    """The derived tables a kernel takes: reversible partners (net changes of opposite
    sign), reactant flags and the highest-order flags of each species (Cao 2006)."""
    o, nu = crn.orders, crn.stoich
    M, N = o.shape
    partner = -np.ones(M, np.int64)
    n_pairs = 0
    for j in range(M):
        for k in range(j + 1, M):
            if partner[j] < 0 and partner[k] < 0 and nu[j].any() and (nu[j] == -nu[k]).all():
                partner[j], partner[k] = k, j
                n_pairs += 1
    isreact = (o > 0).any(0).astype(np.int64)
    hor = np.zeros(N, np.int64)
    flag = {(1, 1): 1, (2, 1): 2, (2, 2): 4, (3, 1): 8, (3, 2): 16, (3, 3): 32}
    for j in range(M):
        tot = int(o[j].sum())
        for s in range(N):
            if o[j, s] > 0:
                hor[s] |= flag[(tot, int(o[j, s]))]
    NM, MM = next(v for v in VARIANTS if N <= v[0] and M <= v[1])
    fields = [N, M, NM, MM, n_pairs, *o.ravel(), *nu.ravel(), *partner, *isreact, *hor]
    return " ".join(str(int(v)) for v in fields) + " " + " ".join(repr(float(r)) for r in crn.rates)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = B._nvcc()
    os.makedirs(B.BUILD, exist_ok=True)
    B._write_jit_sources()
    exe = str(tmp_path_factory.mktemp("jit") / "jit_check")
    cmd = [nvcc, "-std=c++17", "-O1", "-I", B.CSRC, "-I", B.BUILD, "-I", B.INCLUDE,
           os.path.join(HERE, "jit_check.cu"), os.path.join(B.CSRC, "jit.cu"), "-o", exe,
           "-L", B._cuda_lib_dir(nvcc), "-lnvrtc", "-Xlinker", "-rpath",
           "-Xlinker", B._cuda_lib_dir(nvcc)]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-3000:]
    return exe


# (driver, reference precision, occupancy build): driver 0 round-based, 1 pool, 2 sequential
CASES = [
    (W.immigration_death(), [(0, 0, 0)]),
    (W.dimerisation(), [(2, 0, 0), (2, 1, 0)]),        # a pair: implicit leaps, both precisions
    (W.gene_expression(), [(1, 0, 0), (1, 0, 1)]),     # the pool driver, both register budgets
    (_generic_network(), [(0, 0, 1), (1, 1, 0)]),      # orders 2 and 3, a pair, 8 x 16 variant
]


def test_specialized_sources_compile(checker):
    stdin = "".join(f"{len(c)} " + " ".join(f"{d} {r} {o}" for d, r, o in c) + " " +
                    _tables(m) + "\n" for m, c in CASES)
    res = subprocess.run([checker], input=stdin, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-4000:] + res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("ok ")]
    assert len(lines) == sum(len(c) for _, c in CASES)
    assert all(int(ln.split()[-1]) > 0 for ln in lines)
