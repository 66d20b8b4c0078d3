"""A model read from an SBML file goes through the CUDA path: the golden Level 2 file of
the stiff decaying-dimerizing network (the paper's third Table 1 model) is parsed by the
package's reader and simulated by ml_simulate in reference precision, bit-identical to the
oracle on the same network (thread and warp kernels)."""
import os

import numpy as np
import pytest

from paper_1608_07058_gb300 import sbml
from tests.test_gpu_parity import assert_bit_parity, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "decaying_dimerizing_l2.xml")


@pytest.fixture(scope="module")
def ml():
    import torch
    from paper_1608_07058_gb300 import build, matleap
    assert torch.cuda.is_available()
    build.build()
    matleap.lib()
    return matleap


@pytest.mark.parametrize("shape", [0, 2])
def test_sbml_model_bit_parity(ml, oracle, shape):
    m = sbml.load_sbml(GOLDEN)
    g = run_gpu(ml, m.crn, 2000, m.x0, [0.2], seed=15, shape=shape)
    o = run_oracle(oracle, m.crn, 2000, m.x0, [0.2], seed=15)
    assert_bit_parity(g, o, f"sbml shape {shape}")
    assert (g["counters"][:, 1] > 0).all()  # the stiff pair takes implicit leaps
