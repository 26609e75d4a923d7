"""The kernels on the stored oracle fixtures (tests/golden/), FP32, within
the FP32 parity gates: a check that needs no oracle run on the GPU host."""
import json
import os

import numpy as np
import pytest
import torch

from paper_1803_05619_gb300 import _lib as L
from paper_1803_05619_gb300.layer import gf_backward, gf_forward
from tests.helpers import assert_fwd, assert_grad, f64

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = sorted(f[:-5] for f in os.listdir(GOLDEN) if f.endswith(".json"))


@pytest.mark.parametrize("name", NAMES)
def test_kernels_match_stored_fixture(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        g = json.load(f)
    x = {k: torch.tensor(np.asarray(v), dtype=torch.float32).cuda() for k, v in g["inputs"].items()}
    r, eps = g["r"], g["eps"]
    out = gf_forward(x["p_l"], x["I_l"], x["I_h"], r, eps)
    dp, dil, dih, _ = gf_backward(x["R"], x["p_l"], x["I_l"], x["I_h"], r, eps)
    torch.cuda.synchronize()
    e = {k: np.asarray(v) for k, v in g["expected"].items()}
    assert_fwd(f64(out), e["O_h"], torch.float32, eps)
    assert_grad(f64(dp), e["dp_l"], torch.float32, "dp_l")
    assert_grad(f64(dil), e["dI_l"], torch.float32, "dI_l")
    assert_grad(f64(dih), e["dI_h"], torch.float32, "dI_h")
    assert L.dgf_device_status() == 0
