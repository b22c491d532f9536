"""Mixed precision (params.precision = 1): BF16 face weights in the sweeps,
exact FP32 defect passes.  The fixed point is the FP32 system's, so the result
meets the same parity bar against the FP64 oracle as the plain path."""
import numpy as np
import pytest

import oracle as O
from paper_2111_11866_gb300 import _lib, synth

from gpu_common import REL_TOL, gpu_run, label_mismatch_outside_band, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_11866_gb300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_mixed_tiny_config_matches_oracle():
    c = synth.tiny()
    p = _lib.Params.defaults()
    p.precision = 1
    gpu = gpu_run(c.image, c.seeds, c.nsteps, p)
    ref, _ = O.segment(c.image.astype(np.float64), c.seeds, oracle_params(p), nsteps=c.nsteps)
    err = np.abs(gpu["u"] - ref).max()
    assert err <= REL_TOL * np.abs(ref).max(), err
    assert label_mismatch_outside_band(gpu["u"], ref) == 0
    assert gpu["info"]["res_rel"] <= p.tol


@pytest.mark.parametrize("dims", [(69, 21, 13, 5), (33, 18, 9, 3)])
def test_mixed_equals_plain_within_tolerance(dims):
    c = synth.small_nuclei(seed=sum(dims), n=dims, count=3, nsteps=3)
    out = {}
    for prec in (0, 1):
        p = _lib.Params.defaults()
        p.r_ball = p.R_init = 6.0
        p.precision = prec
        out[prec] = gpu_run(c.image, c.seeds, c.nsteps, p)
    u0, u1 = out[0]["u"], out[1]["u"]
    assert np.abs(u1 - u0).max() <= REL_TOL * np.abs(u0).max()
    assert out[1]["info"]["res_rel"] <= p.tol


def test_mixed_is_not_the_bf16_system():
    """Without defect correction the BF16 system's solution is off by the
    weight rounding; the defect passes must win that back: compare against
    the oracle with a tolerance tighter than the BF16 rounding (2^-9)."""
    c = synth.small_nuclei(seed=12, n=(40, 30, 16, 4), count=2, nsteps=2)
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 6.0
    p.precision = 1
    p.tol = 1e-6
    gpu = gpu_run(c.image, c.seeds, c.nsteps, p)
    ref, _ = O.segment(c.image.astype(np.float64), c.seeds, oracle_params(p), nsteps=c.nsteps)
    assert np.abs(gpu["u"] - ref).max() <= 2e-5 * np.abs(ref).max()
