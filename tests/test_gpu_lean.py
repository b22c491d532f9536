"""A lean handle (SEG4D_CREATE_LEAN, 64 B/voxel): the image fields live inside
G during the set-up and the FP32 solve sweeps its correction system unscaled.
The result meets the same parity bar against the oracle; the image fields are
not kept, and new seeds need the image again."""
import numpy as np
import pytest

import oracle as O
from paper_2111_11866_gb300 import _lib, synth

from gpu_common import REL_TOL, label_mismatch_outside_band, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_11866_gb300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(c, p, lean, nsteps):
    with _lib.Seg4D(c.dims, params=p, lean=lean) as s:
        s.set_image(c.image)
        s.set_seeds(c.seeds)
        s.setup()
        G = s.read_field("G")
        info = s.step(nsteps)
        return s.read_u(), G, info


@pytest.mark.parametrize("dims", [(69, 21, 13, 5), (40, 36, 20, 6)])
def test_lean_matches_oracle_and_full_handle(dims):
    c = synth.small_nuclei(seed=sum(dims), n=dims, count=3, nsteps=3)
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 6.0
    u_lean, G_lean, info = _run(c, p, True, c.nsteps)
    u_full, G_full, _ = _run(c, p, False, c.nsteps)
    # the presmoothing solves of the two handles round differently (unscaled
    # vs scaled correction sweeps): G agrees to the set-up's parity bar
    assert np.abs(G_lean - G_full).max() <= 1e-3
    ref, _ = O.segment(c.image.astype(np.float64), c.seeds, oracle_params(p), nsteps=c.nsteps)
    for u in (u_lean, u_full):
        assert np.abs(u - ref).max() <= REL_TOL * np.abs(ref).max()
        assert label_mismatch_outside_band(u, ref) == 0
    assert info["res_rel"] <= p.tol


def test_lean_keeps_no_image_and_needs_it_for_new_seeds():
    c = synth.small_nuclei(seed=5, n=(30, 20, 10, 4), count=2, nsteps=1)
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 5.0
    dims = c.dims
    assert _lib.Seg4D.device_bytes(dims, lean=True) < _lib.Seg4D.device_bytes(dims)
    with _lib.Seg4D(dims, params=p, lean=True) as s:
        s.set_image(c.image)
        np.testing.assert_array_equal(s.read_field("I0"), c.image)   # before the set-up
        s.set_seeds(c.seeds)
        s.setup()
        for name in ("I0", "ITH", "Isig0", "IsigTH"):
            with pytest.raises(_lib.Seg4DError) as e:
                s.read_field(name)
            assert e.value.status == _lib.ERR_STATE
        s.set_seeds(c.seeds[:1])
        with pytest.raises(_lib.Seg4DError) as e:
            s.step(1)
        assert e.value.status == _lib.ERR_STATE
        s.set_image(c.image)
        info = s.step(1)
        assert info["status"] == _lib.OK


def test_lean_mixed_precision_matches_oracle():
    """Mixed precision on a lean handle (the configuration of the paper-scale
    grid in mixed precision): BF16 sweep weights beside the lean arrays, the
    same parity bar against the oracle."""
    c = synth.small_nuclei(seed=77, n=(45, 30, 16, 6), count=3, nsteps=3)
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 6.0
    p.precision = 1
    u, _, info = _run(c, p, True, c.nsteps)
    ref, _ = O.segment(c.image.astype(np.float64), c.seeds, oracle_params(p), nsteps=c.nsteps)
    assert np.abs(u - ref).max() <= REL_TOL * np.abs(ref).max()
    assert label_mismatch_outside_band(u, ref) == 0
    assert info["status"] == _lib.OK
