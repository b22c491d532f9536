"""Batched windows in mixed precision: BF16 face weights in the batched sweeps,
exact FP32 defect passes; same parity bar against the oracle, same
alone-vs-mix bit equality as the FP32 batch."""
import numpy as np
import pytest

import oracle as O
from paper_2111_11866_gb300 import _lib, synth

from gpu_common import REL_TOL, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_11866_gb300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _params(precision):
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 6.0
    p.precision = precision
    return p


def _specs():
    out = {}
    for k, (seed, n) in enumerate([(201, (37, 29, 17, 5)), (202, (24, 24, 24, 4))]):
        c = synth.small_nuclei(seed=seed, n=n, count=2, nsteps=3)
        out[k] = (c.image, c.seeds, 3)
    return out


def _run(specs, p):
    res = {}
    with _lib.Batch(1 << 30, 16, params=p) as b:
        ids = {k: b.add(*v) for k, v in specs.items()}
        for _ in range(3):
            b.advance()
        for k, wid in ids.items():
            assert b.poll(wid)["state"] == "done"
            res[k] = b.read_u(wid)
    return res


def test_mixed_batch_matches_oracle_and_is_mix_independent():
    specs = _specs()
    p = _params(1)
    mix = _run(specs, p)
    P = oracle_params(p)
    for k, (img, seeds, nsteps) in specs.items():
        ref, _ = O.segment(img.astype(np.float64), seeds, P, nsteps=nsteps)
        assert np.abs(mix[k] - ref).max() <= REL_TOL * np.abs(ref).max()
        alone = _run({k: specs[k]}, p)
        np.testing.assert_array_equal(alone[k], mix[k])


def test_precision_fixed_while_windows_resident():
    specs = _specs()
    with _lib.Batch(1 << 30, 4, params=_params(0)) as b:
        b.add(*specs[0])
        with pytest.raises(_lib.Seg4DError):
            b.set_params(precision=1)
    assert _lib.Batch.window_bytes((24, 24, 24, 4), 1, 1) > _lib.Batch.window_bytes((24, 24, 24, 4))


def test_sampled_config4_windows_match_oracle():
    """Windows of the batched workload itself (per-nucleus windows of the
    medium generator, cubic edge 24-64, 8-16 frames, 30 steps), in the mode
    the bench runs them (mixed precision, all in one batch): the four smallest
    of the first 64 windows against the FP64 oracle, per-voxel bound and
    labels outside a one-voxel band."""
    from gpu_common import label_mismatch_outside_band
    wins = synth.windows(64)
    pick = sorted(range(len(wins)), key=lambda k: wins[k][0].size)[:4]
    specs = {k: wins[k] for k in pick}
    p = _lib.Params.defaults()
    p.precision = 1
    with _lib.Batch(4 << 30, 16, params=p) as b:
        ids = {k: b.add(*v) for k, v in specs.items()}
        for _ in range(max(v[2] for v in specs.values())):
            b.advance()
        res = {}
        for k, wid in ids.items():
            info = b.poll(wid)
            assert info["state"] == "done" and info["steps_done"] == specs[k][2], info
            res[k] = b.read_u(wid)
    P = oracle_params(p)
    for k, (img, seeds, nsteps) in specs.items():
        ref, info = O.segment(img.astype(np.float64), seeds, P, nsteps=nsteps)
        assert info["status"] == O.OR_OK
        err = np.abs(res[k] - ref).max()
        assert err <= REL_TOL * np.abs(ref).max(), (k, img.shape, err)
        assert label_mismatch_outside_band(res[k], ref) == 0, k
