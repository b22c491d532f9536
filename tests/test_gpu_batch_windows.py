"""Windows of the batched workload against the FP64 oracle across the whole
size range: the per-nucleus windows of the medium generator (cubic edge
24-64, 8-16 frames), in the mode the bench runs them (mixed precision, all
in one batch).

- all of the first 64 windows, 3 steps each (the oracle's runs in a pool of
  host processes);
- the largest of them (64^3 x 16) and the median one, the workload's 30
  steps (the oracle on its OpenMP build).

Bars: |u - u_oracle| <= 1e-4 max|u_oracle| per voxel and identical labels
outside a one-voxel band of the oracle's level set."""
import numpy as np
import pytest

import oracle as O
from paper_2111_11866_gb300 import _lib, synth

from gpu_common import (REL_TOL, label_mismatch_outside_band, oracle_params,
                        oracle_segment_many)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_11866_gb300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _batched(specs, p):
    need = sum(_lib.Batch.window_bytes(tuple(reversed(v[0].shape)), len(v[1]), p.precision)
               for v in specs.values())
    with _lib.Batch(int(need * 1.1) + (256 << 20), len(specs) + 1, params=p) as b:
        ids = {k: b.add(*v) for k, v in specs.items()}
        for _ in range(max(v[2] for v in specs.values())):
            b.advance()
        res = {}
        for k, wid in ids.items():
            info = b.poll(wid)
            assert info["state"] == "done" and info["steps_done"] == specs[k][2], info
            res[k] = b.read_u(wid)
    return res


def _check(k, u, ref, shape):
    err = float(np.abs(u - ref).max())
    assert err <= REL_TOL * float(np.abs(ref).max()), (k, shape, err)
    assert label_mismatch_outside_band(u, ref) == 0, (k, shape)


def test_all_64_sampled_windows_three_steps():
    wins = synth.windows(64, nsteps=3)
    specs = dict(enumerate(wins))
    p = _lib.Params.defaults()
    p.precision = 1
    res = _batched(specs, p)
    refs = oracle_segment_many(wins, oracle_params(p))
    sizes = []
    for k, (img, _, _) in specs.items():
        ref, info = refs[k]
        assert info["status"] == O.OR_OK
        _check(k, res[k], ref, img.shape)
        sizes.append(img.size)
    assert max(sizes) == 64 ** 3 * 16 and min(sizes) < 200000   # the whole size range


def test_largest_and_median_windows_thirty_steps():
    try:
        O.lib(omp=True)
    except OSError as e:
        pytest.skip(f"oracle OpenMP build unavailable: {e}")
    wins = synth.windows(64)
    order = sorted(range(len(wins)), key=lambda k: wins[k][0].size)
    pick = [order[-1], order[len(order) // 2]]
    specs = {k: wins[k] for k in pick}
    assert wins[pick[0]][0].shape == (16, 64, 64, 64)
    p = _lib.Params.defaults()
    p.precision = 1
    res = _batched(specs, p)
    P = oracle_params(p)
    for k, (img, seeds, nsteps) in specs.items():
        assert nsteps == 30
        ref, info = O.segment(img.astype(np.float64), seeds, P, nsteps=nsteps, omp=True)
        assert info["status"] == O.OR_OK
        _check(k, res[k], ref, img.shape)
