"""Batched windows (seg4d_batch_*): each window runs the scheme of the
single-grid path; results match the FP64 oracle, do not depend on the other
windows in the batch (bit for bit), and admission follows the arena budget."""
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


def _window(seed, n, nsteps=3):
    c = synth.small_nuclei(seed=seed, n=n, count=2, nsteps=nsteps)
    return c.image, c.seeds, nsteps


def _params():
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 6.0
    return p


WINDOWS = [(101, (37, 29, 17, 5)), (102, (24, 24, 24, 4)), (103, (50, 21, 13, 6))]


def _run_batch(specs, params, arena=1 << 30, extra_rounds=0):
    out = {}
    with _lib.Batch(arena, 64, params=params) as b:
        ids = {}
        for key, (img, seeds, nsteps) in specs.items():
            ids[key] = b.add(img, seeds, nsteps)
            assert ids[key] is not None
        for _ in range(max(s[2] for s in specs.values()) + extra_rounds):
            b.advance()
        for key, wid in ids.items():
            out[key] = (b.read_u(wid), b.poll(wid))
    return out


def test_batch_windows_match_oracle():
    p = _params()
    specs = {k: _window(*k_n) for k, k_n in enumerate(WINDOWS)}
    res = _run_batch(specs, p)
    P = oracle_params(p)
    for key, (img, seeds, nsteps) in specs.items():
        u, info = res[key]
        assert info["state"] == "done" and info["steps_done"] == nsteps
        ref, _ = O.segment(img.astype(np.float64), seeds, P, nsteps=nsteps)
        err = np.abs(u - ref).max()
        assert err <= REL_TOL * np.abs(ref).max(), (key, err)
        assert label_mismatch_outside_band(u, ref) == 0


def test_batch_result_same_alone_and_in_mix():
    p = _params()
    specs = {k: _window(*k_n) for k, k_n in enumerate(WINDOWS)}
    mix = _run_batch(specs, p)
    for key in specs:
        alone = _run_batch({key: specs[key]}, p)
        np.testing.assert_array_equal(alone[key][0], mix[key][0])
        assert alone[key][1]["sweeps"] == mix[key][1]["sweeps"]


def test_batch_matches_single_grid_path():
    """Same scheme as seg4d_step, up to rounding (the single grid solves the
    symmetrically scaled form of the same system) and the stopping rule's
    check schedule."""
    p = _params()
    img, seeds, nsteps = _window(*WINDOWS[0])
    res = _run_batch({0: (img, seeds, nsteps)}, p)
    with _lib.Seg4D((img.shape[3], img.shape[2], img.shape[1], img.shape[0]), params=p) as s:
        s.set_image(img)
        s.set_seeds(seeds)
        s.step(nsteps)
        u1 = s.read_u()
    assert np.abs(res[0][0] - u1).max() <= REL_TOL * np.abs(u1).max()


def test_batch_admission_by_budget_and_reuse():
    p = _params()
    img, seeds, _ = _window(*WINDOWS[1])
    need = _lib.Batch.window_bytes((24, 24, 24, 4), len(seeds))
    with _lib.Batch(int(2.5 * need), 8, params=p) as b:
        a = b.add(img, seeds, 1)
        c = b.add(img, seeds, 1)
        assert a is not None and c is not None
        assert b.add(img, seeds, 1) is None          # refused: arena full
        b.advance()
        assert b.poll(a)["state"] == "done"
        b.remove(a)
        d = b.add(img, seeds, 1)                     # the space came back
        assert d is not None
        b.advance()
        np.testing.assert_array_equal(b.read_u(d), b.read_u(c))


def test_batch_window_joining_later_gets_same_result():
    """Continuous batching: a window admitted while others are mid-run gets
    the result it gets alone."""
    p = _params()
    specs = {k: _window(*k_n) for k, k_n in enumerate(WINDOWS)}
    with _lib.Batch(1 << 30, 16, params=p) as b:
        first = b.add(*specs[0])
        b.advance()
        b.advance()
        late = b.add(*specs[1])
        for _ in range(4):
            b.advance()
        assert b.poll(first)["state"] == "done" and b.poll(late)["state"] == "done"
        u_late = b.read_u(late)
    alone = _run_batch({1: specs[1]}, p)
    np.testing.assert_array_equal(u_late, alone[1][0])


def test_batch_device_input_and_errors():
    import torch
    p = _params()
    img, seeds, nsteps = _window(*WINDOWS[2])
    with _lib.Batch(1 << 28, 4, params=p) as b:
        wid = b.add(torch.from_numpy(img).cuda(), seeds, 1)
        with pytest.raises(_lib.Seg4DError) as e:
            b.read_u(wid)                             # set-up not run yet
        assert e.value.status == _lib.ERR_STATE
        b.advance()
        out = torch.empty(img.shape, dtype=torch.float32, device="cuda")
        b.read_u(wid, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), b.read_u(wid))
        with pytest.raises(_lib.Seg4DError):
            b.poll(12345)


def test_failed_window_is_reported_and_the_others_go_on():
    """A window whose residual is not finite (a NaN in its image) fails on the
    device's decision; the batch stays usable and every other window gets
    the result it gets alone."""
    p = _params()
    specs = {k: _window(*k_n) for k, k_n in enumerate(WINDOWS[:2])}
    bad = specs[1][0].copy()
    bad[1, 3, 4, 5] = np.nan
    mix = {0: specs[0], 1: (bad, specs[1][1], specs[1][2])}
    with _lib.Batch(1 << 30, 8, params=p) as b:
        ids = {k: b.add(*v) for k, v in mix.items()}
        for _ in range(3):
            b.advance()
        assert b.poll(ids[1])["state"] == "failed"
        assert b.poll(ids[0])["state"] == "done"
        u0 = b.read_u(ids[0])
    alone = _run_batch({0: specs[0]}, p)
    np.testing.assert_array_equal(u0, alone[0][0])


def test_max_iters_reached_fails_every_window():
    p = _params()
    p.max_iters = 4
    specs = {k: _window(*k_n) for k, k_n in enumerate(WINDOWS[:2])}
    with _lib.Batch(1 << 30, 8, params=p) as b:
        ids = {k: b.add(*v) for k, v in specs.items()}
        b.advance()
        b.advance()
        for wid in ids.values():
            assert b.poll(wid)["state"] == "failed"
