"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Bars (from the arithmetic of each stage):
- integer and copy work is bit-exact: ball owners, the thresholded image;
- the FP32 presmoothing solves stop at ||r|| <= 1e-6 ||b|| (the oracle at
  1e-12): |diff| <= 2e-5 max|I|;
- face coefficients G are FP32 functions of the presmoothed images:
  |diff| <= 1e-3 (absolute; G in (0, 1]) -- dominated by the 1e-5 image
  differences amplified by K|grad I|/h;
- u after the stated steps: |diff| <= 1e-4 max|u_oracle| per voxel, and
  identical labels (u >= 0.5) outside a one-voxel band of the oracle's level set.
"""
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


def _small_case():
    # odd sizes: ragged rows (n1 odd), several 32-slot chunks, 8-row blocks with a tail
    c = synth.small_nuclei(seed=7, n=(69, 21, 13, 5), count=5, nsteps=3)
    seeds = c.seeds.copy()
    # seeds in several frames, one near a corner, overlapping balls
    extra = np.array([[2, 3, 1, 2], [60, 17, 11, 4], [30, 10, 6, 1], [33, 11, 6, 1]], float)
    return c.image, np.concatenate([seeds, extra]), c.nsteps


@pytest.fixture(scope="module")
def small():
    image, seeds, nsteps = _small_case()
    p = _lib.Params.defaults()
    p.r_ball = 6.0
    p.R_init = 6.0
    gpu = gpu_run(image, seeds, nsteps, p, fields=("owner", "ITH", "Isig0", "IsigTH", "G", "u"))
    P = oracle_params(p)
    img = image.astype(np.float64)
    ref = {"owner": O.owner(image.shape, seeds, P.r_ball),
           "ITH": O.threshold(img, seeds, P.r_ball, P.lambda_th)}
    ref["Isig0"], _ = O.presmooth(img, P.h, P.sigma_t)
    ref["IsigTH"], _ = O.presmooth(ref["ITH"], P.h, P.sigma_t)
    ref["G"] = O.face_G(ref["Isig0"], ref["IsigTH"], P.h, P.K, P.delta, P.vartheta)
    ref["u0"] = O.rescale(O.init_u(image.shape, seeds, P.R_init, P.v_init), seeds, P.r_ball)
    ref["u"], ref["info"] = O.segment(img, seeds, P, nsteps=nsteps)
    return gpu, ref, p


def test_owner_bit_exact(small):
    gpu, ref, _ = small
    np.testing.assert_array_equal(gpu["f_owner"].astype(np.int64), ref["owner"].astype(np.int64))
    assert (ref["owner"] >= 0).sum() > 1000


def test_threshold_bit_exact(small):
    gpu, ref, _ = small
    np.testing.assert_array_equal(gpu["f_ITH"], ref["ITH"].astype(np.float32))


def test_presmoothing(small):
    gpu, ref, _ = small
    for name in ("Isig0", "IsigTH"):
        scale = np.abs(ref[name]).max()
        assert np.abs(gpu["f_" + name] - ref[name]).max() <= 2e-5 * scale, name


def test_face_coefficients(small):
    gpu, ref, _ = small
    d = np.abs(gpu["f_G"] - ref["G"])
    assert d.max() <= 1e-3, d.max()
    assert (gpu["f_G"] > 0).all() and (gpu["f_G"] <= 1).all()


def test_face_coefficients_on_identical_images(small):
    """G from the GPU's own presmoothed images, oracle against GPU: the only
    difference left is FP32 arithmetic.  The diamond differences of FP32
    images carry about 1e-5 of absolute error in |grad I| (h = 0.01), and
    |dG/ds| s / G <= 2 sqrt(K) s/(1 + K s^2) <= 1, so 2e-5 relative bounds it;
    a coefficient wrong by 100 % at the edges, where G is about 1e-3, fails."""
    gpu, _, p = small
    P = oracle_params(p)
    G = O.face_G(gpu["f_Isig0"].astype(np.float64), gpu["f_IsigTH"].astype(np.float64), P.h,
                 P.K, P.delta, P.vartheta)
    rel = np.abs(gpu["f_G"] - G) / G
    assert rel.max() <= 2e-5, rel.max()
    assert G.min() < 0.05   # the case has real edges


def test_initial_condition(small):
    gpu, ref, _ = small
    np.testing.assert_allclose(gpu["f_u"], ref["u0"], atol=1e-6)


def test_pipeline_small(small):
    gpu, ref, p = small
    u, r = gpu["u"], ref["u"]
    err = np.abs(u - r).max()
    assert err <= REL_TOL * np.abs(r).max(), err
    assert label_mismatch_outside_band(u, r) == 0
    info = gpu["info"]
    assert info["steps_done"] == 3 and info["status"] == 0
    assert info["res_rel"] <= p.tol


@pytest.fixture(scope="module")
def tiny():
    c = synth.tiny()
    p = _lib.Params.defaults()
    gpu = gpu_run(c.image, c.seeds, c.nsteps, p)
    ref_u, ref_info = O.segment(c.image.astype(np.float64), c.seeds, oracle_params(p),
                                nsteps=c.nsteps)
    return gpu, ref_u, ref_info, p


def test_pipeline_tiny_config(tiny):
    """32x32x32x16 moving ball with a wedge gap, 10 steps."""
    gpu, r, ref_info, p = tiny
    u = gpu["u"]
    err = np.abs(u - r).max()
    assert err <= REL_TOL * np.abs(r).max(), err
    assert label_mismatch_outside_band(u, r) == 0
    assert gpu["info"]["steps_done"] == 10
    # the segmentation is not trivial
    assert (r >= 0.5).sum() > 100


def test_solve_alone_from_given_u():
    """The step system alone: set u, one solve (no rescale), compare with the
    oracle's assembly + SOR from the same u and the oracle's own G."""
    rng = np.random.default_rng(3)
    c = synth.small_nuclei(seed=11, n=(40, 24, 18, 7), count=3, nsteps=1)
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 6.0
    P = oracle_params(p)
    u0 = np.clip(rng.normal(0.4, 0.2, size=c.image.shape), 0, 1).astype(np.float32)
    dims = c.dims
    with _lib.Seg4D(dims, params=p) as s:
        s.set_image(c.image)
        s.set_seeds(c.seeds)
        s.setup()
        s.set_u(u0)
        info = s.solve()
        ug = s.read_u()
        off_g = s.read_field("off")
        diag_g = s.read_field("diag")
        G_g = s.read_field("G")
    img = c.image.astype(np.float64)
    ITH = O.threshold(img, c.seeds, P.r_ball, P.lambda_th)
    G = O.face_G(O.presmooth(img, P.h, P.sigma_t)[0], O.presmooth(ITH, P.h, P.sigma_t)[0], P.h,
                 P.K, P.delta, P.vartheta)
    diag, off = O.assemble(u0.astype(np.float64), G, P.h, P.tau, P.eps)
    ur, _ = O.solve(diag, off, u0.astype(np.float64), omega=1.8, tol=1e-12)
    # identical inputs (the GPU's own G and the same u): FP32 arithmetic only
    diag_i, off_i = O.assemble(u0.astype(np.float64), G_g.astype(np.float64), P.h, P.tau, P.eps)
    np.testing.assert_allclose(diag_g, diag_i, rtol=1e-5)
    inner = off_g != 0
    np.testing.assert_allclose(off_g[inner], off_i[inner], rtol=1e-5)
    np.testing.assert_allclose(diag_g, diag, rtol=2e-3)
    # interior faces only (the ABI reports faces to the boundary as 0)
    interior = off_g != 0
    np.testing.assert_allclose(off_g[interior], off[interior], rtol=2e-3, atol=1e-3)
    assert np.abs(ug - ur).max() <= REL_TOL * np.abs(ur).max()
    assert info["res_rel"] <= p.tol


@pytest.mark.parametrize("dims", [(1, 1, 1, 1), (1, 5, 3, 2), (7, 1, 1, 3), (2, 2, 2, 2),
                                  (33, 9, 1, 1)])
def test_degenerate_grids(dims):
    rng = np.random.default_rng(sum(dims))
    n1, n2, n3, n4 = dims
    img = rng.uniform(size=(n4, n3, n2, n1)).astype(np.float32)
    seeds = [((n1 - 1) / 2, (n2 - 1) / 2, (n3 - 1) / 2, 0)]
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 3.0
    gpu = gpu_run(img, seeds, 2, p)
    r, _ = O.segment(img.astype(np.float64), seeds, oracle_params(p), nsteps=2)
    assert np.abs(gpu["u"] - r).max() <= REL_TOL * max(np.abs(r).max(), 1e-30)


def test_no_seeds_keeps_zero():
    img = np.random.default_rng(0).uniform(size=(3, 4, 5, 6)).astype(np.float32)
    gpu = gpu_run(img, np.zeros((0, 4)), 2)
    assert (gpu["u"] == 0).all()


def test_errors_are_reported():
    with _lib.Seg4D((8, 8, 8, 2)) as s:
        with pytest.raises(_lib.Seg4DError) as e:
            s.step(1)
        assert e.value.status == _lib.ERR_STATE
        with pytest.raises(_lib.Seg4DError) as e:
            s.set_params(omega=2.5)
        assert e.value.status == _lib.ERR_INVALID
        s.set_params(omega=1.8)
        bad = np.zeros((2, 8, 8, 8), np.float32)
        bad[0, 0, 0, 0] = np.nan
        with pytest.raises(_lib.Seg4DError):
            s.set_image(bad)
        with pytest.raises(ValueError):
            s.set_image(np.zeros(10, np.float32))


def test_non_finite_image_is_refused_on_the_device():
    """The image is checked for NaN/Inf after the copy, for host and device
    input alike; a refused image leaves the handle without an image."""
    import torch
    c = synth.small_nuclei(seed=5, n=(24, 20, 12, 4), count=2, nsteps=1)
    with _lib.Seg4D(c.dims) as s:
        s.set_image(c.image)
        s.set_seeds(c.seeds)
        bad = c.image.copy()
        bad[1, 2, 3, 4] = np.inf
        with pytest.raises(_lib.Seg4DError) as e:
            s.set_image(bad)
        assert e.value.status == _lib.ERR_INVALID
        with pytest.raises(_lib.Seg4DError) as e:
            s.step(1)
        assert e.value.status == _lib.ERR_STATE
        bad_d = torch.from_numpy(c.image).cuda()
        bad_d[0, 0, 0, 0] = float("nan")
        with pytest.raises(_lib.Seg4DError) as e:
            s.set_image(bad_d)
        assert e.value.status == _lib.ERR_INVALID
        s.set_image(torch.from_numpy(c.image).cuda())
        assert s.step(1)["status"] == _lib.OK


def test_not_converged_is_reported_and_u_kept():
    c = synth.small_nuclei(seed=5, n=(24, 20, 12, 4), count=2, nsteps=1)
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 5.0
    with _lib.Seg4D(c.dims, params=p) as s:
        s.set_image(c.image)
        s.set_seeds(c.seeds)
        s.setup()
        s.set_params(max_iters=2, check_every=1, tol=1e-12)
        with pytest.raises(_lib.Seg4DError) as e:
            s.solve()
        assert e.value.status == _lib.ERR_NOT_CONVERGED
        info = s.solve(allow_not_converged=True)
        assert info["iters"] == 2 and info["status"] == _lib.ERR_NOT_CONVERGED
        assert np.isfinite(s.read_u()).all()


def test_checkpoint_resume_equals_uninterrupted():
    c = synth.small_nuclei(seed=9, n=(30, 22, 14, 5), count=3, nsteps=4)
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 6.0
    with _lib.Seg4D(c.dims, params=p) as s:
        s.set_image(c.image)
        s.set_seeds(c.seeds)
        s.step(4)
        u_all = s.read_u()
    with _lib.Seg4D(c.dims, params=p) as s:
        s.set_image(c.image)
        s.set_seeds(c.seeds)
        s.step(2)
        ck = s.read_u()
    with _lib.Seg4D(c.dims, params=p) as s:
        s.set_image(c.image)
        s.set_seeds(c.seeds)
        s.setup()
        s.set_u(ck)
        s.step(2)
        u_res = s.read_u()
    np.testing.assert_array_equal(u_res, u_all)


def test_device_pointers_roundtrip():
    import torch
    c = synth.small_nuclei(seed=3, n=(20, 16, 8, 3), count=2, nsteps=1)
    img_d = torch.from_numpy(c.image).cuda()
    out_d = torch.empty_like(img_d)
    with _lib.Seg4D(c.dims, stream=torch.cuda.current_stream()) as s:
        s.set_image(img_d)
        s.read_field("I0", out_d)
        torch.cuda.synchronize()
        assert torch.equal(out_d, img_d)
        s.set_seeds(c.seeds)
        s.set_params(r_ball=5.0, R_init=5.0)
        s.step(1)
        u_host = s.read_u()
        s.read_u(out_d)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out_d.cpu().numpy(), u_host)


# ------------------------------------------------------- ragged row layouts

SWEEP_DIMS = [(69, 21, 13, 5), (40, 17, 6, 1), (31, 9, 5, 2), (64, 24, 12, 7), (3, 2, 1, 4),
              (201, 7, 5, 3), (130, 9, 4, 2), (1100, 5, 3, 2)]


@pytest.mark.parametrize("dims", SWEEP_DIMS)
@pytest.mark.parametrize("lean", [False, True])
def test_ragged_layouts_match_oracle(dims, lean):
    """Rows of one to nine warps' 64 slots with ragged ends, odd y-blocks,
    n4 = 1 and 2, on the full handle (scaled sweeps) and the lean one
    (unscaled sweeps): two steps against the oracle, per-voxel bound; both
    ways of reading the black pass's weights give the same bits."""
    n1, n2, n3, n4 = dims
    image = synth.random_field(sum(dims), dims)
    seeds = [(n1 // 2, n2 // 2, n3 // 2, 0), (n1 // 3, n2 // 3, n3 // 3, n4 - 1)]
    out = {}
    for variant in (1, 2):
        p = _lib.Params.defaults()
        p.r_ball = p.R_init = 5.0
        p.sweep_variant = variant
        with _lib.Seg4D(dims, params=p, lean=lean) as s:
            s.set_image(image)
            s.set_seeds(seeds)
            info = s.step(2)
            out[variant] = (s.read_u(), info["sweeps_total"])
    # the black pass reading the weights by black end (1) or across the faces
    # (2) gives the same bits and the same sweep counts
    np.testing.assert_array_equal(out[1][0], out[2][0])
    assert out[1][1] == out[2][1]
    u = out[1][0]
    r, _ = O.segment(image.astype(np.float64), seeds, oracle_params(p), nsteps=2)
    assert np.abs(u - r).max() <= REL_TOL * max(np.abs(r).max(), 1e-30)
