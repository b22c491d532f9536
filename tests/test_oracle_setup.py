"""Pins of the oracle's set-up stages: thresholding and ball owners
(Section 3.1), presmoothing (the linear heat equation, Section 3.1), the face
edge coefficients (Eq. 10th with g of Eq. eg1), the initial condition
(Eq. initialcond) and the local rescaling (Remark, Eq. 841)."""
import numpy as np
import pytest

import oracle as O

# --------------------------------------------------------------------------
# owners and thresholding
# --------------------------------------------------------------------------


def test_ball_membership_inclusive_and_frame_local():
    shape = (2, 11, 11, 11)
    own = O.owner(shape, [(5, 5, 5, 0)], r=5.0)
    assert own[0, 5, 5, 10] == 0          # distance exactly 5 (inclusive)
    assert own[0, 5, 9, 8] == 0           # (3, 4, 0): distance 5
    assert own[0, 5, 9, 9] == -1          # (4, 4, 0): distance 5.66
    assert (own[1] == -1).all()           # balls live in their own frame
    assert (own[0] == 0).sum() == 515     # lattice points in a closed ball of radius 5


def test_owner_is_nearest_seed_ties_to_lowest_index():
    shape = (1, 1, 1, 9)
    own = O.owner(shape, [(2, 0, 0, 0), (6, 0, 0, 0)], r=10.0)
    assert own.reshape(-1).tolist() == [0, 0, 0, 0, 0, 1, 1, 1, 1]  # voxel 4: tie -> 0


def test_threshold_two_level_image_is_unchanged():
    """Section 4 (third experiment): when the image has two levels, the
    thresholded image equals the original one."""
    shape = (1, 15, 15, 15)
    zz, yy, xx = np.meshgrid(np.arange(15), np.arange(15), np.arange(15), indexing="ij")
    inside = (xx - 7) ** 2 + (yy - 7) ** 2 + (zz - 7) ** 2 <= 9
    I0 = np.where(inside, 0.9, 0.2)[None]
    ITH = O.threshold(I0, [(7, 7, 7, 0)], r=6.0, lam=0.87)
    np.testing.assert_array_equal(ITH, I0)


def test_threshold_three_level_hand_example():
    """Three levels 0.2 / 0.5 / 0.9 inside the ball: alpha = 0.2, beta = 0.9,
    TH = 0.87*0.2 + 0.13*0.9 = 0.291, so 0.5 and 0.9 map to 0.9 and 0.2 stays;
    voxels outside the ball keep their value."""
    shape = (1, 1, 1, 12)
    I0 = np.array([0.5, 0.2, 0.5, 0.9, 0.2, 0.5, 0.9, 0.5, 0.2, 0.5, 0.9, 0.7])[None, None, None]
    ITH = O.threshold(I0, [(5, 0, 0, 0)], r=4.0, lam=0.87)
    expect = np.array([0.5, 0.2, 0.9, 0.9, 0.2, 0.9, 0.9, 0.9, 0.2, 0.9, 0.9, 0.7])
    np.testing.assert_allclose(ITH.reshape(-1), expect, rtol=0, atol=0)


def test_threshold_overlapping_balls_follow_owner():
    shape = (1, 1, 1, 10)
    I0 = np.array([0.1, 0.4, 0.6, 0.3, 0.5, 0.56, 0.8, 0.2, 0.9, 0.3])[None, None, None]
    seeds = [(2, 0, 0, 0), (7, 0, 0, 0)]
    ITH = O.threshold(I0, seeds, r=3.0, lam=0.5).reshape(-1)
    # seed 0 ball = voxels 0..5: alpha 0.1, beta 0.6, TH 0.35
    # seed 1 ball = voxels 4..9: alpha 0.2, beta 0.9, TH 0.55 (0.56 lies above it)
    # owners: 0..4 -> seed 0 (voxel 4 is nearer to seed 0), 5..9 -> seed 1
    expect = [0.1, 0.6, 0.6, 0.1, 0.6, 0.9, 0.9, 0.2, 0.9, 0.2]
    np.testing.assert_allclose(ITH, expect, rtol=0, atol=0)


# --------------------------------------------------------------------------
# presmoothing
# --------------------------------------------------------------------------


@pytest.mark.parametrize("k", [(1, 0, 2, 1), (0, 3, 1, 2)])
def test_presmooth_neumann_cosine_eigenmode(k):
    """cos(pi k_d (i_d + 1/2)/N_d) is an eigenvector of the path Laplacian with
    zero-Neumann ends (eigenvalue 2(1 - cos(pi k_d/N_d))), so one implicit step
    divides the mode by 1 + sum_d sigma_t/h_d^2 * 2(1 - cos(pi k_d/N_d))."""
    shape = (5, 6, 4, 7)
    n = [shape[3], shape[2], shape[1], shape[0]]
    h = (0.01, 0.02, 0.01, 0.03)
    sigma_t = 0.01**2 / 8
    ax = [np.cos(np.pi * k[d] * (np.arange(n[d]) + 0.5) / n[d]) for d in range(4)]
    mode = np.einsum("l,k,j,i->lkji", ax[3], ax[2], ax[1], ax[0])
    out, info = O.presmooth(mode, h, sigma_t, tol=1e-14)
    lam = 1.0 + sum(sigma_t / h[d] ** 2 * 2 * (1 - np.cos(np.pi * k[d] / n[d])) for d in range(4))
    np.testing.assert_allclose(out, mode / lam, atol=1e-12)


def test_presmooth_conserves_mean_and_constants():
    rng = np.random.default_rng(3)
    I = rng.uniform(size=(4, 5, 6, 7))
    out, _ = O.presmooth(I, 0.01, 0.01**2 / 8, tol=1e-14)
    np.testing.assert_allclose(out.mean(), I.mean(), rtol=1e-12)
    assert out.std() < I.std()
    c = np.full((3, 3, 3, 3), 0.7)
    outc, _ = O.presmooth(c, 0.01, 0.01**2 / 8)
    np.testing.assert_allclose(outc, c, rtol=1e-14)


# --------------------------------------------------------------------------
# face edge coefficients
# --------------------------------------------------------------------------


def test_constant_image_gives_unit_G():
    """g(0) = 1 (Eq. eg1): a constant image has zero gradient on every face,
    including the boundary faces (Neumann ghosts repeat the edge)."""
    I = np.full((3, 4, 5, 6), 0.4)
    G = O.face_G(I, I, 0.01, K=3.0, delta=0.5, vartheta=0.5)
    assert (G == 1.0).all()


def test_ramp_image_closed_form():
    """I = a.x on voxel centres: every interior face sees |grad I| = |a|, so
    G = 1/(1 + K ((delta + vartheta)|a|)^2) when both images are the ramp."""
    shape = (5, 5, 6, 7)
    h = 0.01
    a = np.array([0.3, -0.2, 0.1, 0.25])
    n4, n3, n2, n1 = shape
    l, k, j, i = np.meshgrid(*(np.arange(s) for s in shape), indexing="ij")
    I = a[0] * i * h + a[1] * j * h + a[2] * k * h + a[3] * l * h
    K, dl, vt = 2.0, 0.7, 0.3
    G = O.face_G(I, I, h, K, dl, vt)
    expect = 1.0 / (1.0 + K * ((dl + vt) * np.linalg.norm(a)) ** 2)
    np.testing.assert_allclose(G[1:-1, 1:-1, 1:-1, 1:-1], expect, rtol=1e-12)


def test_delta_vartheta_equivalence_when_images_agree():
    """Section 4: (delta, vartheta) = (1,0), (0,1), (0.5,0.5) give the same
    result when the thresholded and original images coincide."""
    rng = np.random.default_rng(9)
    I = rng.uniform(size=(3, 4, 5, 6))
    G10 = O.face_G(I, I, 0.01, 1.0, 1.0, 0.0)
    G01 = O.face_G(I, I, 0.01, 1.0, 0.0, 1.0)
    G55 = O.face_G(I, I, 0.01, 1.0, 0.5, 0.5)
    np.testing.assert_allclose(G10, G01, rtol=1e-15)
    np.testing.assert_allclose(G10, G55, rtol=1e-14)
    assert (G10 > 0).all() and (G10 <= 1).all()


# --------------------------------------------------------------------------
# initial condition and rescaling
# --------------------------------------------------------------------------


def test_init_u_closed_form():
    shape = (2, 1, 1, 20)
    u = O.init_u(shape, [(3, 0, 0, 0)], R=12.0, v=1.0).reshape(2, -1)
    d = np.abs(np.arange(20) - 3.0)
    expect = np.where(d <= 12, 1.0 / (d + 1.0) - 1.0 / 13.0, 0.0)
    np.testing.assert_allclose(u[0], expect, rtol=1e-15)
    assert u[0, 15] == 0.0 and (u[1] == 0).all()   # d = 12 gives exactly zero
    # overlapping peaks take the maximum
    u2 = O.init_u((1, 1, 1, 10), [(2, 0, 0, 0), (6, 0, 0, 0)], R=5.0, v=1.0).reshape(-1)
    assert u2[2] == pytest.approx(1 - 1 / 6) and u2[6] == pytest.approx(1 - 1 / 6)
    assert u2[4] == pytest.approx(1 / 3 - 1 / 6)


def test_rescale_maps_each_ball_onto_unit_interval():
    rng = np.random.default_rng(5)
    shape = (3, 9, 10, 11)
    u = rng.uniform(0.2, 0.7, size=shape)
    seeds = [(3, 4, 4, 0), (8, 5, 4, 0), (5, 5, 5, 2)]
    own = O.owner(shape, seeds, r=3.0)
    out = O.rescale(u, seeds, r=3.0)
    np.testing.assert_array_equal(out[own < 0], u[own < 0])
    for m in range(3):
        sel = own == m
        assert out[sel].max() <= 1.0 + 1e-15 and out[sel].min() >= -1e-15
        # affine on the owned set: correlation 1 with the input
        assert np.corrcoef(out[sel], u[sel])[0, 1] > 1 - 1e-12
    # a ball that owns its own min and max reaches 0 and 1 exactly
    sel = own == 2
    assert out[sel].min() == 0.0 and out[sel].max() == 1.0


def test_threshold_tie_goes_to_beta():
    """Section 3.1 sends I0 >= TH to beta: with alpha = 0, beta = 1 and
    lambda = 1/2, TH is exactly 0.5 and a voxel of value 0.5 maps to 1."""
    I0 = np.array([0.0, 0.5, 1.0, 0.25])[None, None, None]
    ITH = O.threshold(I0, [(1, 0, 0, 0)], r=2.0, lam=0.5).reshape(-1)
    np.testing.assert_array_equal(ITH, [0.0, 1.0, 1.0, 0.0])


# --------------------------------------------------------------------------
# overlapping balls: statistics over the whole ball, applied to owned voxels
# --------------------------------------------------------------------------
#
# Section 3.1 defines alpha_m, beta_m as the min and max of I0 over the whole
# ball B(c_m, r), and the Remark on local rescaling (Section 3.2) defines
# mu_m, xi_m over the whole ball too.  Where balls overlap, a voxel follows
# its nearest seed, but the statistics of a ball still include the voxels of
# the ball that another seed owns.  In the two cases below the extremes of
# each ball sit on voxels owned by the other seed, so statistics taken over
# the owned voxels only give different values.  Geometry: seeds at x = 2 and
# x = 7 on a line of 10 voxels, r = 3; ball 0 = voxels 0..5, ball 1 = voxels
# 4..9; voxel 4 is nearer seed 0, voxel 5 nearer seed 1.


def test_threshold_overlap_uses_whole_ball_statistics():
    I0 = np.array([0.02, 0.4, 0.5, 0.35, 0.05, 0.95, 0.6, 0.7, 0.5, 1.0])[None, None, None]
    seeds = [(2, 0, 0, 0), (7, 0, 0, 0)]
    own = O.owner(I0.shape, seeds, r=3.0).reshape(-1)
    assert own.tolist() == [0, 0, 0, 0, 0, 1, 1, 1, 1, 1]
    ITH = O.threshold(I0, seeds, r=3.0, lam=0.5).reshape(-1)
    # ball 0: alpha 0.02 (voxel 0), beta 0.95 (voxel 5, owned by seed 1):
    #   TH = 0.485, so 0.5 -> 0.95 and 0.4, 0.35, 0.05 -> 0.02
    # ball 1: alpha 0.05 (voxel 4, owned by seed 0), beta 1.0 (voxel 9):
    #   TH = 0.525, so 0.5 -> 0.05 and 0.95, 0.6, 0.7, 1.0 -> 1.0
    expect = [0.02, 0.02, 0.95, 0.02, 0.02, 1.0, 1.0, 1.0, 0.05, 1.0]
    np.testing.assert_array_equal(ITH, expect)
    # statistics over the owned voxels would give ball 0 beta = 0.5 (TH 0.26)
    # and ball 1 alpha = 0.5: voxel 1 would map to 0.5 and voxel 8 to 0.5
    assert ITH[1] != 0.5 and ITH[8] != 0.5


def test_rescale_overlap_uses_whole_ball_statistics():
    u = np.array([0.05, 0.4, 0.5, 0.35, 0.1, 0.9, 0.6, 0.7, 0.5, 0.8])[None, None, None]
    seeds = [(2, 0, 0, 0), (7, 0, 0, 0)]
    out = O.rescale(u, seeds, r=3.0).reshape(-1)
    x = u.reshape(-1)
    # ball 0: mu 0.05 (voxel 0), xi 0.9 (voxel 5, owned by seed 1)
    # ball 1: mu 0.1 (voxel 4, owned by seed 0), xi 0.9 (voxel 5)
    expect = np.concatenate([(x[:5] - 0.05) / 0.85, (x[5:] - 0.1) / 0.8])
    np.testing.assert_allclose(out, expect, rtol=1e-15, atol=0)
    # so seed 0's owned voxels do not reach 1, and seed 1's do not reach 0
    assert out[:5].max() < 0.6 and out[5:].min() > 0.4
