"""Pins of the oracle's whole time step and pipeline.

- Theorem of Section 3.3 (discrete min-max principle): every solved u^n lies
  between the min and max of u^{resc,n-1} over the grid and its zero
  Dirichlet boundary.
- Rescaling keeps u in [0, 1] inside every ball after every step (Remark,
  Eq. 841).
- Mirror symmetry: an image and seeds symmetric under x -> N1-1-x give a
  symmetric u (a wrong neighbour offset or face index breaks it).
- A constant image gives G = 1 (g(0) = 1), so the run equals the G = 1 run.
"""
import numpy as np

import oracle as O


def _ball_image(shape, c, r, rng, noise=0.05):
    n4, n3, n2, n1 = shape
    l, k, j, i = np.meshgrid(*(np.arange(s) for s in shape), indexing="ij")
    d2 = (i - c[0]) ** 2 + (j - c[1]) ** 2 + (k - c[2]) ** 2
    img = np.where(d2 <= r * r, 1.0, 0.0)
    return img + noise * rng.normal(size=shape)


def test_min_max_principle_and_rescale_range_each_step():
    rng = np.random.default_rng(0)
    shape = (4, 8, 10, 12)
    I0 = _ball_image(shape, (6, 5, 4), 3, rng)
    seeds = [(6, 5, 4, 0), (5, 5, 4, 2)]
    P = O.OracleParams(r_ball=4.0, R_init=4.0)
    Ith = O.threshold(I0, seeds, P.r_ball, P.lambda_th)
    Is0, _ = O.presmooth(I0, P.h, P.sigma_t)
    IsT, _ = O.presmooth(Ith, P.h, P.sigma_t)
    G = O.face_G(Is0, IsT, P.h, P.K, P.delta, P.vartheta)
    u = O.rescale(O.init_u(shape, seeds, P.R_init, P.v_init), seeds, P.r_ball)
    own = O.owner(shape, seeds, P.r_ball)
    for _ in range(3):
        diag, off = O.assemble(u, G, P.h, P.tau, P.eps)
        un, info = O.solve(diag, off, u, omega=P.omega, tol=1e-12)
        assert info["status"] == O.OR_OK
        assert min(0.0, u.min()) - 1e-12 <= un.min() and un.max() <= max(0.0, u.max()) + 1e-12
        u = O.rescale(un, seeds, P.r_ball)
        assert u[own >= 0].min() >= -1e-15 and u[own >= 0].max() <= 1 + 1e-15
    # the pipeline entry point runs the same sequence
    useg, info = O.segment(I0, seeds, P, nsteps=3)
    assert info["status"] == O.OR_OK
    np.testing.assert_allclose(useg, u, atol=1e-10)


def test_mirror_symmetry():
    rng = np.random.default_rng(1)
    shape = (3, 6, 7, 12)
    half = rng.uniform(size=(3, 6, 7, 6))
    I0 = np.concatenate([half, half[..., ::-1]], axis=-1)
    seeds = [(5.5, 3, 3, 0)]
    P = O.OracleParams(r_ball=3.0, R_init=4.0, tol=1e-13)
    u, info = O.segment(I0, seeds, P, nsteps=2)
    np.testing.assert_allclose(u, u[..., ::-1], atol=1e-10)
    assert np.abs(u - u[..., ::-1]).max() < 1e-10


def test_constant_image_equals_unit_G_run():
    shape = (3, 6, 6, 6)
    I0 = np.full(shape, 0.25)
    seeds = [(3, 3, 3, 1)]
    P = O.OracleParams(r_ball=3.0, R_init=3.0)
    u, _ = O.segment(I0, seeds, P, nsteps=2)
    v = O.rescale(O.init_u(shape, seeds, P.R_init, P.v_init), seeds, P.r_ball)
    for _ in range(2):
        diag, off = O.assemble(v, np.ones(shape + (8,)), P.h, P.tau, P.eps)
        v, _ = O.solve(diag, off, v, omega=P.omega, tol=1e-12)
        v = O.rescale(v, seeds, P.r_ball)
    np.testing.assert_allclose(u, v, atol=1e-10)
