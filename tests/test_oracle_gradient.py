"""Pins of the reduced diamond-cell face gradient (Section 3.2).

For a quadratic u(x) = a + b.x + x^T C x sampled at voxel centres, the
diamond-cell formula gives the exact gradient at the face centre: the normal
difference is exact for quadratics along the face normal, the tangential
central difference of the diamond-point averages is exact for quadratics and
for the mixed x_d x_t terms.  So |grad^f u|^2 must equal |grad u(x_face)|^2 to
rounding, on every face whose 14-point stencil lies inside the grid.  A
dropped tangential term, a wrong 1/4 weight, a swapped h_d / h_t or a wrong
neighbour offset fails this test.
"""
import numpy as np
import pytest

import oracle as O


def _coords(shape, h):
    n4, n3, n2, n1 = shape
    idx = np.meshgrid(np.arange(n4), np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    # axis order of the arrays is (l, k, j, i); physical axis d = 0..3 is (i, j, k, l)
    return [idx[3] * h[0], idx[2] * h[1], idx[1] * h[2], idx[0] * h[3]]


@pytest.mark.parametrize("h", [(0.01,) * 4, (0.5, 0.25, 1.0, 2.0)])
def test_diamond_gradient_exact_on_quadratics(h):
    rng = np.random.default_rng(42)
    shape = (5, 6, 5, 7)
    X = _coords(shape, h)
    b = rng.normal(size=4)
    Cm = rng.normal(size=(4, 4))
    u = 0.3 + sum(b[d] * X[d] for d in range(4))
    u = u + sum(Cm[d, e] * X[d] * X[e] for d in range(4) for e in range(4))
    g2 = O.face_grad_sq(u, h, mode="replicate")
    S = Cm + Cm.T
    inner = (slice(1, -1),) * 4
    for f in range(8):
        d, side = f // 2, (1 if f % 2 else -1)
        xf = [X[e].copy() for e in range(4)]
        xf[d] = xf[d] + 0.5 * side * h[d]
        grad = [b[e] + sum(S[e, m] * xf[m] for m in range(4)) for e in range(4)]
        exact = sum(gc**2 for gc in grad)
        np.testing.assert_allclose(g2[..., f][inner], exact[inner], rtol=1e-9, atol=1e-9)


def test_face_value_same_from_both_sides():
    rng = np.random.default_rng(1)
    u = rng.uniform(size=(3, 4, 5, 6))
    g2 = O.face_grad_sq(u, 0.01)
    # +x face of voxel (i) equals -x face of voxel (i+1), etc. (up to the
    # summation order of the four-cell averages)
    eq = lambda a, b: np.testing.assert_allclose(a, b, rtol=1e-13)
    eq(g2[..., :-1, 1], g2[..., 1:, 0])
    eq(g2[..., :-1, :, 3], g2[..., 1:, :, 2])
    eq(g2[:, :-1, :, :, 5], g2[:, 1:, :, :, 4])
    eq(g2[:-1, :, :, :, 7], g2[1:, :, :, :, 6])


def test_dirichlet_ghosts_are_zero():
    """On a grid of one voxel, every face sees only zero ghosts except the
    voxel itself: the normal component is -u/h and each tangential component
    is (1/4)(0 + 0 - 0 - 0)/h = 0."""
    u = np.full((1, 1, 1, 1), 2.0)
    g2 = O.face_grad_sq(u, 0.5)
    np.testing.assert_allclose(g2[0, 0, 0, 0], (2.0 / 0.5) ** 2)
