"""Pins of the oracle's step system and SOR solver.

- Dense LU on grids of at most 4^4 voxels: the matrix of Eq. new is built in
  the test from the neighbour relation alone (A[v,v] = diag, A[v,nb] = -off)
  and solved by LAPACK; the oracle's SOR must agree to 1e-10.
- Theorem of Section 3.3: the matrix is a strictly diagonally dominant
  M-matrix (row sums >= 1 over the grid), so ||A^-1||_inf <= 1 and the solution
  obeys the discrete min-max principle, with the zero Dirichlet value counted
  among the values of the previous step.
- The solution does not depend on the relaxation parameter.
"""
import numpy as np
import pytest

import oracle as O

H = 0.01
TAU = 0.01


def _neighbour(shape, v, f):
    n4, n3, n2, n1 = shape
    l, k, j, i = np.unravel_index(v, shape)
    c = [i, j, k, l]
    n = [n1, n2, n3, n4]
    d = f // 2
    c[d] += 1 if f % 2 else -1
    if c[d] < 0 or c[d] >= n[d]:
        return None
    return np.ravel_multi_index((c[3], c[2], c[1], c[0]), shape)


def _dense(diag, off):
    shape = diag.shape
    N = diag.size
    A = np.zeros((N, N))
    d = diag.reshape(-1)
    o = off.reshape(N, 8)
    for v in range(N):
        A[v, v] = d[v]
        for f in range(8):
            nb = _neighbour(shape, v, f)
            if nb is not None:
                A[v, nb] -= o[v, f]
    return A


def sym_G(shape, rng, lo=0.05, hi=1.0):
    """Random face coefficients that agree from both sides of every face, as
    G of Eq. 10th does (the face value does not depend on the side)."""
    G = rng.uniform(lo, hi, size=shape + (8,))
    # array axes (l, k, j, i) hold physical axes d = 3, 2, 1, 0
    for d in range(4):
        ax = 3 - d
        plus = np.take(G[..., 2 * d + 1], np.arange(shape[ax] - 1), axis=ax)
        idx = [slice(None)] * 4
        idx[ax] = slice(1, None)
        G[tuple(idx) + (2 * d,)] = plus
    return G


def _case(shape, seed, eps=1.0):
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, size=shape)
    G = sym_G(shape, rng)
    diag, off = O.assemble(u, G, H, TAU, eps)
    return u, G, diag, off


@pytest.mark.parametrize("shape,seed", [((2, 3, 2, 3), 1), ((4, 4, 4, 4), 2), ((1, 2, 3, 5), 3),
                                        ((3, 1, 4, 2), 4)])
def test_sor_matches_dense_lu(shape, seed):
    u, G, diag, off = _case(shape, seed)
    A = _dense(diag, off)
    b = u.reshape(-1)
    x_lu = np.linalg.solve(A, b)
    x_sor, info = O.solve(diag, off, u, omega=1.6, tol=1e-13)
    assert info["status"] == O.OR_OK
    np.testing.assert_allclose(x_sor.reshape(-1), x_lu, rtol=0, atol=1e-10 * np.abs(x_lu).max())


def test_m_matrix_row_sums_and_inverse_bound():
    u, G, diag, off = _case((3, 3, 4, 4), 7)
    A = _dense(diag, off)
    offd = A - np.diag(np.diag(A))
    assert (offd <= 0).all()
    row = np.diag(A) - np.abs(offd).sum(axis=1)
    assert (row >= 1.0 - 1e-12).all()
    # interior rows (all 8 neighbours inside) have row sum exactly 1
    n4, n3, n2, n1 = u.shape
    interior = np.zeros(u.shape, bool)
    interior[1:-1, 1:-1, 1:-1, 1:-1] = True
    np.testing.assert_allclose(row[interior.reshape(-1)], 1.0, atol=1e-9)
    Ainv = np.linalg.inv(A)
    assert np.abs(Ainv).sum(axis=1).max() <= 1.0 + 1e-10


def test_min_max_principle_and_residual_bound():
    rng = np.random.default_rng(11)
    shape = (3, 4, 5, 6)
    u, G, diag, off = _case(shape, 11)
    b = rng.uniform(0.2, 0.9, size=shape)
    x, info = O.solve(diag, off, b, omega=1.7, tol=1e-13)
    # the ghost value u^D = 0 takes part in the bound (the proof's extremal row
    # argument needs every neighbour, ghosts included, inside [min, max])
    assert min(0.0, b.min()) - 1e-12 <= x.min() and x.max() <= max(0.0, b.max()) + 1e-12
    assert x.max() <= b.max() + 1e-12
    # a loosely converged iterate: the error is bounded by the residual (||A^-1|| <= 1)
    x_loose, _ = O.solve(diag, off, b, omega=1.0, tol=1e-3, check_every=1)
    r = O.residual(diag, off, b, x_loose)
    assert np.abs(x_loose - x).max() <= np.abs(r).max() + 1e-12


def test_solution_independent_of_omega():
    u, G, diag, off = _case((2, 4, 4, 6), 5)
    ref, _ = O.solve(diag, off, u, omega=1.0, tol=1e-13)
    for w in (0.7, 1.5, 1.9):
        x, info = O.solve(diag, off, u, omega=w, tol=1e-12)
        assert info["status"] == O.OR_OK
        np.testing.assert_allclose(x, ref, atol=1e-11)


def test_sym_G_helper_is_face_symmetric():
    G = sym_G((2, 3, 4, 5), np.random.default_rng(0))
    np.testing.assert_array_equal(G[..., :-1, 1], G[..., 1:, 0])
    np.testing.assert_array_equal(G[:-1, ..., 7], G[1:, ..., 6])


@pytest.mark.parametrize("h", [(H,) * 4, (0.01, 0.02, 0.015, 0.05)])
def test_assembly_closed_form_for_constant_u(h):
    """Constant u inside the grid: interior faces carry zero gradient, so
    A_f = Abar = eps there and the coefficient of Eq. new1 reduces to
    tau m(e)/(m(V) m(sigma)) * G_f = tau/h_d^2 * G_f for a face on axis d."""
    shape = (4, 4, 4, 4)
    u = np.full(shape, 0.3)
    G = sym_G(shape, np.random.default_rng(3), 0.1, 1.0)
    eps = 0.5
    diag, off = O.assemble(u, G, h, TAU, eps)
    g2 = O.face_grad_sq(u, h)
    inner = (slice(1, -1),) * 4  # voxels whose whole 33-point stencil is inside
    assert np.all(g2[inner] == 0.0)
    assert np.all(g2[0, 0, 0, 0] > 0.0)  # boundary faces see the zero ghosts
    hd2 = np.array([h[f // 2] ** 2 for f in range(8)])
    np.testing.assert_allclose(off[inner], TAU / hd2 * G[inner], rtol=1e-14)
    np.testing.assert_allclose(diag[inner], 1.0 + (TAU / hd2 * G[inner]).sum(-1), rtol=1e-14)


def test_openmp_build_reaches_the_same_solution():
    """The OpenMP build (a timed CPU baseline: the paper's frame-split
    red-black sweeps) solves the same systems: the whole pipeline agrees with
    the plain build's to the 1e-12 solve, with similar sweep counts."""
    from paper_2111_11866_gb300 import synth
    O.build(omp=True)
    c = synth.small_nuclei(3, n=(24, 20, 10, 5), count=3, nsteps=2)
    P = O.OracleParams()
    img = c.image.astype(np.float64)
    u0, i0 = O.segment(img, c.seeds, P, nsteps=2)
    u1, i1 = O.segment(img, c.seeds, P, nsteps=2, omp=True)
    assert i0["status"] == i1["status"] == O.OR_OK
    assert np.abs(u1 - u0).max() <= 1e-9 * max(1.0, np.abs(u0).max())
    assert all(0.5 * a <= b <= 2 * a for a, b in zip(i0["iters"], i1["iters"]))
    assert O.threads(False) == 1 and O.threads(True) >= 1
