"""Parity at the benchmark sizes, in the launch configuration bench.py times.

The FP64 oracle cannot solve a 33.5M- or 1.61G-voxel system, but it can
compute single rows of it.  For sampled voxels it rebuilds, from a crop of the
device's own presmoothed images and right-hand side b, the face edge
coefficients G and the row of the step matrix (Eq. new1), and evaluates that
row's residual on the GPU's solution.  Every row residual is bounded by the
2-norm of the residual vector the GPU reports (|r_v| <= ||r||_2), up to the
FP32 rounding of the GPU's coefficients.  Over the whole grid the discrete
min-max principle (Theorem of Section 3.3) must hold for the solution, up to
the same residual bound (||A^-1||_inf <= 1 for this M-matrix).
"""
import numpy as np
import pytest

import oracle as O
from paper_2111_11866_gb300 import _lib, synth

from gpu_common import oracle_params

pytestmark = pytest.mark.gpu

CROP = 3          # crop radius: the centre row needs b within 2 voxels, G within 2
ROW_REL = 1e-5    # slack for the FP32 coefficients, relative to the row's magnitude


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_11866_gb300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _samples(shape, seeds, count, rng):
    """Random voxels, voxels on every face of the grid, and seed centres."""
    n4, n3, n2, n1 = shape
    pts = [tuple(int(rng.integers(0, m)) for m in shape) for _ in range(count)]
    for ax in range(4):
        for side in (0, shape[ax] - 1):
            p = [int(rng.integers(0, m)) for m in shape]
            p[ax] = side
            pts.append(tuple(p))
    for x, y, z, f in seeds[: max(1, count // 20)]:
        pts.append((int(f), int(z), int(y), int(x)))
    return pts


def _row_residuals(pts, b, u, Is0, IsTH, p):
    """Oracle row residual b_v - (A u)_v and the row magnitude at each point."""
    P = oracle_params(p)
    shape = b.shape
    out = []
    for c in pts:
        lo = [max(0, c[a] - CROP) for a in range(4)]
        hi = [min(shape[a], c[a] + CROP + 1) for a in range(4)]
        sl = tuple(slice(lo[a], hi[a]) for a in range(4))
        G = O.face_G(Is0[sl], IsTH[sl], P.h, P.K, P.delta, P.vartheta)
        diag, off = O.assemble(b[sl], G, P.h, P.tau, P.eps)
        loc = tuple(c[a] - lo[a] for a in range(4))
        r = float(b[c]) - diag[loc] * float(u[c])
        mag = abs(diag[loc] * float(u[c])) + abs(float(b[c]))
        for f in range(8):
            d, side = f // 2, (1 if f % 2 else -1)
            ax = 3 - d
            nb = list(c)
            nb[ax] += side
            if 0 <= nb[ax] < shape[ax]:
                t = off[loc + (f,)] * float(u[tuple(nb)])
                r += t
                mag += abs(t)
        out.append((r, mag))
    return out


def _check_solve(seg, p, seeds, count, rng):
    b = seg.read_u()
    info = seg.solve()
    assert info["status"] == _lib.OK and info["res_rel"] <= p.tol, info
    u = seg.read_u()
    res = info["res_l2"]
    # min-max principle of the step system, the zero Dirichlet value included
    lo = min(0.0, float(b.min())) - res
    hi = max(0.0, float(b.max())) + res
    assert float(u.min()) >= lo - 1e-6 and float(u.max()) <= hi + 1e-6, (u.min(), u.max(), lo, hi)
    Is0 = seg.read_field("Isig0")
    IsTH = seg.read_field("IsigTH")
    pts = _samples(b.shape, seeds, count, rng)
    worst = 0.0
    for r, mag in _row_residuals(pts, b, u, Is0, IsTH, p):
        excess = abs(r) - (res + ROW_REL * mag)
        worst = max(worst, excess)
    assert worst <= 0.0, worst
    return info


def test_medium_workload_rows_and_min_max():
    """Medium 128x128x64 x 32 frames (33.5M voxels): the first step solve, then
    two more whole steps (each meets the stopping rule)."""
    c = synth.medium()
    p = _lib.Params.defaults()
    with _lib.Seg4D(c.dims, params=p) as seg:
        seg.set_image(c.image)
        seg.set_seeds(c.seeds)
        seg.setup()
        _check_solve(seg, p, c.seeds, 400, np.random.default_rng(21))
        for _ in range(2):
            info = seg.step(1)
            assert info["status"] == _lib.OK and info["res_rel"] <= p.tol, info
            assert 0.0 - 1e-6 <= info["umin"] and info["umax"] <= 1.0 + 1e-6, info


def test_large_workload_rows_and_min_max():
    """Large 512x512x128 x 48 frames (1.61G voxels, about 142 GB on the device),
    built on the device: the first step solve."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    dims = (512, 512, 128, 48)
    need = _lib.Seg4D.device_bytes(dims) + 24 * 2 ** 30
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of free device memory")
    img, seeds, _, _ = synth.large("cuda")
    p = _lib.Params.defaults()
    with _lib.Seg4D(dims, params=p) as seg:
        seg.set_image(img)
        del img
        torch.cuda.empty_cache()
        seg.set_seeds(seeds)
        seg.setup()
        _check_solve(seg, p, seeds, 300, np.random.default_rng(22))


def test_tiled_plane_order_reaches_every_plane():
    """A grid whose planes are large enough for the tiled plane order to
    group the 9 z-planes in tiles of 2 (a ragged last tile with a hole), with
    rows of 552 slots per colour (nine 64-slot chunks, the last one ragged):
    after the first step solve, oracle rows at sampled voxels of every (k, l)
    plane and at the grid faces, and the min-max bound over the whole grid.
    A plane that the sweeps, the coefficient pass or the defect pass skipped
    or visited twice fails the row check there."""
    dims = (1100, 600, 9, 2)
    n1, n2, n3, n4 = dims
    img = synth.random_field(31, dims, 0.0, 0.3)
    seeds = [(550, 300, 4, 0), (200, 100, 2, 1), (900, 500, 7, 1)]
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 6.0
    rng = np.random.default_rng(23)
    with _lib.Seg4D(dims, params=p) as seg:
        seg.set_image(img)
        seg.set_seeds(seeds)
        seg.setup()
        b = seg.read_u()
        info = seg.solve()
        assert info["status"] == _lib.OK and info["res_rel"] <= p.tol, info
        u = seg.read_u()
        res = info["res_l2"]
        lo = min(0.0, float(b.min())) - res
        hi = max(0.0, float(b.max())) + res
        assert float(u.min()) >= lo - 1e-6 and float(u.max()) <= hi + 1e-6
        Is0 = seg.read_field("Isig0")
        IsTH = seg.read_field("IsigTH")
    pts = _samples(b.shape, [], 40, rng)
    for l in range(n4):
        for k in range(n3):
            for _ in range(3):
                pts.append((l, k, int(rng.integers(0, n2)), int(rng.integers(0, n1))))
    worst = 0.0
    for r, mag in _row_residuals(pts, b, u, Is0, IsTH, p):
        worst = max(worst, abs(r) - (res + ROW_REL * mag))
    assert worst <= 0.0, worst
