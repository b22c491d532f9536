"""The experimental order of convergence of Section 3.4 on the GPU.

G = 1 (delta = vartheta = 0), no rescaling, the exact solution
u = (|x|^2 - 1)/6 + t of the 4D level-set flow on [-1.25, 1.25]^4 as initial
condition and as Dirichlet data on the ghost cells (seg4d_set_dirichlet),
tau = h^2 and the eps = h reading of the table (the same reading the oracle's
pin uses).  At N = 10, 20, 40 the GPU's error must equal the FP64 oracle's up
to the FP32 solve.  At N = 80 and 160, past what the oracle runs in a test,
the orders are checked against the printed rows (see the tests for row 5).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2111_11866_gb300 import _lib

pytestmark = pytest.mark.gpu

L_HALF, T_END = 1.25, 0.0625
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eoc_table.txt")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2111_11866_gb300 import build
    build.build()
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _table():
    rows = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            n, h, steps, err, eoc = line.split()
            rows[int(n)] = (float(h), int(steps), float(err), None if eoc == "-" else float(eoc))
    return rows


def _exact(coords, t):
    s = sum(c * c for c in coords)
    return (s - 1.0) / 6.0 + t


def _ghosts(n, h, t, dev):
    """The 8 face slabs of the padded grid (seg4d_set_dirichlet's layout),
    built on the device: padded index a in 0..n+1 sits at x(a) = -L + (a - 1/2) h."""
    import torch
    x = -L_HALF + (torch.arange(n + 2, device=dev, dtype=torch.float64) - 0.5) * h
    out = []
    for d in range(4):
        for side in (0, n + 1):
            axes = [x[side:side + 1] if e == d else x for e in (3, 2, 1, 0)]   # x fastest
            grids = torch.meshgrid(*axes, indexing="ij")
            out.append(_exact(grids, t).to(torch.float32).reshape(-1))
    return torch.cat(out)


def _gpu_eoc(n, steps, tol=1e-6):
    """L2((0,T), L2) error of the GPU run; ghosts, u0 and errors on the device."""
    import torch
    dev = torch.device("cuda")
    h = 2.0 * L_HALF / n
    tau = T_END / steps
    p = _lib.Params.defaults()
    p.h = (h, h, h, h)
    p.tau = tau
    p.eps = h
    p.delta = p.vartheta = 0.0
    p.tol = tol
    dims = (n, n, n, n)
    xc = -L_HALF + (torch.arange(1, n + 1, device=dev, dtype=torch.float64) - 0.5) * h
    r2 = (xc[:, None, None, None] ** 2 + xc[None, :, None, None] ** 2 +
          xc[None, None, :, None] ** 2 + xc[None, None, None, :] ** 2)
    u = torch.empty((n, n, n, n), device=dev, dtype=torch.float32)
    err2 = 0.0
    with _lib.Seg4D(dims, params=p) as s:
        s.set_image(torch.zeros((n, n, n, n), device=dev, dtype=torch.float32))
        s.set_seeds([])
        s.setup()
        s.set_u(((r2 - 1.0) / 6.0).to(torch.float32))
        assert s.dirichlet_count(dims) == _ghosts(n, h, 0.0, dev).numel()
        for k in range(1, steps + 1):
            s.set_dirichlet(_ghosts(n, h, (k - 1) * tau, dev), _ghosts(n, h, k * tau, dev))
            info = s.solve()
            assert info["status"] == _lib.OK and info["res_rel"] <= tol, info
            s.read_u(u)
            e = u.to(torch.float64) - ((r2 - 1.0) / 6.0 + k * tau)
            err2 += tau * h ** 4 * float((e * e).sum())
    return math.sqrt(err2)


@pytest.mark.parametrize("n", [10, 20, 40])
def test_gpu_eoc_error_equals_oracle(n):
    h, steps, _, _ = _table()[n]
    ref, info = O.eoc(n, steps, T=T_END, L=L_HALF, eps_factor=1.0 / h, omega=1.5, tol=1e-12)
    assert info["status"] == O.OR_OK
    gpu = _gpu_eoc(n, steps)
    assert abs(gpu - ref) <= 2e-3 * ref, (n, gpu, ref)


@pytest.fixture(scope="module")
def gpu_errs():
    """Errors at N = 40 (1e-6 is far below its discretisation error), 80 and
    160 (solved to 3e-7: at N = 160 a 1e-6 solve changes the error by tens of
    percent)."""
    table = _table()
    return {40: _gpu_eoc(40, table[40][1]), 80: _gpu_eoc(80, table[80][1], tol=3e-7),
            160: _gpu_eoc(160, table[160][1], tol=3e-7)}


def test_gpu_eoc_order_40_80_matches_table(gpu_errs):
    """Row 4 of the table (N = 80: 41M voxels, 64 steps), past what the oracle
    runs in a test; absolute errors the printed ones up to the oracle's factor."""
    table = _table()
    eoc = math.log2(gpu_errs[40] / gpu_errs[80])
    assert abs(eoc - table[80][3]) < 0.05, (eoc, table[80][3])
    ratios = [table[n][2] / gpu_errs[n] for n in (40, 80)]
    assert all(2.2 < r < 2.7 for r in ratios), ratios


def test_gpu_eoc_order_80_160_is_second_order(gpu_errs):
    """Row 5 (N = 160: 655M voxels, 256 steps).  The table prints 1.861 there;
    solved to 3e-7 the scheme is second order (about 2.03).  The printed value
    is matched only by looser solves (1e-6 gives about 1.78): at N = 160 the
    row depends on the solve tolerance, which the paper does not give."""
    eoc = math.log2(gpu_errs[80] / gpu_errs[160])
    assert 1.9 < eoc < 2.15, eoc
