"""seg4d_residual_norms_noalloc, the entry point for callers that cannot
allocate device memory (their memory belongs to their own pool or budget, or
they cannot take the synchronisation cudaMalloc/cudaFree may imply): it must
give the same residual norms as the allocating solve path and as the FP64
oracle's residual of the same arrays, call after call.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import oracle as O
from paper_2111_11866_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4   # the parity tolerance of the other GPU tests


def _reference_and_inputs(dims, seed):
    """Solve a few sweeps through a handle (not converged on purpose, so the
    residual is far above rounding) and return the handle's own residual norms
    together with the step system read back as plain device arrays."""
    import torch
    n1, n2, n3, n4 = dims
    c = synth.small_nuclei(seed=seed, n=dims, count=3, nsteps=1)
    rng = np.random.default_rng(seed)
    u0 = np.clip(rng.normal(0.4, 0.2, size=c.image.shape), 0, 1).astype(np.float32)
    p = _lib.Params.defaults()
    p.r_ball = p.R_init = 6.0
    with _lib.Seg4D(dims, params=p) as s:
        s.set_image(c.image)
        s.set_seeds(c.seeds)
        s.setup()
        # one heavily under-relaxed sweep: the iterate stays far from the
        # solution, so the residual is orders of magnitude above FP32 rounding
        s.set_params(omega=0.05, max_iters=1, check_every=1)
        s.set_u(u0)
        info = s.solve(allow_not_converged=True)
        shape = (n4, n3, n2, n1)
        u = torch.empty(shape, dtype=torch.float32, device="cuda")
        diag = torch.empty(shape, dtype=torch.float32, device="cuda")
        off = torch.empty(shape + (8,), dtype=torch.float32, device="cuda")
        s.read_u(u)
        s.read_field("diag", diag)
        s.read_field("off", off)
    b = torch.from_numpy(u0).cuda()
    torch.cuda.synchronize()
    return info, (u, b, diag, off)


def test_noalloc_matches_allocating_path_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_11866_gb300 import build
    build.build()
    # larger grid first, then a smaller one: the second call must not pick up
    # records the first call left in the shared scratch array
    cases = [((45, 30, 19, 6), 31), ((21, 14, 9, 3), 32)]
    for dims, seed in cases:
        info, (u, b, diag, off) = _reference_and_inputs(dims, seed)
        assert info["status"] == _lib.ERR_NOT_CONVERGED and info["res_rel"] > 1.0
        result = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        _lib.residual_norms_noalloc(dims, u, b, diag, off, result, stream)
        torch.cuda.synchronize()
        rn, bn = result.tolist()
        assert abs(rn - info["res_l2"]) <= REL_TOL * info["res_l2"], (dims, rn, info["res_l2"])
        assert abs(bn - info["bnorm"]) <= REL_TOL * info["bnorm"], (dims, bn, info["bnorm"])
        # and the FP64 oracle's residual of the very same arrays
        r = O.residual(diag.cpu().numpy(), off.cpu().numpy(), b.cpu().numpy(), u.cpu().numpy())
        ro = float(np.sqrt((r * r).sum()))
        bo = float(torch.sqrt((b.double() ** 2).sum()))
        assert abs(rn - ro) <= REL_TOL * ro, (dims, rn, ro)
        assert abs(bn - bo) <= REL_TOL * bo, (dims, bn, bo)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    r = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.Seg4DError) as e:
        _lib.residual_norms_noalloc((4, 4096, 1025, 1), t, t, t, t, r)   # 4,198,400 x-lines
    assert e.value.status == _lib.ERR_INVALID
    assert "too large" in str(e.value)
