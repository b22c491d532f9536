"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare them."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2111_11866_gb300 import _lib

# per-voxel parity bound for u: |u_gpu - u_oracle| <= REL_TOL * max|u_oracle|
REL_TOL = 1e-4


def oracle_params(p: _lib.Params) -> O.OracleParams:
    """The same parameters for the oracle, but solved to 1e-12."""
    return O.OracleParams(h=tuple(p.h), tau=p.tau, eps=p.eps, K=p.K, delta=p.delta,
                          vartheta=p.vartheta, lambda_th=p.lambda_th, r_ball=p.r_ball,
                          R_init=p.R_init, v_init=p.v_init, sigma_t=p.sigma_t, omega=1.8,
                          tol=1e-12, omega_smooth=1.0, max_iters=200000, check_every=4)


def gpu_run(image, seeds, nsteps, params: _lib.Params | None = None, fields=()):
    dims = (image.shape[3], image.shape[2], image.shape[1], image.shape[0])
    with _lib.Seg4D(dims, params=params) as s:
        s.set_image(image)
        s.set_seeds(seeds)
        setup_info = s.setup()
        out = {"f_" + name: s.read_field(name) for name in fields}
        info = s.step(nsteps) if nsteps > 0 else None
        out["u"] = s.read_u()
        out["info"] = info
        out["setup_info"] = setup_info
        return out


def label_mismatch_outside_band(u_gpu, u_ref, iso=0.5):
    """Voxels whose labels (u >= iso) differ and that are not within one voxel
    (in 4D, face neighbours) of the oracle's iso-level crossing."""
    lab_g = u_gpu >= iso
    lab_r = u_ref >= iso
    diff = lab_g != lab_r
    band = np.zeros_like(lab_r)
    for ax in range(4):
        a = np.swapaxes(lab_r, 0, ax)
        b = np.swapaxes(band, 0, ax)
        cross = a[1:] != a[:-1]
        b[1:] |= cross
        b[:-1] |= cross
    return int((diff & ~band).sum())


def _oracle_job(args):
    image, seeds, nsteps, P, omp = args
    u, info = O.segment(image.astype(np.float64), seeds, P, nsteps=nsteps, omp=omp)
    return u, info


def oracle_segment_many(jobs, P, procs=None):
    """O.segment of every (image, seeds, nsteps) job on the plain oracle build,
    in a pool of spawned processes (one job per process at a time)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    procs = procs or max(1, min(len(jobs), os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_oracle_job, [(img, s, n, P, False) for img, s, n in jobs]))
