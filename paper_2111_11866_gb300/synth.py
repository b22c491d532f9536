"""Seeded synthetic 3D+time inputs shaped like the paper's microscopy data.

The paper's datasets (zebrafish hindbrain and pectoral fin, Section 4) are not
available; these generators stand in for them.  They produce only images and
seed points -- none of the segmentation arithmetic lives here, so both the
CUDA path and the CPU oracle can be fed from this module.

Arrays are float32 of shape (n4, n3, n2, n1): frames, z, y, x (x fastest).
Seeds are (x, y, z, frame) in 0-based voxel units, rounded to voxel centres.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Case:
    name: str
    image: np.ndarray           # float32 (n4, n3, n2, n1)
    seeds: np.ndarray           # float64 (m, 4): x, y, z, frame
    nsteps: int
    meta: dict

    @property
    def dims(self):
        n4, n3, n2, n1 = self.image.shape
        return (n1, n2, n3, n4)


# --------------------------------------------------------------------------
# tiny: one moving ball with a wedge gap (full-grid, oracle-sized)
# --------------------------------------------------------------------------

def tiny(seed: int = 1, n=(32, 32, 32, 16), radius: float = 8.0, speed: float = 0.5,
         noise: float = 0.1, gap_deg: float = 60.0, nsteps: int = 10) -> Case:
    """A 3D ball of radius 8 (intensity 1 inside, 0 outside) whose centre moves
    0.5 voxel per frame along x, a 60-degree wedge cut from its boundary shell
    (6 <= rho <= 8) in the x-y angle, and additive Gaussian noise of sigma 0.1.
    One seed at the frame-0 centre."""
    rng = np.random.default_rng(seed)
    n1, n2, n3, n4 = n
    cx0, cy, cz = n1 / 2 - 4.0, float(n2 // 2), float(n3 // 2)
    z, y, x = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    img = np.zeros((n4, n3, n2, n1), np.float32)
    for l in range(n4):
        cx = cx0 + speed * l
        dx, dy, dz = x - cx, y - cy, z - cz
        rho = np.sqrt(dx * dx + dy * dy + dz * dz)
        ang = np.degrees(np.arctan2(dy, dx)) % 360.0
        ball = rho <= radius
        wedge = (rho >= radius - 2.0) & (ang < gap_deg)
        img[l] = np.where(ball & ~wedge, 1.0, 0.0)
    img += rng.normal(0.0, noise, size=img.shape).astype(np.float32)
    seeds = np.array([[round(cx0), cy, cz, 0]], dtype=np.float64)
    return Case("tiny 32x32x32x16 moving ball", img, seeds, nsteps,
                {"radius": radius, "speed": speed, "noise": noise, "gap_deg": gap_deg})


def moving_sphere(seed: int = 6, n=(32, 32, 32, 20), radius: float = 6.0, speed: float = 0.5,
                  noise: float = 0.05, missing=(5, 10, 15), nsteps: int = 10) -> Case:
    """A sphere of radius `radius` (1 inside, 0 outside) moving `speed` voxels
    per frame along x, with Gaussian noise, and the frames in `missing` blanked
    (background only): the missing-frame experiment of Section 4.  Seeds at the
    sphere centre of every frame (the path is known; only the image data of the
    missing frames is absent)."""
    rng = np.random.default_rng(seed)
    n1, n2, n3, n4 = n
    cx0, cy, cz = n1 / 2 - speed * (n4 - 1) / 2, float(n2 // 2), float(n3 // 2)
    z, y, x = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    img = np.zeros((n4, n3, n2, n1), np.float32)
    truth = np.zeros((n4, n3, n2, n1), bool)
    for l in range(n4):
        cx = cx0 + speed * l
        truth[l] = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= radius ** 2
        if l not in missing:
            img[l] = truth[l]
    img += rng.normal(0.0, noise, size=img.shape).astype(np.float32)
    seeds = np.array([[round(cx0 + speed * l), cy, cz, l] for l in range(n4)], dtype=np.float64)
    return Case(f"moving sphere {n1}x{n2}x{n3}x{n4}, frames {tuple(missing)} missing", img, seeds,
                nsteps, {"truth": truth, "missing": tuple(missing), "radius": radius})


# --------------------------------------------------------------------------
# nuclei: ellipsoids with Gaussian profiles on smooth trajectories
# --------------------------------------------------------------------------

def _trajectories(rng, m, n4, lo, hi, vmax=1.0):
    """Cubic-spline paths through random control points, scaled so that the
    speed never exceeds vmax voxels per frame."""
    from scipy.interpolate import CubicSpline

    knots = np.unique(np.r_[np.arange(0, n4, 8), n4 - 1]) if n4 > 1 else np.array([0])
    starts = rng.uniform(lo, hi, size=(m, 3))
    paths = np.repeat(starts[:, None, :], n4, axis=1)
    if n4 == 1 or len(knots) < 2:
        return paths
    t = np.arange(n4)
    for a in range(m):
        ctrl = starts[a] + np.cumsum(rng.normal(0.0, 3.0, size=(len(knots), 3)), axis=0)
        ctrl[0] = starts[a]
        cs = CubicSpline(knots, ctrl, axis=0)
        p = cs(t)
        v = np.linalg.norm(np.diff(p, axis=0), axis=1).max()
        if v > vmax:
            p = starts[a] + (p - starts[a]) * (vmax / v)
        paths[a] = p
    return paths


def nuclei(seed: int, n, count: int | None = None, density_per_voxel: float | None = None,
           axes=(4.0, 9.0), peak=(0.5, 1.0), background: float = 0.05,
           photons: float = 1000.0, read_noise: float = 0.05, nsteps: int = 50,
           margin: float = 10.0, name: str = "nuclei") -> Case:
    """Ellipsoidal nuclei (semi-axes uniform in `axes`) with Gaussian intensity
    profiles (peak uniform in `peak`) moving on cubic-spline trajectories at
    <= 1 voxel per frame, over a background of 0.05 with Poisson-like shot
    noise (photon count = I * photons) plus Gaussian read noise.  Seeds at
    every nucleus centre in frame 0."""
    rng = np.random.default_rng(seed)
    n1, n2, n3, n4 = n
    if count is None:
        count = max(1, int(round(n1 * n2 * n3 * density_per_voxel)))
    lo = np.array([margin, margin, min(margin, n3 / 4)])
    hi = np.array([n1 - margin, n2 - margin, n3 - min(margin, n3 / 4)])
    paths = _trajectories(rng, count, n4, lo, hi)
    semi = rng.uniform(axes[0], axes[1], size=(count, 3))
    peaks = rng.uniform(peak[0], peak[1], size=count)
    img = np.full((n4, n3, n2, n1), background, np.float32)
    for l in range(n4):
        frame = img[l]
        for a in range(count):
            c = paths[a, l]
            ext = 2.0 * semi[a]
            x0, x1 = max(0, int(c[0] - ext[0])), min(n1, int(c[0] + ext[0]) + 2)
            y0, y1 = max(0, int(c[1] - ext[1])), min(n2, int(c[1] + ext[1]) + 2)
            z0, z1 = max(0, int(c[2] - ext[2])), min(n3, int(c[2] + ext[2]) + 2)
            if x0 >= x1 or y0 >= y1 or z0 >= z1:
                continue
            zz, yy, xx = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1),
                                     indexing="ij")
            r2 = (((xx - c[0]) / semi[a, 0]) ** 2 + ((yy - c[1]) / semi[a, 1]) ** 2 +
                  ((zz - c[2]) / semi[a, 2]) ** 2)
            val = (peaks[a] * np.exp(-2.0 * r2)).astype(np.float32)
            sub = frame[z0:z1, y0:y1, x0:x1]
            np.maximum(sub, val, out=sub)
    shot = rng.poisson(np.clip(img, 0, None) * photons).astype(np.float32) / photons
    img = shot + rng.normal(0.0, read_noise, size=img.shape).astype(np.float32)
    cen = np.rint(paths[:, 0, :])
    cen[:, 0] = np.clip(cen[:, 0], 0, n1 - 1)
    cen[:, 1] = np.clip(cen[:, 1], 0, n2 - 1)
    cen[:, 2] = np.clip(cen[:, 2], 0, n3 - 1)
    seeds = np.concatenate([cen, np.zeros((count, 1))], axis=1)
    return Case(name, img.astype(np.float32), seeds, nsteps,
                {"count": count, "semi_axes": semi, "peaks": peaks, "paths": paths})


def nuclei_frames(seed: int, n, density_per_voxel: float, device, axes=(4.0, 9.0),
                  peak=(0.5, 1.0), background: float = 0.05, photons: float = 1000.0,
                  read_noise: float = 0.05, margin: float = 10.0):
    """The nuclei() recipe frame by frame on `device`, for grids too large to
    build at once: the per-nucleus draws (paths, semi-axes, peaks) come from
    the same seeded numpy generator, each frame's image and noise from a seeded
    torch generator.  Returns (seeds (m, 4), count, generator of the n4 frames
    as (n3, n2, n1) float32 tensors on the device, in order)."""
    import torch

    rng = np.random.default_rng(seed)
    n1, n2, n3, n4 = n
    count = max(1, int(round(n1 * n2 * n3 * density_per_voxel)))
    lo = np.array([margin, margin, min(margin, n3 / 4)])
    hi = np.array([n1 - margin, n2 - margin, n3 - min(margin, n3 / 4)])
    paths = _trajectories(rng, count, n4, lo, hi)
    semi = rng.uniform(axes[0], axes[1], size=(count, 3))
    peaks = rng.uniform(peak[0], peak[1], size=count)
    cen = np.rint(paths[:, 0, :])
    cen[:, 0] = np.clip(cen[:, 0], 0, n1 - 1)
    cen[:, 1] = np.clip(cen[:, 1], 0, n2 - 1)
    cen[:, 2] = np.clip(cen[:, 2], 0, n3 - 1)
    seeds = np.concatenate([cen, np.zeros((count, 1))], axis=1)

    def frames():
        ar = [torch.arange(m, dtype=torch.float32, device=device) for m in (n1, n2, n3)]
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        for l in range(n4):
            frame = torch.full((n3, n2, n1), background, dtype=torch.float32, device=device)
            for a in range(count):
                c = paths[a, l]
                ext = 2.0 * semi[a]
                x0, x1 = max(0, int(c[0] - ext[0])), min(n1, int(c[0] + ext[0]) + 2)
                y0, y1 = max(0, int(c[1] - ext[1])), min(n2, int(c[1] + ext[1]) + 2)
                z0, z1 = max(0, int(c[2] - ext[2])), min(n3, int(c[2] + ext[2]) + 2)
                if x0 >= x1 or y0 >= y1 or z0 >= z1:
                    continue
                rx = ((ar[0][x0:x1] - float(c[0])) / float(semi[a, 0])) ** 2
                ry = ((ar[1][y0:y1] - float(c[1])) / float(semi[a, 1])) ** 2
                rz = ((ar[2][z0:z1] - float(c[2])) / float(semi[a, 2])) ** 2
                r2 = rz[:, None, None] + ry[None, :, None] + rx[None, None, :]
                sub = frame[z0:z1, y0:y1, x0:x1]
                torch.maximum(sub, float(peaks[a]) * torch.exp(-2.0 * r2), out=sub)
            frame.copy_(torch.poisson(frame.clamp_(min=0.0) * photons, generator=g) / photons +
                        read_noise * torch.randn(frame.shape, generator=g, device=device))
            yield frame

    return seeds, count, frames()


def nuclei_device(seed: int, n, density_per_voxel: float, device, nsteps: int = 20,
                  name: str = "nuclei (device)", **kw):
    """nuclei_frames assembled into one (n4, n3, n2, n1) tensor on the device.
    Returns (image, seeds (m, 4), nsteps, meta)."""
    import torch

    seeds, count, frames = nuclei_frames(seed, n, density_per_voxel, device, **kw)
    n1, n2, n3, n4 = n
    img = torch.empty((n4, n3, n2, n1), dtype=torch.float32, device=device)
    for l, f in enumerate(frames):
        img[l].copy_(f)
    return img, seeds, nsteps, {"count": count, "name": name}


def large(device, seed: int = 3, frames: int = 48, depth: int = 128):
    """512x512x128 space x 48 frames (1.61G voxels), one nucleus per 40^3
    voxels (about 524), 20 steps; built on the device (nuclei_device).  Fewer
    frames (or z-planes) give the same 512x512 rows at a size a profiler can
    replay."""
    return nuclei_device(seed, (512, 512, depth, frames), 1.0 / 40 ** 3, device, nsteps=20,
                         name=f"large 512x512x{depth}x{frames}, 1 nucleus per 40^3")


def paper_scale(device, seed: int = 7):
    """The size of the paper's largest stack (567x577x147 x 70 frames,
    3,366,466,110 voxels; Section 4, the zebrafish pectoral fin), with the
    nucleus generator at one nucleus per 40^3 voxels.  Returns
    (dims, seeds, count, frame generator) as nuclei_frames."""
    n = (567, 577, 147, 70)
    seeds, count, frames = nuclei_frames(seed, n, 1.0 / 40 ** 3, device)
    return n, seeds, count, frames


def medium(seed: int = 2) -> Case:
    """128x128x64 space x 32 frames (33.5M voxels), 60 nuclei, 50 steps."""
    return nuclei(seed, (128, 128, 64, 32), count=60, nsteps=50,
                  name="medium 128x128x64x32, 60 nuclei")


def small_nuclei(seed: int, n=(40, 36, 20, 6), count: int = 4, nsteps: int = 3) -> Case:
    """A reduced nucleus field for parity tests (odd sizes, several tiles)."""
    return nuclei(seed, n, count=count, nsteps=nsteps, margin=6.0,
                  name=f"nuclei {n[0]}x{n[1]}x{n[2]}x{n[3]}")


def random_field(seed: int, n, lo=0.0, hi=1.0) -> np.ndarray:
    n1, n2, n3, n4 = n
    return np.random.default_rng(seed).uniform(lo, hi, size=(n4, n3, n2, n1)).astype(np.float32)


# --------------------------------------------------------------------------
# per-nucleus windows (batched / served workloads)
# --------------------------------------------------------------------------

def _cut(volume: Case, a: int, edge, frames: int):
    """Window of spatial size edge (x, y, z) and `frames` frames around
    nucleus a of `volume`, starting at frame 0, shifted to lie inside."""
    n4, n3, n2, n1 = volume.image.shape
    ex, ey, ez = (min(int(e), m) for e, m in zip(edge, (n1, n2, n3)))
    fr = min(int(frames), n4)
    c = volume.meta["paths"][a, 0]
    x0 = int(np.clip(round(c[0]) - ex // 2, 0, n1 - ex))
    y0 = int(np.clip(round(c[1]) - ey // 2, 0, n2 - ey))
    z0 = int(np.clip(round(c[2]) - ez // 2, 0, n3 - ez))
    img = np.ascontiguousarray(volume.image[:fr, z0:z0 + ez, y0:y0 + ey, x0:x0 + ex])
    seed = np.array([[np.clip(round(c[0]) - x0, 0, ex - 1), np.clip(round(c[1]) - y0, 0, ey - 1),
                      np.clip(round(c[2]) - z0, 0, ez - 1), 0]], dtype=np.float64)
    return img, seed


def windows(count: int, seed: int = 4, edge=(24, 64), frames=(8, 16), nsteps: int = 30,
            volumes: int = 2):
    """`count` per-nucleus windows cut from `volumes` medium-generator volumes
    (seeds seed, seed+1, ...): cubic spatial edge uniform in `edge`, frame
    count uniform in `frames`, one seed at the nucleus centre in frame 0.
    Returns a list of (image, seeds, nsteps)."""
    rng = np.random.default_rng(seed)
    vols = [nuclei(seed + v, (128, 128, 64, 32), count=60, nsteps=nsteps) for v in range(volumes)]
    out = []
    for k in range(count):
        vol = vols[k % volumes]
        a = (k // volumes) % vol.meta["count"]
        e = int(rng.integers(edge[0], edge[1] + 1))
        f = int(rng.integers(frames[0], frames[1] + 1))
        img, s = _cut(vol, a, (e, e, e), f)
        out.append((img, s, nsteps))
    return out


def request_window(seed: int, edge: int, frames: int, nsteps: int = 30):
    """One served request: a window of edge^3 voxels x `frames` frames holding
    one nucleus (semi-axes scaled to the window) and a seed at its centre."""
    e = int(edge)
    c = nuclei(seed, (e, e, e, int(frames)), count=1, axes=(min(4.0, e / 6), min(9.0, e / 3)),
               margin=e / 3, nsteps=nsteps, name=f"request {e}^3x{frames}")
    return c.image, c.seeds, nsteps


def request_sizes(count: int, seed: int = 5, lo: float = 16.0, hi: float = 96.0):
    """Window edges log-uniform in [lo, hi] with frames = round(edge/4): the
    sizes of the served requests (16^3 x 4 to 96^3 x 24)."""
    rng = np.random.default_rng(seed)
    e = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))
    edges = np.rint(e).astype(int)
    return [(int(s), int(s), int(s), max(1, int(round(s / 4)))) for s in edges]
