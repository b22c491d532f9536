"""Continuous-batching service of per-nucleus segmentation requests.

A request is one window (image, seeds, number of time steps).  Requests arrive
on their own clock (open loop).  Each engine iteration of `Server.run`
  1. moves every request whose arrival time has passed into a FIFO queue,
  2. admits queued requests into the batch while the arena has room (the
     device-memory budget is the admission control; a refused request stays
     queued),
  3. advances every resident window by one time step (newly admitted windows
     first run their set-up) -- one batched launch per kernel for all of them,
  4. retires finished windows: records their latency (completion - arrival)
     and returns their arena space.
Work of requests that arrive while others are on the GPU therefore overlaps
with them on the device; each result is the same as the request run alone
(the batch engine guarantees it bit for bit).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import _lib


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds from the start of the run
    image: object                  # (n4, n3, n2, n1) float32, numpy or CUDA tensor
    seeds: np.ndarray
    nsteps: int
    admitted: float | None = None
    done: float | None = None
    window: int | None = None
    result: np.ndarray | None = None
    state: str = "queued"


@dataclass
class ServeStats:
    served: int = 0
    failed: int = 0
    refused_admissions: int = 0      # admission attempts refused for lack of room
    iterations: int = 0
    wall_s: float = 0.0
    latencies: list = field(default_factory=list)
    queue_waits: list = field(default_factory=list)
    window_sweeps: int = 0
    launches: int = 0
    max_resident: int = 0
    max_arena_used: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.array([np.nan])
        q = np.array(self.queue_waits) if self.queue_waits else np.array([np.nan])
        return {"served": self.served, "failed": self.failed,
                "seg_per_s": self.served / self.wall_s if self.wall_s > 0 else None,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(np.mean(lat) * 1e3),
                "queue_p50_ms": float(np.percentile(q, 50) * 1e3),
                "refused_admissions": self.refused_admissions,
                "iterations": self.iterations, "wall_s": self.wall_s,
                "window_sweeps": self.window_sweeps, "launches": self.launches,
                "max_resident": self.max_resident, "max_arena_used": self.max_arena_used}


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times of an open-loop Poisson process (seeded)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


class Server:
    """`budget_bytes` is the device-memory admission budget (the batch arena).
    `max_resident_voxels` also caps the voxels in flight: beyond the point
    where the batched launches saturate the GPU, more resident windows only
    lengthen every engine iteration (each request needs one iteration per time
    step), so latency grows with no gain in throughput."""

    def __init__(self, budget_bytes: int, max_windows: int = 4096, params=None, stream=None,
                 keep_results: bool = False, max_resident_voxels: float = 64e6):
        self.batch = _lib.Batch(budget_bytes, max_windows, stream=stream, params=params)
        self.keep_results = keep_results
        self.max_resident_voxels = max_resident_voxels

    def close(self):
        self.batch.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, requests: list[Request], horizon_s: float | None = None,
            clock=time.perf_counter, sync=None) -> ServeStats:
        """Serve `requests` (sorted by arrival) until all are done, or until
        `horizon_s` seconds have passed (then the rest is left unserved)."""
        st = ServeStats()
        pending = list(requests)
        queue: list[Request] = []
        resident: dict[int, Request] = {}
        resident_vox = 0
        t0 = clock()
        nxt = 0
        while nxt < len(pending) or queue or resident:
            now = clock() - t0
            if horizon_s is not None and now > horizon_s:
                break
            while nxt < len(pending) and pending[nxt].arrival <= now:
                queue.append(pending[nxt])
                nxt += 1
            # FIFO admission while the arena has room and the voxel cap allows
            while queue:
                r = queue[0]
                nv = int(np.prod(r.image.shape))
                if resident and resident_vox + nv > self.max_resident_voxels:
                    break
                wid = self.batch.add(r.image, r.seeds, r.nsteps)
                if wid is None:
                    st.refused_admissions += 1
                    break
                queue.pop(0)
                r.window = wid
                r.admitted = clock() - t0
                r.state = "resident"
                resident[wid] = r
                resident_vox += nv
            if not resident:
                # idle until the next arrival
                if nxt < len(pending):
                    wait = pending[nxt].arrival - (clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                continue
            info = self.batch.advance()
            if sync is not None:
                sync()
            st.iterations += 1
            st.window_sweeps += info["window_sweeps"]
            st.launches += info["launches"]
            st.max_resident = max(st.max_resident, len(resident))
            st.max_arena_used = max(st.max_arena_used, info["arena_used"])
            now = clock() - t0
            for wid in list(resident):
                w = self.batch.poll(wid)
                if w["state"] in ("done", "failed"):
                    r = resident.pop(wid)
                    resident_vox -= int(np.prod(r.image.shape))
                    r.done = now
                    r.state = w["state"]
                    if w["state"] == "done":
                        st.served += 1
                        st.latencies.append(r.done - r.arrival)
                        st.queue_waits.append(r.admitted - r.arrival)
                        if self.keep_results:
                            r.result = self.batch.read_u(wid)
                    else:
                        st.failed += 1
                    self.batch.remove(wid)
        st.wall_s = clock() - t0
        return st
