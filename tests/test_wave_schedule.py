"""The work-item schedule of the fused red-black frame pipeline
(k_sweep_wave, solve_kernels.cu), modelled on the CPU.

Item (g, T): red of frame g mod Ts and black of the frame whose red ran at
step g - 2, on tile T; Ts = max(n4, 4) steps per sweep; CTAs take items in
ticket order, and an item starts once tile T has completed step g - 1 and its
neighbour tiles (T +- 1 in the z-plane, T +- tpp across planes) have completed
step g - 2.  Under random CTA timing every read must see exactly the values
red-then-black sweeps would see, and no two running items may touch the same
data in conflict.  Weaker rules (neighbours one step less, Ts = 3) must fail,
so that the model can tell a wrong rule from a right one.
"""
import random

import pytest


def _run(tpp, n3, n4, nsweeps, ctas, seed, lag_nb=1, ts_min=4):
    rnd = random.Random(seed)
    Tf = tpp * n3
    Ts = max(n4, ts_min)
    total = (nsweeps * Ts + 2) * Tf
    red_steps = nsweeps * Ts
    done = [0] * Tf
    ver = {}   # (colour, frame, tile) -> completed updates

    def item(tk):
        g, t = divmod(tk, Tf)
        tt, kk = t % tpp, t // tpp
        nb = [t]
        if tt > 0:
            nb.append(t - 1)
        if tt + 1 < tpp:
            nb.append(t + 1)
        if kk > 0:
            nb.append(t - tpp)
        if kk + 1 < n3:
            nb.append(t + tpp)
        work = []
        s = g % Ts
        if g < red_steps and s < n4:
            reads = [(1, s, x) for x in nb] + [(1, f, t) for f in (s - 1, s + 1) if 0 <= f < n4]
            work.append(((0, s, t), reads, g // Ts))
        if g >= 2:
            gb = g - 2
            f = gb % Ts
            if gb < red_steps and f < n4:
                reads = [(0, f, x) for x in nb] + [(0, e, t) for e in (f - 1, f + 1) if 0 <= e < n4]
                work.append(((1, f, t), reads, gb // Ts + 1))
        return g, t, nb, work

    def ready(g, t, nb):
        if g > 0 and done[t] < g:
            return False
        return all(not (g > lag_nb and done[x] < g - lag_nb) for x in nb[1:])

    nxt = 0
    cta = []
    for _ in range(ctas):
        cta.append([nxt, False])
        nxt += 1
    running = {}
    finished = 0
    while finished < ctas:
        c = rnd.randrange(ctas)
        tk, busy = cta[c]
        if tk is None:
            continue
        if tk >= total:
            cta[c][0] = None
            finished += 1
            continue
        g, t, nb, work = item(tk)
        if not busy:
            if not ready(g, t, nb):
                continue
            for w, reads, want in work:
                for r in reads:
                    assert ver.get(r, 0) == want, ("stale read", tk, w, r)
            for og, ot, onb, owork in running.values():
                for w, reads, _ in work:
                    for ow, oreads, _ in owork:
                        assert w != ow and w not in oreads and ow not in reads, ("conflict", tk)
            running[c] = (g, t, nb, work)
            cta[c][1] = True
        else:
            for w, _, _ in work:
                ver[w] = ver.get(w, 0) + 1
            done[t] = g + 1
            del running[c]
            cta[c] = [nxt, False]
            nxt += 1
    assert all(v == nsweeps for v in ver.values())


SHAPES = [(3, 2, 5, 3, 4), (2, 3, 1, 3, 5), (4, 1, 2, 2, 7), (2, 2, 4, 3, 9), (1, 1, 3, 4, 3),
          (5, 3, 6, 2, 20)]


@pytest.mark.parametrize("shape", SHAPES)
def test_schedule_gives_red_black_sweeps(shape):
    for seed in range(12):
        _run(*shape, seed)


def test_weaker_rules_are_caught():
    with pytest.raises(AssertionError):
        for seed in range(40):
            for shape in SHAPES:
                _run(*shape, seed, lag_nb=2)
    with pytest.raises(AssertionError):
        for seed in range(40):
            for shape in SHAPES:
                _run(*shape, seed, ts_min=3)
