"""The named-barrier hand-over of the small-group encounter kernel (k_bs_ws),
modelled on the CPU: warp 0 posts evaluation points and takes their
accelerations, warps 1 and 2 take the mutual terms of the even and odd
points, warp 3 the stellar term of every point; each of the four barriers
(positions and accelerations, by parity) is met by three warps.  Random
interleavings and random stop rounds over several substeps must never
deadlock, every barrier generation must complete with exactly three warps,
and a protocol with the stellar warp's second position barrier left out at
the stop must be caught (the model is not vacuous).
"""
import random

import pytest


def run(seed, nsub=6, maxm=16, stop_second_sync=True):
    rnd = random.Random(seed)
    gens = {b: [] for b in ("P0", "P1", "A0", "A1")}   # current generation's participants
    completed = {b: 0 for b in gens}
    state = {"stop": False}
    waiting = {}      # warp -> (barrier, generation index) it waits for

    def arrive(w, b, blocking):
        gens[b].append(w)
        assert len(gens[b]) <= 3, (b, gens[b])
        g = completed[b]
        if len(gens[b]) == 3:
            completed[b] += 1
            gens[b] = []
        if blocking:
            return ("wait", b, g)
        return None

    def w0():
        for sub in range(nsub):
            stop_m = rnd.randint(2, maxm)
            state["stop"] = False
            yield arrive(0, "P0", False)
            yield arrive(0, "P1", False)
            m = 0
            while True:
                par = m & 1
                yield arrive(0, "A1" if par else "A0", True)
                yield arrive(0, "P1" if par else "P0", False)
                if m >= stop_m or m == maxm:
                    yield arrive(0, "A0" if par else "A1", True)
                    yield arrive(0, "A1" if par else "A0", True)
                    state["stop"] = True
                    yield arrive(0, "P0", False)
                    yield arrive(0, "P1", False)
                    break
                m += 1
            yield ("block",)

    def weval(w, par):
        for sub in range(nsub):
            m = par
            while True:
                yield arrive(w, "P1" if par else "P0", True)
                if state["stop"]:
                    break
                yield arrive(w, "A1" if par else "A0", False)
                m += 2
            yield ("block",)

    def w3():
        for sub in range(nsub):
            m = 0
            while True:
                par = m & 1
                yield arrive(3, "P1" if par else "P0", True)
                if state["stop"]:
                    if stop_second_sync:
                        yield arrive(3, "P0" if par else "P1", True)
                    break
                yield arrive(3, "A1" if par else "A0", False)
                m += 1
            yield ("block",)

    gens_ = {0: w0(), 1: weval(1, 0), 2: weval(2, 1), 3: w3()}
    blockbar = set()
    nblock = 0
    pending = {w: None for w in gens_}
    done = set()
    steps = 0
    while len(done) < 4:
        steps += 1
        assert steps < 100000, "livelock"
        ready = []
        for w in gens_:
            if w in done:
                continue
            p = pending[w]
            if p is None:
                ready.append(w)
            elif p[0] == "wait" and completed[p[1]] > p[2]:
                ready.append(w)
            elif p[0] == "block" and nblock > p[1]:
                ready.append(w)
        assert ready, ("deadlock", pending, gens, completed)
        w = rnd.choice(ready)
        try:
            r = next(gens_[w])
        except StopIteration:
            done.add(w)
            pending[w] = None
            continue
        if r is not None and r[0] == "block":
            blockbar.add(w)
            r = ("block", nblock)
            if len(blockbar) == 4:
                blockbar.clear()
                nblock += 1
        pending[w] = r
    for b in gens:
        assert gens[b] == [], (b, gens[b])
    return completed


def test_protocol_never_deadlocks():
    for seed in range(400):
        run(seed)


def test_a_missing_barrier_is_caught():
    with pytest.raises(AssertionError, match="deadlock"):
        for seed in range(50):
            run(seed, stop_second_sync=False)
