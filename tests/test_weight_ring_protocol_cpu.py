"""The Poisson-weight ring of the register mRNA/protein chain, as a CPU model
under random interleavings of its warps.

Weights of jumps [c C, (c+1) C) ("chunk c") go by cp.async into ring slots
j mod 2C; every warp copies its share.  Per jump k a warp: (events, before the
CTA barrier) waits for its own copies at k = -1 mod C and, at k = 1 mod C
(k > 1), starts copying chunk (k-1)/C + 1 into the slots of chunk (k-1)/C - 1;
meets the others at the barrier of jump k; then reads slot k mod 2C for its
observations of rho_k.  Before the loop chunks 0 and 1 are started and chunk
0 has landed.

A copy lands at its copier's wait, and another warp sees it only after a
barrier that completed once it had landed.  The model checks that every read
finds its jump's weight landed and published, and that no copy starts into a
slot whose previous jump some warp has not read yet (every warp reads every
jump: the worst case).  Staging one jump earlier, waiting for the copies one
jump late, or (with the wait one jump late) reading before the barrier, is
caught.  (Reading before the barrier with the wait in place is correct: the
chunk was published at the barrier that ended the previous chunk.)"""
import random

import pytest


def run(W, C, K, seed, stage_at=1, wait_at=None, read_after_barrier=True):
    rng = random.Random(seed)
    S = 2 * C
    wait_at = C - 1 if wait_at is None else wait_at
    ring = {}        # slot -> [jump it holds, copier, landed]
    reads_done = [-1] * W
    arrived = {}     # jump -> warps at its barrier
    published = {}   # jump -> {slot: jump} landed when its barrier completed

    def start_chunk(c, w):
        for j in range(c * C, min((c + 1) * C, K + 1)):
            if j % W != w:
                continue
            old = ring.get(j % S)
            if old is not None and old[0] > min(reads_done):
                return f"warp {w} started jump {j} over slot {j % S} (jump {old[0]}) before every warp read it"
            ring[j % S] = [j, w, False]
        return None

    def wait_own(w):
        for v in ring.values():
            if v[1] == w:
                v[2] = True

    def landed():
        return {sl: v[0] for sl, v in ring.items() if v[2]}

    def read(w, k, view):
        if view.get(k % S) != k:
            return f"warp {w} read jump {k}'s slot and found jump {view.get(k % S)}"
        reads_done[w] = k
        return None

    # prologue: chunks 0 and 1 started by every warp, chunk 0 waited for,
    # a barrier, then jump 0 read by every warp.
    for w in range(W):
        start_chunk(0, w)
        start_chunk(1, w)
    for v in ring.values():
        if v[0] < C:
            v[2] = True
    view = {w: landed() for w in range(W)}
    for w in range(W):
        err = read(w, 0, view[w])
        assert err is None, err

    st = [{"k": 1, "pc": "events"} for _ in range(W)]
    while any(s["k"] <= K for s in st):
        movable = [w for w in range(W) if st[w]["k"] <= K and
                   not (st[w]["pc"] == "barrier" and st[w]["k"] not in published)]
        if not movable:
            return "deadlock"
        w = rng.choice(movable)
        s = st[w]
        k = s["k"]
        if s["pc"] == "events":
            if k % C == wait_at:
                wait_own(w)
            if k % C == stage_at and k > 1 and ((k - 1) // C + 1) * C <= K:
                err = start_chunk((k - 1) // C + 1, w)
                if err:
                    return err
            if not read_after_barrier:
                err = read(w, k, view[w])
                if err:
                    return err
            arrived.setdefault(k, set()).add(w)
            if len(arrived[k]) == W:
                published[k] = landed()
            s["pc"] = "barrier"
        else:
            view[w] = published[k]
            if read_after_barrier:
                err = read(w, k, view[w])
                if err:
                    return err
            s["k"], s["pc"] = k + 1, "events"
    return None


@pytest.mark.parametrize("W,C", [(2, 4), (3, 4), (4, 8)])
@pytest.mark.parametrize("read_after_barrier", [True, False])
def test_weight_ring_reads_are_published_and_never_overwritten(W, C, read_after_barrier):
    for seed in range(200):
        err = run(W, C, 6 * C, seed, read_after_barrier=read_after_barrier)
        assert err is None, (seed, err)


@pytest.mark.parametrize("mutation", [dict(stage_at=0), dict(wait_at=1), dict(wait_at=0, read_after_barrier=False)])
def test_weight_ring_model_catches_broken_orders(mutation):
    fails = [run(3, 4, 24, seed, **mutation) for seed in range(200)]
    assert any(f is not None for f in fails), mutation
