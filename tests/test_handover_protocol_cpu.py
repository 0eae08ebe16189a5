"""The row hand-over between the two CTAs of a cluster in the register
mRNA/protein chain, as a CPU model under random interleavings.

Each boundary thread, at jump k: reads the neighbour CTA's row of rho_{k-1}
from its halo slot (parity (k-1) mod 2), sends its own row of rho_k into the
neighbour's slot of parity k mod 2 (st.async: the bytes and their count on
the neighbour's mbarrier of that parity), meets its CTA at the barrier, then
waits for the phase of its own parity-(k mod 2) mbarrier that counts the
neighbour's rows of rho_k; the column-quad-0 thread re-arms that barrier
(arrive + expect_tx of all the rows) for jump k + 2.  Before the loop the rows
of rho_0 are in place and the barriers of parity 1 (jump 1) and 0 (jump 2)
are armed.

The model checks what the protocol's correctness rests on: every read sees
exactly the neighbour's row of rho_{k-1} (never an older one, never one of a
later jump written over it), no barrier phase is completed by bytes or an
arrival of another jump, and no schedule deadlocks.  Mutated protocols (one
halo slot instead of two, no wait, re-arming before the wait) are caught by
the same checks, so the model can see the races it rules out."""
import random

import pytest


class Barrier:
    """mbarrier with an arrival count of 1 and a transaction count."""

    def __init__(self):
        self.phase, self.pending, self.tx, self.tag = 0, 1, 0, None

    def arm(self, nbytes, tag):
        assert self.pending == 1, "arrival on a phase that already had its arrival"
        assert self.tag is None or self.tag == tag, "arm of another jump's phase"
        self.pending -= 1
        self.tx += nbytes
        self.tag = tag
        self._settle()

    def complete_tx(self, nbytes, tag):
        assert self.tag is None or self.tag == tag, "bytes of another jump counted on this phase"
        self.tag = tag
        self.tx -= nbytes
        self._settle()

    def _settle(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending, self.tag = 1, None

    def done(self, parity):
        return (self.phase & 1) != parity


def run(n, K, seed, slots=2, wait=True, arm_early=False):
    """One random schedule of two CTAs with n boundary threads each for K
    jumps; returns None on success or a description of the failure."""
    rng = random.Random(seed)
    ROW = 16
    halo = [[[(1 - c, q, 0) for q in range(n)] for _ in range(slots)] for c in range(2)]  # rho_0 in place
    bars = [[Barrier(), Barrier()] for _ in range(2)]
    for c in range(2):  # parity 1 armed for jump 1, parity 0 for jump 2
        bars[c][1].arm(ROW * n, 1)
        bars[c][0].arm(ROW * n, 2)
    # per thread: jump, stage, phase bits
    th = {(c, q): {"k": 1, "st": "read", "hph": [0, 0]} for c in range(2) for q in range(n)}
    at_barrier = [dict() for _ in range(2)]  # jump -> threads arrived

    def slot(k):
        return k % slots

    steps = 0
    while True:
        live = [t for t, s in th.items() if s["k"] <= K]
        if not live:
            return None
        movable = []
        for t in live:
            s = th[t]
            c, q = t
            if s["st"] == "barrier" and len(at_barrier[c].get(s["k"], ())) < n:
                continue
            if s["st"] == "wait" and wait:
                b = bars[c][s["k"] % 2]
                if not b.done(s["hph"][s["k"] % 2]):
                    continue
            movable.append(t)
        if not movable:
            return f"deadlock at step {steps}"
        t = rng.choice(movable)
        s = th[t]
        c, q = t
        k = s["k"]
        nb = 1 - c
        try:
            if s["st"] == "read":
                got = halo[c][slot(k - 1)][q]
                if got != (nb, q, k - 1):
                    return f"thread {t} at jump {k} read {got}, expected the neighbour's row of jump {k - 1}"
                s["st"] = "send"
            elif s["st"] == "send":
                halo[nb][slot(k)][q] = (c, q, k)
                bars[nb][k % 2].complete_tx(ROW, k)
                s["st"] = "barrier"
                at_barrier[c].setdefault(k, set()).add(q)
            elif s["st"] == "barrier":
                if arm_early and q == 0 and k + 2 <= K:
                    bars[c][k % 2].arm(ROW * n, k + 2)  # before this jump's phase has completed
                s["st"] = "wait"
            elif s["st"] == "wait":
                par = k % 2
                s["hph"][par] ^= 1
                if q == 0 and k + 2 <= K and not arm_early:
                    bars[c][par].arm(ROW * n, k + 2)
                s["k"] = k + 1
                s["st"] = "read"
        except AssertionError as e:
            return f"thread {t} at jump {k}: {e}"
        steps += 1


@pytest.mark.parametrize("n", [1, 3, 5])
def test_handover_protocol_holds_under_random_schedules(n):
    for seed in range(300):
        err = run(n, 9, seed)
        assert err is None, (seed, err)


@pytest.mark.parametrize("mutation", [dict(slots=1), dict(wait=False), dict(arm_early=True)])
def test_handover_model_catches_broken_protocols(mutation):
    fails = [run(3, 9, seed, **mutation) for seed in range(300)]
    assert any(f is not None for f in fails), mutation
