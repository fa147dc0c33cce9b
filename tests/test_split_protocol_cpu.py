"""Model check of the message protocol of the cluster-split local solve (k_local_split.cu).

Two CTAs share one subdomain of nb block rows; CTA 1 owns the chunks whose tiles lie at
least T rows below the diagonal.  Messages travel through rings of D slots, each slot
guarded by an mbarrier whose phase completes once per message (32 lane arrivals):
  forward:  CTA 1 -> CTA 0 partial of row b   (slot b mod D, the wait expects parity (b div D) mod 2)
            CTA 0 -> CTA 1 v_b, b <= nb-1-T   (slot b mod D)
  backward: CTA 0 -> CTA 1 x_b                (slot o mod D, o = nb-1-b: the message's place)
            CTA 1 -> CTA 0 update of block j  (slot o mod D, o = nb-1-j), sent after row
                                              j + T, or at the start when j + T > nb-1.
The model replays each CTA's sends and waits in the kernel's order under random
interleavings and checks, for every wait, that the barrier has completed exactly the
phase it expects (a phase completed twice would hang the wait or hand it the next
message), that no data slot is overwritten before its reader took it, and that no
interleaving deadlocks.  It also checks that the two alternatives the design rules out
fail: backward slots indexed by the block instead of its place in the sweep, and a
ring smaller than the lag T (the protocol needs D >= T; the kernel keeps D = 2 T).
"""
import random

import pytest


class Ring:
    def __init__(self, D):
        self.D = D
        self.arrived = [0] * D      # completed phases per slot
        self.taken = [0] * D        # messages the receiver has taken per slot

    def send(self, slot, seq):
        if self.arrived[slot] != seq:
            raise AssertionError(f"slot {slot}: message {seq} sent after {self.arrived[slot]} arrivals")
        if self.taken[slot] != seq:
            raise AssertionError(f"slot {slot}: message {seq} overwrites an unread one")
        self.arrived[slot] += 1

    def ready(self, slot, seq):
        # mbarrier.try_wait.parity(seq mod 2) succeeds once the phase count's parity differs
        return (self.arrived[slot] & 1) != (seq & 1)

    def take(self, slot, seq):
        if self.arrived[slot] != seq + 1:
            raise AssertionError(f"slot {slot}: wait for message {seq} saw {self.arrived[slot]} arrivals")
        self.taken[slot] += 1


def programs(nb, T, D, ordinal=True):
    """The two CTAs' message operations, in program order: ('send'|'wait', ring, slot, seq)."""
    def place(b, sweep):
        o = b if sweep == 0 or not ordinal else nb - 1 - b
        return o % D, o // D

    c0, c1 = [], []
    for b in range(nb):                       # forward
        if b - T >= 0:
            c1.append(("wait", "v", *place(b - T, 0)))
        c1.append(("send", "p", *place(b, 0)))
        c0.append(("wait", "p", *place(b, 0)))
        if b <= nb - 1 - T:
            c0.append(("send", "v", *place(b, 0)))
    for j in range(nb - 1, -1, -1):           # backward: blocks CTA 1 never updates
        if j + T > nb - 1:
            c1.append(("send", "d", *place(j, 1)))
    for b in range(nb - 1, -1, -1):
        c0.append(("wait", "d", *place(b, 1)))
        c0.append(("send", "x", *place(b, 1)))
        c1.append(("wait", "x", *place(b, 1)))
        if b - T >= 0:
            c1.append(("send", "d", *place(b - T, 1)))
    return c0, c1


def run(nb, T, D, seed, ordinal=True):
    rings = {k: Ring(D) for k in "pvdx"}
    # v is written straight into the peer's vector: only its barrier phases matter
    rings["v"].taken = None
    progs = programs(nb, T, D, ordinal)
    pc = [0, 0]
    rng = random.Random(seed)
    while pc[0] < len(progs[0]) or pc[1] < len(progs[1]):
        enabled = []
        for c in (0, 1):
            if pc[c] < len(progs[c]):
                op, ring, slot, seq = progs[c][pc[c]]
                if op == "send" or rings[ring].ready(slot, seq):
                    enabled.append(c)
        if not enabled:
            raise AssertionError(f"deadlock at {pc}")
        c = rng.choice(enabled)
        op, ring, slot, seq = progs[c][pc[c]]
        r = rings[ring]
        if op == "send":
            if r.taken is None:  # the v barrier: only the arrival count
                if r.arrived[slot] != seq:
                    raise AssertionError(f"v slot {slot}: publish {seq} after {r.arrived[slot]}")
                r.arrived[slot] += 1
            else:
                r.send(slot, seq)
        else:
            if r.taken is None:
                if r.arrived[slot] != seq + 1:
                    raise AssertionError(f"v slot {slot}: wait for {seq} saw {r.arrived[slot]} publishes")
            else:
                r.take(slot, seq)
        pc[c] += 1


@pytest.mark.parametrize("nb", [1, 2, 7, 8, 9, 16, 17, 40, 61])
def test_protocol_holds(nb):
    T, D = 8, 16  # the kernel's constants: 256-column chunks of 32-column tiles, a ring of 16 rows
    for seed in range(60):
        run(nb, T, D, seed)


def test_forward_indexing_of_backward_slots_fails():
    with pytest.raises(AssertionError):
        for seed in range(60):
            run(45, 8, 16, seed, ordinal=False)


def test_ring_smaller_than_the_lag_fails():
    for seed in range(60):
        run(40, 8, 8, seed)  # D = T holds
    with pytest.raises(AssertionError):
        for seed in range(200):
            run(40, 8, 7, seed)
