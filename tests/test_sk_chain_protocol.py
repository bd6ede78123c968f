"""The persistent SK sweep's waits inside one chain CTA, modelled step by step on the CPU.

`k_sk_persist` (paper_1906_11195_gb300/csrc/sk_persist.cu) runs, in every chain CTA, a staging
warp (stages block k + S ahead into a ring of S stages: an mbarrier `fullc` per stage with an
expected byte count, released through `emptyc` by every replica and fold warp), W replica
warps (wait for the stage and for their fold warp's hand-over `hrdy`, decide, write the
block's spin changes, count `done_cnt`, arrive on `cdone` and `emptyc`), W fold warps (wait
for the stage and for their replica warp's `cdone` of block k - 2, fold blocks k - L .. k - 2
into the fields, write the hand-over buffer of block parity k & 1, arrive on `hrdy` and
`emptyc`) and a release warp (tells the field CTAs once every replica warp has written a
block).  The field CTAs are one actor here: they apply block k once it is released and publish
the fields a block needs (block k needs every block before k - L applied) and free ring slots.
The model runs the actors in random interleavings with the kernel's mbarrier phases and checks:
  * every parity wait is unambiguous (the barrier is in the awaited phase or the next one),
  * a stage is refilled only after all 2W warps released its previous block, and every warp
    reads the block it expects from it,
  * a replica warp reads the hand-over of its own block, which the fold warp wrote after the
    replica warp had read the previous one in that buffer,
  * a fold warp folds only blocks its replica warp has finished,
  * the launch always finishes.
Planted mistakes (a single hand-over buffer, `emptyc` counting only the replica warps, the
`cdone` phase taken from the block's parity instead of its pair index) are each caught.
"""
import random
import re

import pytest


class ProtocolError(AssertionError):
    pass


class MBar:
    def __init__(self, count):
        self.count, self.pending, self.tx, self.phase = count, count, 0, 0

    def _step(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def arrive(self):
        self.pending -= 1
        self._step()

    def arrive_expect_tx(self, nbytes):
        self.tx += nbytes
        self.arrive()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        self._step()

    def done(self, phase_index):
        if not (phase_index <= self.phase <= phase_index + 1):
            raise ProtocolError(f"ambiguous parity wait: barrier at phase {self.phase}, "
                                f"waiting for {phase_index}")
        return (self.phase & 1) != (phase_index & 1)


def run_chain_cta(W, S, L, nk, seed, mutant=None, max_steps=300000):
    """One chain CTA of W replicas over nk blocks (S staged blocks, lookahead L); returns when
    every actor finished, raises ProtocolError otherwise."""
    rng = random.Random(seed)
    fullc = [MBar(1) for _ in range(S)]
    emptyc = [MBar(W if mutant == "emptyc_counts_replicas_only" else 2 * W) for _ in range(S)]
    nbuf = 1 if mutant == "single_handover_buffer" else 2
    cdone = [[MBar(1) for _ in range(2)] for _ in range(W)]
    hrdy = [[MBar(1) for _ in range(nbuf)] for _ in range(W)]
    stage = [None] * S                      # block held by each stage (None while landing)
    stage_users = [set() for _ in range(S)]  # warps that have not released the stage yet
    hb = [[None] * nbuf for _ in range(W)]   # block whose folded fields each buffer holds
    hb_read = [[True] * nbuf for _ in range(W)]
    chain_done = [-1] * W                    # latest block each replica warp finished
    done_cnt = [0] * W
    released = [0]                           # blocks released to the field CTAs
    applied = [0]                            # blocks the field CTAs applied
    events = []

    def staging():
        def prefetch(k):
            s = k % S
            # field side: the block's fields hold every block before k - L (published after
            # block k - L - 1 is applied) and ring slots are freed as blocks are applied
            yield lambda: applied[0] >= k - L
            if stage_users[s]:
                raise ProtocolError(f"stage {s} refilled for block {k} while in use")
            stage[s] = None
            stage_users[s] = {("chain", w) for w in range(W)} | {("fold", w) for w in range(W)}
            fullc[s].arrive_expect_tx(1)

            def land(s=s, k=k):
                stage[s] = k
                fullc[s].complete_tx(1)
            events.append(land)
        for k in range(min(S, nk)):
            yield from prefetch(k)
        for k in range(nk):
            yield lambda k=k: emptyc[k % S].done(k // S)
            if k + S < nk:
                yield from prefetch(k + S)

    def replica(w):
        for k in range(nk):
            s = k % S
            yield lambda k=k, s=s: fullc[s].done(k // S)
            yield lambda k=k: hrdy[w][k % nbuf].done(k // nbuf)
            if stage[s] != k:
                raise ProtocolError(f"replica {w}: stage {s} holds {stage[s]}, expected {k}")
            b = k % nbuf
            if hb[w][b] != k:
                raise ProtocolError(f"replica {w}: hand-over buffer holds {hb[w][b]}, expected {k}")
            hb_read[w][b] = True
            chain_done[w] = k
            done_cnt[w] = k + 1
            cdone[w][k & 1].arrive()
            stage_users[s].discard(("chain", w))
            emptyc[s].arrive()

    def fold(w):
        for k in range(nk):
            s = k % S
            yield lambda k=k, s=s: fullc[s].done(k // S)
            if k >= 2:
                ph = (k - 2) & 1 if mutant == "cdone_phase_from_parity" else (k - 2) >> 1
                yield lambda k=k, ph=ph: cdone[w][k & 1].done(ph)
            if stage[s] != k:
                raise ProtocolError(f"fold {w}: stage {s} holds {stage[s]}, expected {k}")
            if chain_done[w] < k - 2:
                raise ProtocolError(f"fold {w}: block {k - 2} folded before its replica warp finished it")
            b = k % nbuf
            if not hb_read[w][b]:
                raise ProtocolError(f"fold {w}: hand-over of block {hb[w][b]} overwritten before it was read")
            hb[w][b] = k
            hb_read[w][b] = False
            hrdy[w][b].arrive()
            stage_users[s].discard(("fold", w))
            emptyc[s].arrive()

    def release():
        for k in range(nk):
            yield lambda k=k: all(c >= k + 1 for c in done_cnt)
            released[0] = k + 1

    def field():
        for k in range(nk):
            yield lambda k=k: released[0] >= k + 1
            applied[0] = k + 1

    actors = [staging(), release(), field()] + [replica(w) for w in range(W)] + \
             [fold(w) for w in range(W)]
    waits = [None] * len(actors)
    live = set(range(len(actors)))

    def advance(i):
        try:
            return next(actors[i])
        except StopIteration:
            live.discard(i)
            return None

    for i in list(live):
        waits[i] = advance(i)
    for _ in range(max_steps):
        if not live and not events:
            return
        runnable = [i for i in live if waits[i] is None or waits[i]()]
        choices = runnable + (["event"] if events else [])
        if not choices:
            raise ProtocolError("deadlock: every warp waits and no copy is in flight")
        pick = rng.choice(choices)
        if pick == "event":
            events.pop(rng.randrange(len(events)))()
        else:
            waits[pick] = advance(pick)
    raise ProtocolError("step limit reached")


@pytest.mark.parametrize("W", [1, 4, 8])
@pytest.mark.parametrize("L", [4, 6, 8])
def test_chain_cta_waits_are_consistent_and_finish(W, L):
    for seed in range(6):
        run_chain_cta(W, S=3, L=L, nk=40, seed=seed)


@pytest.mark.parametrize("mutant,match", [
    ("single_handover_buffer", "overwritten|holds|ambiguous|deadlock"),
    ("emptyc_counts_replicas_only", "refilled|holds|ambiguous"),
    ("cdone_phase_from_parity", "ambiguous|folded before|deadlock"),
])
def test_planted_chain_mistakes_are_caught(mutant, match):
    caught = 0
    for seed in range(30):
        try:
            run_chain_cta(4, S=3, L=6, nk=40, seed=seed, mutant=mutant)
        except ProtocolError as e:
            assert re.search(match, str(e)), str(e)
            caught += 1
    assert caught > 0
