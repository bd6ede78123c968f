"""The persistent SK sweep's cross-CTA protocol, modelled step by step on the CPU.

The persistent launch (one per sweep) has three kinds of actors: the helper warp of every
chain CTA (stages block b two ahead, publishes D_count once its replica warps are done with a
block), the replica warps of every chain CTA (wait for the staged block, fold the flips of the
blocks not yet in the staged fields, decide, write the ring slot b mod Q), and the issuer of
every field CTA (waits for D_count[k], reads the slot, releases D_free, applies block k to its
tiles, publishes a tile t once block t - L - 1 is applied).  The model runs these actors in
random interleavings with the kernel's waits as blocking conditions and checks:
  * the launch always finishes (no wait that nothing will satisfy),
  * the fields a chain block starts from, plus the blocks it folds in itself, are exactly the
    blocks before it, each once (the sequential order of the sweep),
  * a field CTA reads every ring slot before it is overwritten, and reads the block it expects.
Planted mistakes (no lookahead with a two-deep staging ring, a fold window one block short, no
D_free wait) are each caught.
"""
import random

import pytest


def run_protocol(nb, nC, nG, TPC, L, Q, S_C=2, seed=0, fold_short=False, skip_free=False,
                 max_steps=200000):
    rng = random.Random(seed)
    D_count = [0] * Q
    D_free = [0] * Q
    H_ready = [False] * nb
    slot = [None] * Q           # block held by each ring slot (per chain CTA: same schedule)
    slot_writes = [[0] * Q for _ in range(nC)]
    published = {}              # tile -> set of blocks applied when published
    tiles = {j: [t for t in (j + u * nG for u in range(TPC)) if t < nb] for j in range(nG)}
    applied = {t: set() for t in range(nb)}
    errors = []

    # chain CTA state: the helper runs its operations in program order, as the kernel does:
    # stage blocks 0 .. S_C - 1, then for every block b: publish D(b), stage b + S_C
    ops = [("stage", b) for b in range(min(S_C, nb))]
    for b in range(nb):
        ops.append(("publish", b))
        if b + S_C < nb:
            ops.append(("stage", b + S_C))
    helper_pc = [0] * nC
    staged = [dict() for _ in range(nC)]   # block -> fields (set of blocks included)
    chain_b = [0] * nC          # next block the replica warps process
    done_chain = [set() for _ in range(nC)]
    # field CTA state
    gemm_k = [0] * nG

    def helper_ready(c):
        if helper_pc[c] >= len(ops):
            return False
        op, b = ops[helper_pc[c]]
        if op == "publish":
            return b in done_chain[c]
        if b >= Q and not skip_free and D_free[b % Q] < (b // Q) * nG:
            return False
        return b <= L or H_ready[b]

    steps = 0
    while True:
        steps += 1
        if steps > max_steps:
            errors.append("step limit")
            break
        actions = []
        for c in range(nC):
            if helper_ready(c):
                actions.append(("helper", c))
            cb = chain_b[c]
            if cb < nb and cb in staged[c]:
                actions.append(("chain", c))
        for j in range(nG):
            k = gemm_k[j]
            if k < nb and D_count[k % Q] >= (k // Q + 1) * nC:
                actions.append(("gemm", j))
        if not actions:
            break
        kind, x = rng.choice(actions)
        if kind == "helper":
            op, b = ops[helper_pc[x]]
            if op == "publish":
                D_count[b % Q] += 1
            else:
                staged[x][b] = set() if b <= L else set(published[b])
            helper_pc[x] += 1
        elif kind == "chain":
            c, b = x, chain_b[x]
            fields = staged[c].pop(b)
            p0 = b - L if b > L else 0
            if fold_short and b > L:
                p0 += 1
            folded = set(range(p0, b))
            if fields & folded or (fields | folded) != set(range(b)):
                errors.append(f"chain {c} block {b}: fields {sorted(fields)} folded {sorted(folded)}")
            # write ring slot b mod Q
            s = b % Q
            if slot_writes[c][s] != b // Q:
                errors.append(f"chain {c}: slot {s} written out of order")
            slot_writes[c][s] += 1
            if c == 0:
                slot[s] = b
            done_chain[c].add(b)
            chain_b[c] += 1
        else:  # field CTA issuer
            j, k = x, gemm_k[x]
            if slot[k % Q] != k:
                errors.append(f"field CTA {j}: slot {k % Q} holds {slot[k % Q]}, expected block {k}")
            D_free[k % Q] += 1
            for t in tiles[j]:
                applied[t].add(k)
            for t in tiles[j]:
                if t == k + L + 1:
                    published[t] = set(applied[t])
                    H_ready[t] = True
            gemm_k[j] += 1
    finished = all(cb == nb for cb in chain_b) and all(k == nb for k in gemm_k)
    return finished, errors


CONFIGS = [
    # nb, nC, nG, TPC, L, Q
    (64, 64, 64, 1, 6, 8),    # N = 8192, R = 256
    (128, 32, 64, 2, 6, 8),   # N = 16384, R = 128
    (4, 4, 4, 1, 3, 8),       # N = 512: no tile is ever published (L >= nb - 1)
    (5, 8, 3, 2, 1, 2),       # smallest lookahead and ring
    (17, 3, 9, 2, 2, 3),      # ragged tile ownership
    (1, 4, 1, 1, 0, 8),       # one block
]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_protocol_finishes_and_keeps_the_sequential_order(cfg):
    nb, nC, nG, TPC, L, Q = cfg
    for seed in range(12):
        finished, errors = run_protocol(nb, nC, nG, TPC, L, Q, seed=seed)
        assert not errors, errors[:3]
        assert finished, f"deadlock with seed {seed}"


def test_no_lookahead_with_two_staged_blocks_deadlocks():
    finished, errors = run_protocol(8, 4, 4, 2, 0, 8, seed=1)
    assert not finished


def test_fold_window_one_block_short_is_caught():
    _, errors = run_protocol(16, 4, 8, 2, 3, 4, seed=2, fold_short=True)
    assert errors


def test_missing_ring_release_wait_is_caught():
    caught = False
    for seed in range(20):
        _, errors = run_protocol(24, 4, 8, 3, 6, 2, seed=seed, skip_free=True)
        caught |= any("holds" in e or "out of order" in e for e in errors)
    assert caught
