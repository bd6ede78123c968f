"""The persistent SK sweep's cross-CTA protocol, modelled step by step on the CPU.

The persistent launch has four kinds of actors: the staging warp of every chain CTA (stages
block k + S_C once its replica and fold warps are done with block k), the release warp of every
chain CTA (adds to D_count[k] once its replica warps have written block k, in block order), the
replica warps of every chain CTA (wait for the staged block, fold the flips of the blocks not
yet in the staged fields, decide, write the ring slot k mod Q), and the issuer of every field CTA
(waits for D_count[k], reads the slot, releases D_free, applies block k to its tiles, publishes
a tile t once block t - L - 1 is applied).  The model runs these actors in
random interleavings with the kernel's waits as blocking conditions and checks:
  * the launch always finishes (no wait that nothing will satisfy),
  * the fields a chain block starts from, plus the blocks it folds in itself, are exactly the
    blocks before it, each once (the sequential order of the sweep),
  * a field CTA reads every ring slot before it is overwritten, and reads the block it expects.
Several sweeps run in one launch (blocks k = s nb + b; the fold window and the publishes run
across sweep boundaries).  Planted mistakes (a fold window one block short, no D_free wait) are
each caught, and so are the deadlocks of the earlier form in which the staging warp itself
released D_count (no lookahead; a ring shallower than the staging).
"""
import random

import pytest


def run_protocol(nb, nC, nG, TPC, L, Q, S_C=2, n_sweeps=1, seed=0, fold_short=False,
                 skip_free=False, release_in_staging=False, max_steps=400000):
    """One launch of n_sweeps sweeps; blocks are numbered k = s nb + b over the launch."""
    rng = random.Random(seed)
    nk = n_sweeps * nb
    D_count = [0] * Q
    D_free = [0] * Q
    H_ready = [0] * nb          # chain block + 1 of the latest publish of each tile
    slot = [None] * Q           # block held by each ring slot (per chain CTA: same schedule)
    slot_writes = [[0] * Q for _ in range(nC)]
    published = {}              # tile -> set of blocks applied when published
    tiles = {j: [t for t in (j + u * nG for u in range(TPC)) if t < nb] for j in range(nG)}
    applied = {t: set() for t in range(nb)}
    errors = []

    # chain CTA state: the staging warp runs its operations in program order, as the kernel
    # does: stage blocks 0 .. S_C - 1, then for every block k: wait until block k is done
    # ("free"), stage k + S_C; the release warp publishes D(k) in block order once block k is done
    # (release_in_staging: the earlier form, the staging warp itself publishing D(k) in its
    # program order, after block k is done and before it stages k + S_C)
    ops = [("stage", k) for k in range(min(S_C, nk))]
    for k in range(nk):
        ops.append(("publish" if release_in_staging else "free", k))
        if k + S_C < nk:
            ops.append(("stage", k + S_C))
    helper_pc = [0] * nC
    released = [0] * nC         # next block each release warp publishes
    staged = [dict() for _ in range(nC)]   # block -> fields (set of blocks included)
    chain_k = [0] * nC          # next block the replica warps process
    done_chain = [set() for _ in range(nC)]
    # field CTA state: the MMA issuer walks the blocks
    gemm_k = [0] * nG

    def helper_ready(c):
        if helper_pc[c] >= len(ops):
            return False
        op, k = ops[helper_pc[c]]
        if op in ("free", "publish"):
            return k in done_chain[c]
        b = k % nb
        if k >= Q and not skip_free and D_free[k % Q] < (k // Q) * nG:
            return False
        return k <= L or H_ready[b] >= k + 1

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
            if not release_in_staging and released[c] < nk and released[c] in done_chain[c]:
                actions.append(("release", c))
            ck = chain_k[c]
            if ck < nk and ck in staged[c]:
                actions.append(("chain", c))
        for j in range(nG):
            k = gemm_k[j]
            if k < nk and D_count[k % Q] >= (k // Q + 1) * nC:
                actions.append(("gemm", j))
        if not actions:
            break
        kind, x = rng.choice(actions)
        if kind == "helper":
            op, k = ops[helper_pc[x]]
            if op == "stage":
                staged[x][k] = set() if k <= L else set(published[k % nb])
            elif op == "publish":
                D_count[k % Q] += 1
            helper_pc[x] += 1
        elif kind == "release":
            D_count[released[x] % Q] += 1
            released[x] += 1
        elif kind == "chain":
            c, k = x, chain_k[x]
            fields = staged[c].pop(k)
            p0 = max(0, k - L)
            if fold_short and k > L:
                p0 += 1
            folded = set(range(p0, k))
            if fields & folded or (fields | folded) != set(range(k)):
                errors.append(f"chain {c} block {k}: fields {sorted(fields)} folded {sorted(folded)}")
            s = k % Q
            if slot_writes[c][s] != k // Q:
                errors.append(f"chain {c}: slot {s} written out of order")
            slot_writes[c][s] += 1
            if c == 0:
                slot[s] = k
            done_chain[c].add(k)
            chain_k[c] += 1
        else:  # field CTA issuer
            j, k = x, gemm_k[x]
            if slot[k % Q] != k:
                errors.append(f"field CTA {j}: slot {k % Q} holds {slot[k % Q]}, expected block {k}")
            D_free[k % Q] += 1
            b = k % nb
            for t in tiles[j]:
                applied[t].add(k)  # block k (block b of its sweep) reaches every tile
            kc = k + L + 1
            if kc < nk and kc % nb in tiles[j]:
                published[kc % nb] = set(applied[kc % nb])
                H_ready[kc % nb] = kc + 1
            gemm_k[j] += 1
    finished = all(ck == nk for ck in chain_k) and all(k == nk for k in gemm_k)
    return finished, errors


CONFIGS = [
    # nb, nC, nG, TPC, L, Q, sweeps, staged blocks
    (64, 64, 64, 1, 4, 8, 1, 3),    # N = 8192, R = 256, one sweep (the kernel's ring: 3)
    (64, 64, 64, 1, 6, 8, 3, 3),    # the same, three sweeps in one launch
    (128, 32, 64, 2, 4, 8, 2, 3),   # N = 16384, R = 128
    (7, 8, 3, 3, 6, 8, 4, 3),       # L = nb - 1: the largest window
    (5, 8, 3, 2, 2, 3, 3, 3),       # smallest lookahead and ring (Q >= staged blocks)
    (17, 3, 9, 2, 4, 3, 2, 2),      # ragged tile ownership, two staged blocks
]


@pytest.mark.parametrize("cfg", CONFIGS)
def test_protocol_finishes_and_keeps_the_sequential_order(cfg):
    nb, nC, nG, TPC, L, Q, S, S_C = cfg
    for seed in range(8):
        finished, errors = run_protocol(nb, nC, nG, TPC, L, Q, S_C=S_C, n_sweeps=S, seed=seed)
        assert not errors, errors[:3]
        assert finished, f"deadlock with seed {seed}"


def test_no_lookahead_deadlocks_when_the_staging_warp_releases():
    """The earlier form (the staging warp publishing D(k) itself, in program order): staging
    block k + 2 waits for fields that need block k + 1 applied, whose release comes after that
    staging.  The release warp breaks the cycle."""
    finished, _ = run_protocol(8, 4, 4, 2, 0, 8, seed=1, release_in_staging=True)
    assert not finished
    finished, errors = run_protocol(8, 4, 4, 2, 0, 8, seed=1)
    assert finished and not errors


def test_fold_window_one_block_short_is_caught():
    _, errors = run_protocol(16, 4, 8, 2, 3, 4, n_sweeps=2, seed=2, fold_short=True)
    assert errors


def test_missing_ring_release_wait_is_caught():
    caught = False
    for seed in range(20):
        _, errors = run_protocol(24, 4, 8, 3, 6, 2, seed=seed, skip_free=True)
        caught |= any("holds" in e or "out of order" in e for e in errors)
    assert caught


def test_ring_smaller_than_the_staging_depth_deadlocks_when_the_staging_warp_releases():
    """Earlier form: staging block k + S_C waits for ring slot k + S_C - Q to be read, but that
    block's spin changes were published only after the staging; with the release warp the
    launch finishes (the kernel keeps Q = 8 >= three staged blocks all the same)."""
    finished, _ = run_protocol(5, 8, 3, 2, 2, 2, S_C=3, n_sweeps=3, seed=0, release_in_staging=True)
    assert not finished
    for seed in range(6):
        finished, errors = run_protocol(5, 8, 3, 2, 2, 2, S_C=3, n_sweeps=3, seed=seed)
        assert finished and not errors
