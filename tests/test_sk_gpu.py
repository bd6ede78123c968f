"""GPU parity of the Sherrington-Kirkpatrick kernels against the CPU oracle (bit-exact).

The blocked kernel (in-block sequential update + tcgen05 e4m3 field GEMM) and the plain kernel
must reproduce the oracle's sequential-order trajectory exactly: spins of every replica and every
C, q, E count.  Block size, padding and replica tiling must not change any result.
"""
import math

import numpy as np
import pytest

import oracle
import sg_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sg = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global sg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_11195_gb300 import _build
    _build.build()
    import paper_1906_11195_gb300 as m
    sg = m


def run_sk(J, temps, seed, kernel, block, sweeps, tw, tm):
    run = sg.SKRun(J, temps, seed, kernel=kernel, block=block, tw=tw, tm=tm)
    run.sweep(sweeps)
    run.synchronize()
    C, q, E = run.results()
    spins = run.spins()
    run.close()
    return spins, C[0, :, 0], q[0, :, 0], E[0, :, 0]


def check(J, temps, seed, sweeps, tw, tm, got, r_first=0, r_count=None):
    spins, C, q, E = got
    R = len(temps)
    rc = R - r_first if r_count is None else r_count
    ref = oracle.sk_run(J, temps, seed, sweeps, tw, tm, r_first=r_first, r_count=rc)
    sl = slice(r_first, r_first + rc)
    assert np.array_equal(spins[sl], ref["spins"])
    assert np.array_equal(C[sl], ref["C"])
    assert np.array_equal(E[sl], ref["E"])
    if rc >= 2:
        assert np.array_equal(q[r_first // 2:r_first // 2 + rc // 2], ref["q"])


@pytest.mark.parametrize("n,R,block", [(256, 32, 64), (300, 16, 128), (1000, 32, 256),
                                       (700, 48, 512), (129, 16, 64)])
def test_blocked_matches_oracle(n, R, block):
    J = sg_inputs.sk_couplings(n, 40 + n)
    temps = [0.4] * (R // 2) + [0.6] * (R // 2)
    tw, tm = sg_inputs.log_schedule([0, 3, 8], 24)
    got = run_sk(J, temps, 5 + n, sg.SG_SK_BLOCKED, block, 24, tw, tm)
    check(J, temps, 5 + n, 24, tw, tm, got)


@pytest.mark.parametrize("warps", [2, 4, 8])
@pytest.mark.parametrize("n,R,block", [(700, 16, 512), (300, 48, 128)])
def test_inblock_replica_split_matches_oracle(monkeypatch, warps, n, R, block):
    # replicas per in-block CTA (the blocked kernel takes R in multiples of 16)
    monkeypatch.setenv("SG_SK_INBLOCK_WARPS", str(warps))
    J = sg_inputs.sk_couplings(n, 70 + n)
    temps = [0.4 + 0.05 * r for r in range(R)]
    tw, tm = sg_inputs.log_schedule([0, 3], 16)
    got = run_sk(J, temps, 11 + warps, sg.SG_SK_BLOCKED, block, 16, tw, tm)
    check(J, temps, 11 + warps, 16, tw, tm, got)


@pytest.mark.parametrize("n,R", [(200, 8), (333, 5), (64, 2)])
def test_plain_matches_oracle(n, R):
    J = sg_inputs.sk_couplings(n, 60 + n)
    temps = [0.4 + 0.1 * r for r in range(R)]
    tw, tm = sg_inputs.log_schedule([0, 3], 16)
    got = run_sk(J, temps, 9, sg.SG_SK_PLAIN, 0, 16, tw, tm)
    check(J, temps, 9, 16, tw, tm, got)


def test_block_size_does_not_change_results():
    n, R = 640, 32
    J = sg_inputs.sk_couplings(n, 3)
    temps = [0.5] * R
    tw, tm = sg_inputs.log_schedule([0, 2], 12)
    outs = [run_sk(J, temps, 2, sg.SG_SK_BLOCKED, b, 12, tw, tm) for b in (64, 128, 256, 512)]
    outs.append(run_sk(J, temps, 2, sg.SG_SK_PLAIN, 0, 12, tw, tm))
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("T", [0.0, math.inf])
def test_zero_and_infinite_temperature(T):
    n, R = 384, 16
    J = sg_inputs.sk_couplings(n, 12)
    temps = [T] * R
    tw, tm = sg_inputs.log_schedule([0, 1], 10)
    got = run_sk(J, temps, 3, sg.SG_SK_BLOCKED, 128, 10, tw, tm)
    check(J, temps, 3, 10, tw, tm, got)


@pytest.mark.parametrize("R,block", [(1024, 512), (512, 128)])
def test_many_replicas_sharing_couplings(R, block):
    """Hundreds of replicas on one coupling matrix (several 128-replica tiles of the field GEMM
    and many in-block CTAs); replicas are independent chains, so the oracle follows a few of
    them, spread over the tiles."""
    n = 1000
    J = sg_inputs.sk_couplings(n, 91)
    temps = [0.4 + 0.2 * (r % 3) for r in range(R)]
    tw, tm = sg_inputs.log_schedule([0, 3], 12)
    got = run_sk(J, temps, 8, sg.SG_SK_BLOCKED, block, 12, tw, tm)
    for r0 in (0, 130, R // 2 + 4, R - 2):
        check(J, temps, 8, 12, tw, tm, got, r_first=r0, r_count=2)


def test_autotuned_block_with_512_padding():
    """n >= 2048 with block = 0: n is padded to a multiple of 512 and the autotuner may pick
    B = 512 (the ragged last block holds padding spins that never flip)."""
    n, R = 2100, 32
    J = sg_inputs.sk_couplings(n, 77)
    temps = [0.4] * (R // 2) + [0.8] * (R // 2)
    tw, tm = sg_inputs.log_schedule([0, 2], 10)
    got = run_sk(J, temps, 6, sg.SG_SK_BLOCKED, 0, 10, tw, tm)
    check(J, temps, 6, 10, tw, tm, got)


def test_thresholds_exported_match_oracle():
    n = 512
    J = sg_inputs.sk_couplings(n, 1)
    temps = [0.4] * 8 + [0.6] * 8
    run = sg.SKRun(J, temps, 1, kernel=sg.SG_SK_BLOCKED, block=128)
    thr = run.thresholds()
    assert np.array_equal(thr[0], oracle.sk_thresholds(0.4, n))
    assert np.array_equal(thr[15], oracle.sk_thresholds(0.6, n))
    run.close()


def test_checkpoint_resume_is_bit_exact():
    n, R = 512, 16
    J = sg_inputs.sk_couplings(n, 21)
    temps = [0.4] * R
    tw, tm = sg_inputs.log_schedule([0, 4], 30)
    straight = run_sk(J, temps, 4, sg.SG_SK_BLOCKED, 128, 30, tw, tm)
    run = sg.SKRun(J, temps, 4, kernel=sg.SG_SK_BLOCKED, block=128, tw=tw, tm=tm)
    run.sweep(11)
    blob = run.save_state()
    run.close()
    run2 = sg.SKRun(J, temps, 4, kernel=sg.SG_SK_BLOCKED, block=128, tw=tw, tm=tm)
    run2.load_state(blob)
    run2.sweep(19)
    C, q, E = run2.results()
    assert np.array_equal(run2.spins(), straight[0])
    assert np.array_equal(C[0, :, 0], straight[1]) and np.array_equal(E[0, :, 0], straight[3])
    run2.close()


# --------------------------------------------------------------------------------------------
# full-size workload: N = 8192, 256 replicas sharing J, T = 0.4, B = 128 (configured) and 512
# --------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def sk_big():
    return sg_inputs.sk_couplings(8192, 3)


@pytest.mark.parametrize("block", [128, 512])
def test_full_size_matches_oracle_on_sampled_replicas(sk_big, block):
    J = sk_big
    R, sweeps = 256, 12
    temps = [0.4] * R
    tw, tm = sg_inputs.log_schedule([0, 3, 8], sweeps)
    got = run_sk(J, temps, 1, sg.SG_SK_BLOCKED, block, sweeps, tw, tm)
    # replicas are independent chains: the oracle follows a few of them one by one
    for r0 in (0, 2, 126, 254):
        check(J, temps, 1, sweeps, tw, tm, got, r_first=r0, r_count=2)
    spins, C, q, E = got
    assert np.all(np.abs(C) <= 8192) and np.all((C - 8192) % 2 == 0)


def test_batched_uneven_samples_with_autotuned_blocks():
    """Uneven SK samples in one handle (one graph branch per sample), block chosen by the
    autotuner (block = 0), T = 0.4 and 0.6 replicas; every sample equals its own oracle run."""
    sizes = [int(x) for x in sg_inputs.log_uniform_sizes(5, 7, 10.5, 9)]
    R = 32
    samples = []
    for k, n in enumerate(sizes):
        samples.append(dict(J=sg_inputs.sk_couplings(n, 900 + k), seed=50 + k,
                            temps=[0.4] * (R // 2) + [0.6] * (R // 2)))
    tw, tm = sg_inputs.log_schedule([0, 3], 20)
    run = sg.SKBatchRun(samples, R, kernel=sg.SG_SK_BLOCKED, block=0, tw=tw, tm=tm)
    run.sweep(20)
    run.synchronize()
    C, q, E = run.results()
    spins = run.spins()
    run.close()
    for b, x in enumerate(samples):
        ref = oracle.sk_run(x["J"], x["temps"], x["seed"], 20, tw, tm)
        assert np.array_equal(spins[b], ref["spins"]), b
        assert np.array_equal(C[b, :, 0], ref["C"]) and np.array_equal(E[b, :, 0], ref["E"])
        assert np.array_equal(q[b, :, 0], ref["q"])


def test_set_schedule_after_attach_matches_oracle():
    """sg_set_schedule on an attached SK handle before any scheduled time: the new times give
    exactly the oracle's measurements."""
    n, R = 600, 32
    J = sg_inputs.sk_couplings(n, 44)
    temps = [0.4] * (R // 2) + [0.6] * (R // 2)
    run = sg.SKRun(J, temps, 9, kernel=sg.SG_SK_BLOCKED, block=128, tw=[5, 6], tm=[7, 8, 9])
    run.sweep(1)
    tw, tm = [2, 4], [2, 6, 11]
    run.set_schedule(tw, tm)
    run.sweep(10)
    C, q, E = run.results()
    spins = run.spins()
    run.close()
    check(J, temps, 9, 11, tw, tm, (spins, C[0, :, 0], q[0, :, 0], E[0, :, 0]))


def test_batch_with_large_samples_and_autotuned_blocks_matches_oracle():
    """The uneven SK batch at its large end: samples with n >= 2048 (padded to a multiple of 512,
    where the autotuner may pick B = 512 and the last block is ragged) up to the batch's largest
    size n = 16384, next to small ones, R = 128 (64 at T = 0.4, 64 at T = 0.6), block = 0; the
    oracle follows sampled replica pairs of every sample (both temperatures)."""
    from oracle_pool import run_parallel
    sizes = [600, 2100, 3000, 5000, 16384]
    R = 128
    samples = [dict(J=sg_inputs.sk_couplings(n, 1300 + n), seed=70 + k,
                    temps=[0.4] * (R // 2) + [0.6] * (R // 2)) for k, n in enumerate(sizes)]
    sweeps = 8
    tw, tm = sg_inputs.log_schedule([0, 3], sweeps)
    run = sg.SKBatchRun(samples, R, kernel=sg.SG_SK_BLOCKED, block=0, tw=tw, tm=tm)
    run.sweep(sweeps)
    run.synchronize()
    C, q, E = run.results()
    spins = run.spins()
    run.close()
    pairs = (0, 62, 64, 126)
    jobs = [("sk_run", (x["J"], x["temps"], x["seed"], sweeps, tw, tm),
             dict(r_first=r0, r_count=2)) for x in samples for r0 in pairs]
    refs = run_parallel(jobs)
    for b in range(len(samples)):
        for j, r0 in enumerate(pairs):
            ref = refs[b * len(pairs) + j]
            sl = slice(r0, r0 + 2)
            assert np.array_equal(spins[b][sl], ref["spins"]), (b, r0)
            assert np.array_equal(C[b, sl, 0], ref["C"]) and np.array_equal(E[b, sl, 0], ref["E"])
            assert np.array_equal(q[b, r0 // 2:r0 // 2 + 1, 0], ref["q"])


# --------------------------------------------------------------------------------------------
# persistent sweep (B = 128, replicas a multiple of 32): one cooperative launch per sweep
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n,R,temps", [
    (1000, 32, None), (2000, 64, None), (4100, 128, None), (700, 96, None),
    (384, 32, 0.0), (1024, 32, math.inf), (129, 32, None)])
def test_persistent_sweep_matches_oracle(n, R, temps):
    J = sg_inputs.sk_couplings(n, 500 + n)
    if temps is None:
        temps = [0.4] * (R // 2) + [0.6] * (R // 2)
    else:
        temps = [temps] * R
    tw, tm = sg_inputs.log_schedule([0, 2, 5], 14)
    got = run_sk(J, temps, 31 + n, sg.SG_SK_BLOCKED, 128, 14, tw, tm)
    r_count = None if R <= 64 else 4
    for r0 in ((0,) if R <= 64 else (0, R // 2, R - 4)):
        check(J, temps, 31 + n, 14, tw, tm, got, r_first=r0, r_count=r_count)


@pytest.mark.parametrize("lookahead", ["4", "6", "8"])
def test_persistent_lookahead_and_fallback_give_the_same_results(monkeypatch, lookahead):
    """The lookahead L (blocks of flips a chain warp folds in itself before the tensor cores
    catch up) and the launch-per-block sequence (SG_SK_PERSISTENT=0) never change a result."""
    n, R = 1800, 64
    J = sg_inputs.sk_couplings(n, 17)
    temps = [0.5] * R
    tw, tm = sg_inputs.log_schedule([0, 3], 12)
    monkeypatch.setenv("SG_SK_LOOKAHEAD", lookahead)
    a = run_sk(J, temps, 4, sg.SG_SK_BLOCKED, 128, 12, tw, tm)
    monkeypatch.setenv("SG_SK_PERSISTENT", "0")
    b = run_sk(J, temps, 4, sg.SG_SK_BLOCKED, 128, 12, tw, tm)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("T", [math.inf, 0.4])
def test_persistent_full_size_matches_oracle(sk_big, T):
    """N = 8192 with 256 replicas (the configured workload's shape).  At T = inf every spin
    flips every sweep, so a sweep moves each field by up to 2N: the tensor-memory accumulators
    must stay exact far from zero."""
    J = sk_big
    R, sweeps = 256, 6
    temps = [T] * R
    tw, tm = sg_inputs.log_schedule([0, 2], sweeps)
    got = run_sk(J, temps, 2, sg.SG_SK_BLOCKED, 128, sweeps, tw, tm)
    for r0 in (0, 100, 254):
        check(J, temps, 2, sweeps, tw, tm, got, r_first=r0, r_count=2)
