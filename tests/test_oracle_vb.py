"""Pin the Viana-Bray oracle against things other than itself.

* Brute force: an independent Python restatement that takes each single-spin Metropolis
  decision from the full Hamiltonian H = -sum_{(ij)} J_ij s_i s_j (Eq. 3), i.e. from
  H(s with s_i flipped) - H(s), with acceptance thresholds computed in arbitrary precision and
  its own colouring (greedy, then one recolouring pass).  Trajectories must agree bit for bit.
* Exact Boltzmann enumeration on N = 6: the long-run state histogram of the oracle's chain.
* T = 0 (energy never rises) and T = infinity (every spin flips every sweep) limits.
* Measurements: C(t_w, t_w) = N, |C| <= N, C = N (mod 2), energies recomputed from spins.
* The high-temperature energy of a sparse random graph, e = -(M/N) tanh(beta).
"""
import math

import mpmath
import numpy as np
import pytest

import oracle
import sg_inputs

mpmath.mp.dps = 50


def thr_exact(beta, dE):
    if dE <= 0:
        return None
    if math.isinf(beta):
        return 0
    v = mpmath.mpf(2) ** 32 * mpmath.e ** (-mpmath.mpf(beta) * dE)
    return min(0xFFFFFFFF, int(mpmath.floor(v)))


def philox_word(seed, c, word):
    return int(oracle.philox4x32_10(c, [seed & 0xFFFFFFFF, seed >> 32])[word])


def energy_lanes(rp, col, jbits, s):
    """Integer sum over undirected edges of J s_i s_j, per lane; s int8[L][N]."""
    n = len(rp) - 1
    L = s.shape[0]
    tot = np.zeros(L, dtype=np.int64)
    lanes = np.arange(L, dtype=np.uint64)
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            j = col[e]
            if j > i:
                J = 1 - 2 * ((np.uint64(jbits[e]) >> lanes) & np.uint64(1)).astype(np.int64)
                tot += J * s[:, i] * s[:, j]
    return tot


def unpack(words, L):
    """uint64[N] -> int8[L][N] spins (bit 1 -> -1)."""
    lanes = np.arange(L, dtype=np.uint64)
    bits = (words[None, :].astype(np.uint64) >> lanes[:, None]) & np.uint64(1)
    return (1 - 2 * bits.astype(np.int64)).astype(np.int8)


def brute_vb(rp, col, jbits, L, temps, seed, n_sweeps):
    n = len(rp) - 1
    R = len(temps)
    colour = [-1] * n
    for i in range(n):
        used = {colour[j] for j in col[rp[i]:rp[i + 1]] if colour[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    # one recolouring pass: greedy again over (decreasing colour, increasing label)
    fresh = [-1] * n
    for i in sorted(range(n), key=lambda i: (-colour[i], i)):
        used = {fresh[j] for j in col[rp[i]:rp[i + 1]] if fresh[j] >= 0}
        c = 0
        while c in used:
            c += 1
        fresh[i] = c
    colour = fresh
    order = sorted(range(n), key=lambda i: (colour[i], i))
    s = np.zeros((R, L, n), dtype=np.int8)
    for r in range(R):
        for i in range(n):
            w = philox_word(seed, [i, 0, r, 1], 0) | (philox_word(seed, [i, 0, r, 1], 1) << 32)
            for k in range(L):
                s[r, k, i] = -1 if (w >> k) & 1 else 1
    traj = [s.copy()]
    for t in range(n_sweeps):
        for i in order:
            for r in range(R):
                beta = 1.0 / temps[r] if temps[r] != 0 else math.inf
                r32 = philox_word(seed, [i, t, r // 4, 0], r % 4)
                H0 = -energy_lanes(rp, col, jbits, s[r])
                s2 = s[r].copy()
                s2[:, i] = -s2[:, i]
                H1 = -energy_lanes(rp, col, jbits, s2)
                for k in range(L):
                    dE = int(H1[k] - H0[k])
                    th = thr_exact(beta, dE)
                    if th is None or r32 < th:
                        s[r, k, i] = -s[r, k, i]
        traj.append(s.copy())
    return np.array(traj)


@pytest.mark.parametrize("n,c,gseed,L,temps,seed", [
    (9, 3.0, 11, 5, [0.7, 1.0, 2.0, 0.45, 1.3], 99),
    (12, 4.0, 12, 3, [1.0, 1.0], 2**40 + 5),
    (7, 1.5, 13, 64, [0.9], 7),
])
def test_vb_oracle_matches_brute_force(n, c, gseed, L, temps, seed):
    rp, col, eid = sg_inputs.poisson_graph(n, c, gseed)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1 if eid.size else 0, gseed)
    sweeps = 5
    res = oracle.vb_run(rp, col, jb, L, temps, seed, sweeps, trajectory=True)
    want = brute_vb(rp, col, jb, L, temps, seed, sweeps)
    got = np.array([[unpack(res["traj"][t, r], L) for r in range(len(temps))]
                    for t in range(sweeps + 1)])
    assert np.array_equal(got, want)


def test_vb_measurements_and_invariants():
    rp, col, eid = sg_inputs.poisson_graph(300, 4.0, 21)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 21)
    L, temps, seed, sweeps = 64, [0.8, 0.8, 1.5, 1.5], 5, 40
    tw = [0, 1, 4, 16]
    tm = [0, 1, 2, 4, 5, 8, 16, 17, 20, 32, 40]
    res = oracle.vb_run(rp, col, jb, L, temps, seed, sweeps, tw, tm, trajectory=True)
    n = 300
    traj = res["traj"]
    for u, tau in enumerate(tm):
        cur = [unpack(traj[tau, r], L) for r in range(4)]
        for r in range(4):
            for w, t0 in enumerate(tw):
                c = res["C"][r, :, w, u]
                if t0 > tau:
                    assert np.all(c == 0)
                    continue
                ref = unpack(traj[t0, r], L)
                assert np.array_equal(c, (cur[r].astype(np.int64) * ref).sum(axis=1))
                assert np.all(np.abs(c) <= n) and np.all((c - n) % 2 == 0)
                if t0 == tau:
                    assert np.all(c == n)
            assert np.array_equal(res["E"][r, :, u], energy_lanes(rp, col, jb, cur[r]))
        for p in range(2):
            want = (cur[2 * p].astype(np.int64) * cur[2 * p + 1]).sum(axis=1)
            assert np.array_equal(res["q"][p, :, u], want)


def test_vb_zero_temperature_energy_never_rises():
    rp, col, eid = sg_inputs.poisson_graph(2000, 4.0, 31)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 31)
    tm = list(range(0, 31))
    res = oracle.vb_run(rp, col, jb, 64, [0.0, 0.0], 3, 30, [], tm)
    E = res["E"]  # E = -H, so it must never decrease
    assert np.all(np.diff(E, axis=2) >= 0)
    assert np.all(E[:, :, -1] > E[:, :, 0])


def test_vb_infinite_temperature_flips_every_spin():
    rp, col, eid = sg_inputs.poisson_graph(400, 4.0, 41)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 41)
    seed, sweeps = 17, 9
    # the only non-flip is r32 == 2^32-1; check none occurs for these counters
    for i in range(400):
        for t in range(sweeps):
            assert int(oracle.philox4x32_10([i, t, 0, 0], [seed, 0])[0]) != 0xFFFFFFFF
    res = oracle.vb_run(rp, col, jb, 64, [math.inf], seed, sweeps, [0], list(range(sweeps + 1)))
    C = res["C"][0, :, 0, :]
    for t in range(sweeps + 1):
        assert np.all(C[:, t] == (-1) ** t * 400)


def _exact_boltzmann(rp, col, jbits, lane, beta):
    n = len(rp) - 1
    states = np.arange(2**n)
    s = 1 - 2 * ((states[:, None] >> np.arange(n)[None, :]) & 1)
    E = np.zeros(2**n)
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            j = col[e]
            if j > i:
                J = -1 if (int(jbits[e]) >> lane) & 1 else 1
                E += J * s[:, i] * s[:, j]
    w = np.exp(beta * E)  # H = -E
    return w / w.sum(), E


def test_vb_long_run_matches_exact_boltzmann():
    n = 6
    ei = np.array([0, 0, 1, 2, 3, 4, 1, 2])
    ej = np.array([1, 2, 3, 4, 5, 5, 4, 5])
    rp, col, eid = sg_inputs.csr_from_edges(n, ei, ej)
    jb = sg_inputs.vb_lane_couplings(eid, 8, 51)
    T, L, sweeps = 1.5, 4, 200000
    res = oracle.vb_run(rp, col, jb, L, [T], 8, sweeps, trajectory=True)
    traj = res["traj"][2000:, 0, :]
    for k in range(L):
        bits = ((traj >> np.uint64(k)) & np.uint64(1)).astype(np.int64)
        idx = (bits << np.arange(n)).sum(axis=1)  # bit 1 means s = -1
        hist = np.bincount(idx, minlength=2**n) / idx.size
        pi, E = _exact_boltzmann(rp, col, jb, k, 1.0 / T)
        assert np.max(np.abs(hist - pi)) < 0.01, k
        assert abs((hist * E).sum() - (pi * E).sum()) < 0.03


def test_vb_paramagnetic_energy():
    """T = 3 > T_c (c tanh^2(beta_c) = 1 gives T_c ~ 1.82 for c = 4): e = -(M/N) tanh(beta)."""
    n, c = 8192, 4.0
    rp, col, eid = sg_inputs.poisson_graph(n, c, 61)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 61)
    T = 3.0
    tm = [100, 150, 200, 250, 300]
    res = oracle.vb_run(rp, col, jb, 16, [T, T], 9, 300, [], tm)
    e = -res["E"].astype(float) / n
    m_edges = (eid.max() + 1)
    assert abs(e.mean() - (-(m_edges / n) * math.tanh(1.0 / T))) < 0.01
