"""Pin the Sherrington-Kirkpatrick oracle (binary couplings, SI section 1) against things other
than itself.

* Brute force: each Metropolis decision in the fixed order i = 0..N-1 (SI section 1) taken from
  the full Hamiltonian of Eq. 1 with J_ij = +-1/sqrt(N): dE = U(s') - U(s) in integer units
  U = -sum_{i<j} J_ij s_i s_j, acceptance floor(2^32 exp(-beta dE / sqrt(N))) in arbitrary
  precision.  Trajectories must agree bit for bit.
* Exact Boltzmann enumeration on N = 8 (long-run histogram).
* T = 0 and T = infinity limits; energies recomputed from spins (checks the incremental fields).
* The paramagnetic energy e = -(beta/2)(N-1)/N for T > T_c = 1.
* Replicas are independent chains: a replica subset reproduces the same slice of a full run.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle
import sg_inputs

mpmath.mp.dps = 50


def philox_word(seed, c, word):
    return int(oracle.philox4x32_10(c, [seed & 0xFFFFFFFF, seed >> 32])[word])


def U(J, s):
    """Integer energy -sum_{i<j} J_ij s_i s_j."""
    return -int(np.triu(J.astype(np.int64) * np.outer(s, s), k=1).sum())


def brute_sk(J, temps, seed, sweeps):
    n = J.shape[0]
    R = len(temps)
    s = np.zeros((R, n), dtype=np.int8)
    for r in range(R):
        for i in range(n):
            s[r, i] = -1 if philox_word(seed, [i, 0, r, 1], 0) & 1 else 1
    traj = [s.copy()]
    for t in range(sweeps):
        for i in range(n):
            for r in range(R):
                s2 = s[r].copy()
                s2[i] = -s2[i]
                dE = U(J, s2) - U(J, s[r])
                r32 = philox_word(seed, [i, t, r // 4, 0], r % 4)
                if dE <= 0:
                    acc = True
                elif temps[r] == 0:
                    acc = False
                else:
                    v = mpmath.mpf(2) ** 32 * mpmath.e ** (-mpmath.mpf(dE) / temps[r] / mpmath.sqrt(n))
                    acc = r32 < min(0xFFFFFFFF, int(mpmath.floor(v)))
                if acc:
                    s[r, i] = -s[r, i]
        traj.append(s.copy())
    return np.array(traj)


@pytest.mark.parametrize("n,temps,seed", [
    (10, [0.4, 0.6, 1.0, 2.0, 0.5, 0.4], 3),
    (13, [0.3, 0.3, 5.0], 2**35 + 1),
])
def test_sk_oracle_matches_brute_force(n, temps, seed):
    J = sg_inputs.sk_couplings(n, 77 + n)
    res = oracle.sk_run(J, temps, seed, 5, trajectory=True)
    want = brute_sk(J, temps, seed, 5)
    assert np.array_equal(res["traj"], want)


def test_sk_measurements_and_energy_from_spins():
    n = 96
    J = sg_inputs.sk_couplings(n, 5)
    temps = [0.4, 0.4, 0.6, 0.6]
    tw = [0, 3, 8]
    tm = [0, 1, 3, 4, 8, 11, 16, 24]
    res = oracle.sk_run(J, temps, 4, 24, tw, tm, trajectory=True)
    traj = res["traj"].astype(np.int64)
    for u, tau in enumerate(tm):
        for r in range(4):
            for w, t0 in enumerate(tw):
                if t0 > tau:
                    assert res["C"][r, w, u] == 0
                else:
                    assert res["C"][r, w, u] == (traj[tau, r] * traj[t0, r]).sum()
            assert res["E"][r, u] == -U(J, traj[tau, r])
        for p in range(2):
            assert res["q"][p, u] == (traj[tau, 2 * p] * traj[tau, 2 * p + 1]).sum()


def test_sk_replica_subset_matches_full_run():
    J = sg_inputs.sk_couplings(64, 8)
    temps = [0.4, 0.5, 0.6, 0.7, 0.8, 0.9]
    full = oracle.sk_run(J, temps, 11, 12, [2], [12])
    part = oracle.sk_run(J, temps, 11, 12, [2], [12], r_first=2, r_count=2)
    assert np.array_equal(full["spins"][2:4], part["spins"])
    assert np.array_equal(full["C"][2:4], part["C"])
    assert np.array_equal(full["q"][1:2], part["q"])


def test_sk_zero_temperature_energy_never_rises():
    J = sg_inputs.sk_couplings(200, 9)
    tm = list(range(0, 21))
    res = oracle.sk_run(J, [0.0, 0.0], 12, 20, [], tm)
    assert np.all(np.diff(res["E"], axis=1) >= 0)


def test_sk_infinite_temperature_flips_every_spin():
    n, seed, sweeps = 50, 21, 6
    for i in range(n):
        for t in range(sweeps):
            assert int(oracle.philox4x32_10([i, t, 0, 0], [seed, 0])[0]) != 0xFFFFFFFF
    J = sg_inputs.sk_couplings(n, 10)
    res = oracle.sk_run(J, [math.inf], seed, sweeps, [0], list(range(sweeps + 1)))
    for t in range(sweeps + 1):
        assert res["C"][0, 0, t] == (-1) ** t * n


def test_sk_long_run_matches_exact_boltzmann():
    n, T, sweeps = 8, 1.0, 150000
    J = sg_inputs.sk_couplings(n, 13)
    res = oracle.sk_run(J, [T, T], 14, sweeps, trajectory=True)
    states = np.arange(2**n)
    s = 1 - 2 * ((states[:, None] >> np.arange(n)[None, :]) & 1)
    Uall = -np.einsum("si,ij,sj->s", s, np.triu(J.astype(np.int64), 1), s)
    w = np.exp(-Uall / T / math.sqrt(n))
    pi = w / w.sum()
    for r in range(2):
        tr = res["traj"][2000:, r, :].astype(np.int64)
        idx = (((1 - tr) // 2) << np.arange(n)).sum(axis=1)
        hist = np.bincount(idx, minlength=2**n) / idx.size
        assert np.max(np.abs(hist - pi)) < 0.01
        assert abs((hist * Uall).sum() - (pi * Uall).sum()) < 0.05


def test_sk_paramagnetic_energy():
    n, T = 256, 2.0
    J = sg_inputs.sk_couplings(n, 15)
    tm = [100, 150, 200]
    res = oracle.sk_run(J, [T] * 16, 16, 200, [], tm)
    e = -res["E"].astype(float) / (n * math.sqrt(n))
    assert abs(e.mean() - (-(1.0 / T) / 2 * (n - 1) / n)) < 0.01
