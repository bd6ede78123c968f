"""The oracle's pins are sensitive: plant plausible mistakes in a copy of the oracle (on the CPU)
and check that the brute-force and limit pins reject every one of them."""
import math

import numpy as np
import pytest

import oracle
import sg_inputs
from test_oracle_sk import U, brute_sk
from test_oracle_vb import brute_vb, energy_lanes, unpack

VB_MUTATIONS = {
    "zero_move_rejected": ("int flip = (m <= 0) || (r32 < th[m]);", "int flip = (m < 0) || (m > 0 && r32 < th[m]);"),
    "wrong_sign_of_field": ("int32_t m = sl[i] * field;", "int32_t m = -sl[i] * field;"),
    "missing_factor_two": ("thr[m] = threshold_from_exponent(-2.0 * beta * m);",
                           "thr[m] = threshold_from_exponent(-1.0 * beta * m);"),
    "coupling_ignored": ("field += J * sl[col[e]];", "field += sl[col[e]];"),
    "rng_word_shared": ("(uint32_t)(r / 4), 0, r % 4);", "(uint32_t)(r / 4), 0, 0);"),
    "sweep_not_in_counter": ("draw_word(seed, (uint32_t)i, t,", "draw_word(seed, (uint32_t)i, 0,"),
    "colour_order_reversed": ("for (int32_t c = 0; c < ncol; ++c)", "for (int32_t c = ncol - 1; c >= 0; --c)"),
    "lane_init_high_word_dropped": ("| ((uint64_t)draw_word(seed, (uint32_t)i, 0, (uint32_t)r, 1, 1) << 32);", ";"),
    # the greedy colouring sets the update order
    "colour_flags_never_cleared": ("if (cj >= 0 && cj <= maxdeg + 1) used[cj] = 0;", ";"),
    "colour_skips_last_neighbour": ("for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {\n            int32_t c = colour[col[e]];",
                                    "for (int32_t e = row_ptr[i]; e + 1 < row_ptr[i + 1]; ++e) {\n            int32_t c = colour[col[e]];"),
    # ... and the recolouring pass after it
    "recolour_skipped": ("if (ncol >= 0) ncol = orc_recolour(N, row_ptr, col, colour);", ";"),
    "recolour_in_increasing_colour": ("for (int32_t c = ncol_in - 1; c >= 0; --c)", "for (int32_t c = 0; c < ncol_in; ++c)"),
}

SK_MUTATIONS = {
    "field_update_wrong_sign": ("hr[j] += 2 * (int32_t)J[(size_t)j * N + i] * sr[i];",
                                "hr[j] -= 2 * (int32_t)J[(size_t)j * N + i] * sr[i];"),
    "field_update_no_factor_two": ("hr[j] += 2 * (int32_t)J[(size_t)j * N + i] * sr[i];",
                                   "hr[j] += (int32_t)J[(size_t)j * N + i] * sr[i];"),
    "no_sqrt_n_scale": ("thr[k] = threshold_from_exponent(-(2.0 * beta * k) / sqrt((double)N));",
                        "thr[k] = threshold_from_exponent(-(2.0 * beta * k));"),
    "transposed_coupling_in_field": ("acc += (int32_t)J[(size_t)i * N + j] * s[(size_t)rl * N + j];",
                                     "acc += (int32_t)J[(size_t)j * N + i] * s[(size_t)rl * N + i];"),
}


@pytest.mark.parametrize("name", sorted(VB_MUTATIONS))
def test_vb_pins_catch_planted_mistake(name, tmp_path):
    old, new = VB_MUTATIONS[name]
    src = oracle.source()
    assert src.count(old) >= 1, name
    variant = oracle.compile_variant(src.replace(old, new), str(tmp_path))
    rp, col, eid = sg_inputs.poisson_graph(9, 3.0, 11)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 11)
    temps, L, sweeps = [0.7, 1.0, 2.0, 0.45, 1.3], 64, 5
    res = variant.vb_run(rp, col, jb, L, temps, 99, sweeps, trajectory=True)
    want = brute_vb(rp, col, jb, L, temps, 99, sweeps)
    got = np.array([[unpack(res["traj"][t, r], L) for r in range(len(temps))]
                    for t in range(sweeps + 1)])
    assert not np.array_equal(got, want)


@pytest.mark.parametrize("name", sorted(SK_MUTATIONS))
def test_sk_pins_catch_planted_mistake(name, tmp_path):
    old, new = SK_MUTATIONS[name]
    src = oracle.source()
    assert src.count(old) >= 1, name
    variant = oracle.compile_variant(src.replace(old, new), str(tmp_path))
    n, temps = 10, [0.4, 0.6, 1.0, 2.0, 0.5, 0.4]
    J = sg_inputs.sk_couplings(n, 77 + n)
    res = variant.sk_run(J, temps, 3, 5, trajectory=True)
    assert not np.array_equal(res["traj"], brute_sk(J, temps, 3, 5))


# mistakes in the measurements (the dynamics stay right): the pins recompute C, q and E from the
# brute-force-pinned trajectory
VB_MEASUREMENT_MUTATIONS = {
    "energy_counts_each_edge_twice": ("if (j <= i) continue;", "if (j == i) continue;"),
    "overlap_of_a_replica_with_itself": ("const int8_t *sb = s + ((size_t)(2 * p + 1) * L + k) * N;",
                                         "const int8_t *sb = s + ((size_t)(2 * p) * L + k) * N;"),
    "correlation_against_the_first_snapshot": ("const int8_t *sw = snap[w] + ((size_t)r * L + k) * N;",
                                               "const int8_t *sw = snap[0] + ((size_t)r * L + k) * N;"),
}

SK_MEASUREMENT_MUTATIONS = {
    "energy_not_halved": ("E_out[(size_t)rl * n_tm + ui] = acc / 2;", "E_out[(size_t)rl * n_tm + ui] = acc;"),
    "overlap_pairs_shifted": ("const int8_t *sb = s + (size_t)(2 * p + 1) * N;",
                              "const int8_t *sb = s + (size_t)((2 * p + 2) % RC) * N;"),
}


def vb_measurements_agree(run, rp, col, jb, L, temps, tw, tm):
    res = run(rp, col, jb, L, temps, 5, max(tm), tw, tm, trajectory=True)
    traj, R = res["traj"], len(temps)
    for u, tau in enumerate(tm):
        cur = [unpack(traj[tau, r], L).astype(np.int64) for r in range(R)]
        for r in range(R):
            for w, t0 in enumerate(tw):
                want = ((cur[r] * unpack(traj[t0, r], L)).sum(axis=1) if t0 <= tau
                        else np.zeros(L, dtype=np.int64))
                if not np.array_equal(res["C"][r, :, w, u], want):
                    return False
            if not np.array_equal(res["E"][r, :, u], energy_lanes(rp, col, jb, cur[r])):
                return False
        for p in range(R // 2):
            if not np.array_equal(res["q"][p, :, u], (cur[2 * p] * cur[2 * p + 1]).sum(axis=1)):
                return False
    return True


@pytest.mark.parametrize("name", sorted(VB_MEASUREMENT_MUTATIONS))
def test_vb_measurement_pins_catch_planted_mistake(name, tmp_path):
    old, new = VB_MEASUREMENT_MUTATIONS[name]
    src = oracle.source()
    assert src.count(old) == 1, name
    variant = oracle.compile_variant(src.replace(old, new), str(tmp_path))
    rp, col, eid = sg_inputs.poisson_graph(60, 4.0, 23)
    jb = sg_inputs.vb_lane_couplings(eid, eid.max() + 1, 23)
    args = (rp, col, jb, 16, [0.8, 0.8, 1.5, 1.5], [0, 2, 5], [0, 1, 2, 5, 8, 12])
    assert vb_measurements_agree(oracle.vb_run, *args)  # the check passes on the oracle itself
    assert not vb_measurements_agree(variant.vb_run, *args)


@pytest.mark.parametrize("name", sorted(SK_MEASUREMENT_MUTATIONS))
def test_sk_measurement_pins_catch_planted_mistake(name, tmp_path):
    old, new = SK_MEASUREMENT_MUTATIONS[name]
    src = oracle.source()
    assert src.count(old) == 1, name
    variant = oracle.compile_variant(src.replace(old, new), str(tmp_path))
    n, temps, tw, tm = 40, [0.4, 0.4, 0.6, 0.6], [0, 3], [0, 2, 3, 6, 10]
    J = sg_inputs.sk_couplings(n, 31)

    def agree(run):
        res = run(J, temps, 4, max(tm), tw, tm, trajectory=True)
        traj = res["traj"].astype(np.int64)
        for u, tau in enumerate(tm):
            for r in range(len(temps)):
                for w, t0 in enumerate(tw):
                    want = (traj[tau, r] * traj[t0, r]).sum() if t0 <= tau else 0
                    if res["C"][r, w, u] != want:
                        return False
                if res["E"][r, u] != -U(J, traj[tau, r]):
                    return False
            for p in range(len(temps) // 2):
                if res["q"][p, u] != (traj[tau, 2 * p] * traj[tau, 2 * p + 1]).sum():
                    return False
        return True

    assert agree(oracle.sk_run)
    assert not agree(variant.sk_run)
