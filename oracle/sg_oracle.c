/*
 * sg_oracle.c -- plain, slow, obviously-correct CPU oracle for the aging-dynamics hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file:
 * only the test suite, the smoke check and the bench's CPU-baseline leg use it.  It shares
 * no code, header, table or constant generator with the CUDA library; the only thing the two
 * have in common is the seeded input data they are given.
 *
 * What it computes (arXiv:1906.11195, "Strong ergodicity breaking in aging of mean field spin
 * glasses"):
 *   - Viana-Bray model, H = -sum_{(ij) in E} J_ij s_i s_j with J_ij = +-1 (Eq. 3), simulated
 *     with single-spin-flip Metropolis dynamics at fixed temperature after a quench from a
 *     random configuration (Methods; SI section 2).  64 disorder samples ("lanes") share one
 *     graph and differ in couplings and initial spins (multispin coding, SI section 2 and the
 *     caption of Table 1).  The graph is updated one independent set at a time (SI section 3:
 *     the bipartite halves are the two-colour case; a greedy colouring generalises it).
 *   - Sherrington-Kirkpatrick model, H = -sum_{i<j} J_ij s_i s_j / sqrt(N) with binary J
 *     (Eq. 1 and SI section 1), Metropolis, spins updated in a fixed order i = 0..N-1.
 *   - Two-time correlation C(t_w+t, t_w) = (1/N) sum_i s_i(t_w+t) s_i(t_w) (the correlation
 *     defined after Eq. 1 and Eq. formula1 of SI section 1), the overlap between the two
 *     clones of a sample (SI section 1), and the energy.  All are returned as integer counts.
 *
 * Readings where the paper is silent (it names no random number generator, no update order
 * inside a colour class, no threshold arithmetic):
 *   - One random number r32 per (replica, sweep, spin) is shared by the 64 lanes of a word.  It
 *     is word (r mod 4) of Philox4x32-10 with key (seed_lo, seed_hi) and counter
 *     (i, t, r / 4, 0): i the vertex (original label), t the sweep index (0-based).
 *   - Initial spins: the 64 lane bits of vertex i, replica r are w0 | w1 << 32 of Philox with
 *     counter (i, 0, r, 1); bit = 1 means s = -1.  SK uses lane bit 0.
 *   - Acceptance: flip iff dE <= 0 or r32 < thr, with thr = min(2^32 - 1,
 *     floor(2^32 * exp(-beta * dE))) evaluated in double precision.
 *   - The colour classes come from a greedy colouring in vertex order followed by one
 *     recolouring pass (greedy again, in the order of decreasing colour and increasing label),
 *     which never adds a colour and removes the thin last classes of the first pass; a sweep
 *     updates class 0, 1, ... in turn.  A colour class is updated in increasing vertex order
 *     (irrelevant: it is an independent set and the random number is keyed by the vertex).
 *   - Time tau = number of completed sweeps; snapshots for C are taken at tau = t_w before the
 *     measurement at the same tau.
 *
 * Parity status: every function here is pinned by the CPU test-suite against something other
 * than itself (an independent Philox implementation, arbitrary-precision thresholds, brute
 * force single-site updates from the full Hamiltonian, exact Boltzmann enumeration, T = 0 and
 * T = infinity limits, high-temperature energies).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------------------------------
 * Philox4x32-10, from J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11.  Each of the ten rounds multiplies counter words 0 and
 * 2 by the two round multipliers, mixes the high halves with words 1 and 3 and the round key,
 * and the key is bumped by the two Weyl constants between rounds.
 * ---------------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mult0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)mult1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static uint32_t draw_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                          int word)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[word];
}

/* Metropolis acceptance threshold for an energy increase dE > 0 at inverse temperature beta:
 * the move is taken iff a uniform 32-bit integer is below floor(2^32 exp(-beta dE)). */
static uint32_t threshold_from_exponent(double x)
{
    double v = ldexp(exp(x), 32);
    if (!(v < 4294967295.0)) return 0xFFFFFFFFu;
    return (uint32_t)floor(v);
}

static double beta_of(double T) { return 1.0 / T; }

/* VB: flipping spin i changes the energy by dE = 2m, where m = s_i sum_j J_ij s_j.
 * thr[m] for m = 1..dmax; thr[0] is set to 2^32-1 (m <= 0 is always accepted). */
void orc_vb_thresholds(double T, int32_t dmax, uint32_t *thr)
{
    double beta = beta_of(T);
    thr[0] = 0xFFFFFFFFu;
    for (int32_t m = 1; m <= dmax; ++m) thr[m] = threshold_from_exponent(-2.0 * beta * m);
}

/* SK: dE = 2k / sqrt(N) with k = s_i sum_j J_ij s_j.  thr[k] for k = 1..N-1; thr[0] = 2^32-1. */
void orc_sk_thresholds(double T, int32_t N, uint32_t *thr)
{
    double beta = beta_of(T);
    thr[0] = 0xFFFFFFFFu;
    for (int32_t k = 1; k < N; ++k)
        thr[k] = threshold_from_exponent(-(2.0 * beta * k) / sqrt((double)N));
}

/* Greedy colouring in vertex order: colour(i) = smallest colour unused by the neighbours
 * coloured before i.  Returns the number of colours, or a negative error. */
int32_t orc_greedy_colour(int32_t N, const int32_t *row_ptr, const int32_t *col, int32_t *colour)
{
    int32_t maxdeg = 0;
    for (int32_t i = 0; i < N; ++i) {
        int32_t d = row_ptr[i + 1] - row_ptr[i];
        if (d > maxdeg) maxdeg = d;
    }
    char *used = (char *)calloc((size_t)maxdeg + 2, 1);
    if (!used) return ORC_ENOMEM;
    for (int32_t i = 0; i < N; ++i) colour[i] = -1;
    int32_t ncol = 0;
    for (int32_t i = 0; i < N; ++i) {
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t c = colour[col[e]];
            if (c >= 0 && c <= maxdeg + 1) used[c] = 1;
        }
        int32_t c = 0;
        while (used[c]) ++c;
        colour[i] = c;
        if (c + 1 > ncol) ncol = c + 1;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t cj = colour[col[e]];
            if (cj >= 0 && cj <= maxdeg + 1) used[cj] = 0;
        }
    }
    free(used);
    return ncol;
}

/* One recolouring pass: the vertices are coloured greedily again, in the order of decreasing
 * colour and, within a colour, increasing label.  The vertices of one old class form an
 * independent set, so the new colouring uses no more colours than the old one (the iterated
 * greedy argument).  colour[] is replaced.  Returns the number of colours, or a negative
 * error. */
int32_t orc_recolour(int32_t N, const int32_t *row_ptr, const int32_t *col, int32_t *colour)
{
    int32_t maxdeg = 0, ncol_in = 0;
    for (int32_t i = 0; i < N; ++i) {
        int32_t d = row_ptr[i + 1] - row_ptr[i];
        if (d > maxdeg) maxdeg = d;
        if (colour[i] + 1 > ncol_in) ncol_in = colour[i] + 1;
    }
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    int32_t *fresh = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    char *used = (char *)calloc((size_t)maxdeg + 2, 1);
    if (!order || !fresh || !used) return ORC_ENOMEM;
    int32_t pos = 0;
    for (int32_t c = ncol_in - 1; c >= 0; --c)
        for (int32_t i = 0; i < N; ++i)
            if (colour[i] == c) order[pos++] = i;
    for (int32_t i = 0; i < N; ++i) fresh[i] = -1;
    int32_t ncol = 0;
    for (int32_t k = 0; k < N; ++k) {
        int32_t i = order[k];
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t c = fresh[col[e]];
            if (c >= 0 && c <= maxdeg + 1) used[c] = 1;
        }
        int32_t c = 0;
        while (used[c]) ++c;
        fresh[i] = c;
        if (c + 1 > ncol) ncol = c + 1;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t cj = fresh[col[e]];
            if (cj >= 0 && cj <= maxdeg + 1) used[cj] = 0;
        }
    }
    for (int32_t i = 0; i < N; ++i) colour[i] = fresh[i];
    free(order);
    free(fresh);
    free(used);
    return ncol;
}

static int32_t index_of(const int64_t *list, int32_t n, int64_t v)
{
    for (int32_t k = 0; k < n; ++k)
        if (list[k] == v) return k;
    return -1;
}

/* ------------------------------------------------------------------------------------------
 * Viana-Bray run.
 *   N, row_ptr[N+1], col[2M]: symmetric simple graph (CSR).
 *   jbits[2M]: coupling word per directed entry; lane k has J = 1 - 2*bit_k.
 *   n_lanes (1..64) lanes and R replicas are simulated; T[R] are the replica temperatures.
 *   The run performs n_sweeps sweeps from tau = 0.
 * Outputs (any may be NULL):
 *   spins_out[R][N]            final spins, bit k = 1 iff s = -1 in lane k
 *   C_out[R][n_lanes][n_tw][n_tm]   sum_i s_i(tm) s_i(tw) when tw <= tm <= n_sweeps, else 0
 *   q_out[R/2][n_lanes][n_tm]       sum_i s_i^(2p)(tm) s_i^(2p+1)(tm)
 *   E_out[R][n_lanes][n_tm]         sum over undirected edges of J_ij s_i s_j
 *   traj_out[n_sweeps+1][R][N]      spins (packed as spins_out) after every sweep; tiny N only
 * ---------------------------------------------------------------------------------------- */
int32_t orc_vb_run(int32_t N, const int32_t *row_ptr, const int32_t *col, const uint64_t *jbits,
                   int32_t n_lanes, int32_t R, const double *T, uint64_t seed, int64_t n_sweeps,
                   const int64_t *tw, int32_t n_tw, const int64_t *tm, int32_t n_tm,
                   uint64_t *spins_out, int64_t *C_out, int64_t *q_out, int64_t *E_out,
                   uint64_t *traj_out)
{
    if (N < 1 || n_lanes < 1 || n_lanes > 64 || R < 1 || n_sweeps < 0) return ORC_EINVAL;
    const int32_t L = n_lanes;
    int32_t dmax = 0;
    for (int32_t i = 0; i < N; ++i) {
        int32_t d = row_ptr[i + 1] - row_ptr[i];
        if (d > dmax) dmax = d;
    }
    int32_t *colour = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int8_t *s = (int8_t *)malloc((size_t)R * L * N);
    uint32_t *thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)R * (dmax + 1));
    int8_t **snap = (int8_t **)calloc((size_t)(n_tw > 0 ? n_tw : 1), sizeof(int8_t *));
    if (!colour || !s || !thr || !snap) return ORC_ENOMEM;
    int32_t ncol = orc_greedy_colour(N, row_ptr, col, colour);
    if (ncol >= 0) ncol = orc_recolour(N, row_ptr, col, colour);
    if (ncol < 0) return ncol;
    for (int32_t r = 0; r < R; ++r) orc_vb_thresholds(T[r], dmax, thr + (size_t)r * (dmax + 1));

    /* quench: random initial configuration */
    for (int32_t r = 0; r < R; ++r)
        for (int32_t i = 0; i < N; ++i) {
            uint64_t w = (uint64_t)draw_word(seed, (uint32_t)i, 0, (uint32_t)r, 1, 0)
                       | ((uint64_t)draw_word(seed, (uint32_t)i, 0, (uint32_t)r, 1, 1) << 32);
            for (int32_t k = 0; k < L; ++k)
                s[((size_t)r * L + k) * N + i] = ((w >> k) & 1) ? -1 : 1;
        }
    if (C_out) memset(C_out, 0, sizeof(int64_t) * (size_t)R * L * n_tw * n_tm);
    if (q_out) memset(q_out, 0, sizeof(int64_t) * (size_t)(R / 2) * L * n_tm);
    if (E_out) memset(E_out, 0, sizeof(int64_t) * (size_t)R * L * n_tm);

    for (int64_t tau = 0;; ++tau) {
        if (traj_out)
            for (int32_t r = 0; r < R; ++r)
                for (int32_t i = 0; i < N; ++i) {
                    uint64_t w = 0;
                    for (int32_t k = 0; k < L; ++k)
                        if (s[((size_t)r * L + k) * N + i] < 0) w |= (uint64_t)1 << k;
                    traj_out[((size_t)tau * R + r) * N + i] = w;
                }
        /* measurements at time tau */
        int32_t wi = index_of(tw, n_tw, tau);
        if (wi >= 0) {
            snap[wi] = (int8_t *)malloc((size_t)R * L * N);
            if (!snap[wi]) return ORC_ENOMEM;
            memcpy(snap[wi], s, (size_t)R * L * N);
        }
        int32_t ui = index_of(tm, n_tm, tau);
        if (ui >= 0) {
            for (int32_t r = 0; r < R; ++r)
                for (int32_t k = 0; k < L; ++k) {
                    const int8_t *sc = s + ((size_t)r * L + k) * N;
                    for (int32_t w = 0; w < n_tw; ++w) {
                        if (tw[w] > tau || !snap[w] || !C_out) continue;
                        const int8_t *sw = snap[w] + ((size_t)r * L + k) * N;
                        int64_t acc = 0;
                        for (int32_t i = 0; i < N; ++i) acc += (int64_t)sc[i] * sw[i];
                        C_out[(((size_t)r * L + k) * n_tw + w) * n_tm + ui] = acc;
                    }
                    if (E_out) {
                        int64_t e_acc = 0;
                        for (int32_t i = 0; i < N; ++i)
                            for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                                int32_t j = col[e];
                                if (j <= i) continue;
                                int32_t J = ((jbits[e] >> k) & 1) ? -1 : 1;
                                e_acc += (int64_t)J * sc[i] * sc[j];
                            }
                        E_out[((size_t)r * L + k) * n_tm + ui] = e_acc;
                    }
                }
            if (q_out)
                for (int32_t p = 0; p < R / 2; ++p)
                    for (int32_t k = 0; k < L; ++k) {
                        const int8_t *sa = s + ((size_t)(2 * p) * L + k) * N;
                        const int8_t *sb = s + ((size_t)(2 * p + 1) * L + k) * N;
                        int64_t acc = 0;
                        for (int32_t i = 0; i < N; ++i) acc += (int64_t)sa[i] * sb[i];
                        q_out[((size_t)p * L + k) * n_tm + ui] = acc;
                    }
        }
        if (tau == n_sweeps) break;

        /* one Metropolis sweep: colour classes in order, each class in increasing i */
        const uint32_t t = (uint32_t)tau;
        for (int32_t c = 0; c < ncol; ++c)
            for (int32_t i = 0; i < N; ++i) {
                if (colour[i] != c) continue;
                for (int32_t r = 0; r < R; ++r) {
                    uint32_t r32 = draw_word(seed, (uint32_t)i, t, (uint32_t)(r / 4), 0, r % 4);
                    const uint32_t *th = thr + (size_t)r * (dmax + 1);
                    for (int32_t k = 0; k < L; ++k) {
                        int8_t *sl = s + ((size_t)r * L + k) * N;
                        int32_t field = 0;
                        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                            int32_t J = ((jbits[e] >> k) & 1) ? -1 : 1;
                            field += J * sl[col[e]];
                        }
                        int32_t m = sl[i] * field; /* dE = 2m */
                        int flip = (m <= 0) || (r32 < th[m]);
                        if (flip) sl[i] = (int8_t)(-sl[i]);
                    }
                }
            }
    }

    if (spins_out)
        for (int32_t r = 0; r < R; ++r)
            for (int32_t i = 0; i < N; ++i) {
                uint64_t w = 0;
                for (int32_t k = 0; k < L; ++k)
                    if (s[((size_t)r * L + k) * N + i] < 0) w |= (uint64_t)1 << k;
                spins_out[(size_t)r * N + i] = w;
            }
    for (int32_t w = 0; w < n_tw; ++w) free(snap[w]);
    free(snap);
    free(thr);
    free(s);
    free(colour);
    return ncol;
}

/* ------------------------------------------------------------------------------------------
 * Sherrington-Kirkpatrick run (binary couplings, SI section 1).
 *   J[N*N]: symmetric int8 +-1, zero diagonal, row-major.  The 1/sqrt(N) scale lives in the
 *   threshold table.  Replicas [r_first, r_first + r_count) of an R-replica run are simulated
 *   (replicas are independent chains; r selects their random numbers and temperature T[r]).
 *   Spins are updated in the fixed order i = 0..N-1; the local field h_i = sum_j J_ij s_j is
 *   kept exactly in integers and refreshed in full on every accepted flip.
 * Outputs (any may be NULL), indexed by the local replica index rl = r - r_first:
 *   spins_out[r_count][N]  int8 +-1
 *   C_out[r_count][n_tw][n_tm], q_out[r_count/2][n_tm] (pairs (2p, 2p+1) local; r_first even),
 *   E_out[r_count][n_tm] = sum_{i<j} J_ij s_i s_j  (= one half of sum_i s_i h_i).
 *   traj_out[n_sweeps+1][r_count][N]  spins after every sweep; tiny N only.
 * ---------------------------------------------------------------------------------------- */
int32_t orc_sk_run(int32_t N, const int8_t *J, int32_t R, const double *T, uint64_t seed,
                   int64_t n_sweeps, int32_t r_first, int32_t r_count,
                   const int64_t *tw, int32_t n_tw, const int64_t *tm, int32_t n_tm,
                   int8_t *spins_out, int64_t *C_out, int64_t *q_out, int64_t *E_out,
                   int8_t *traj_out)
{
    if (N < 1 || R < 1 || r_first < 0 || r_count < 1 || r_first + r_count > R || n_sweeps < 0)
        return ORC_EINVAL;
    const int32_t RC = r_count;
    int8_t *s = (int8_t *)malloc((size_t)RC * N);
    int32_t *h = (int32_t *)malloc(sizeof(int32_t) * (size_t)RC * N);
    uint32_t *thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)RC * N);
    int8_t **snap = (int8_t **)calloc((size_t)(n_tw > 0 ? n_tw : 1), sizeof(int8_t *));
    if (!s || !h || !thr || !snap) return ORC_ENOMEM;
    for (int32_t rl = 0; rl < RC; ++rl) orc_sk_thresholds(T[r_first + rl], N, thr + (size_t)rl * N);

    for (int32_t rl = 0; rl < RC; ++rl) {
        int32_t r = r_first + rl;
        for (int32_t i = 0; i < N; ++i) {
            uint32_t w0 = draw_word(seed, (uint32_t)i, 0, (uint32_t)r, 1, 0);
            s[(size_t)rl * N + i] = (w0 & 1) ? -1 : 1;
        }
        for (int32_t i = 0; i < N; ++i) {
            int32_t acc = 0;
            for (int32_t j = 0; j < N; ++j) acc += (int32_t)J[(size_t)i * N + j] * s[(size_t)rl * N + j];
            h[(size_t)rl * N + i] = acc;
        }
    }
    if (C_out) memset(C_out, 0, sizeof(int64_t) * (size_t)RC * n_tw * n_tm);
    if (q_out) memset(q_out, 0, sizeof(int64_t) * (size_t)(RC / 2) * n_tm);
    if (E_out) memset(E_out, 0, sizeof(int64_t) * (size_t)RC * n_tm);

    for (int64_t tau = 0;; ++tau) {
        if (traj_out) memcpy(traj_out + (size_t)tau * RC * N, s, (size_t)RC * N);
        int32_t wi = index_of(tw, n_tw, tau);
        if (wi >= 0) {
            snap[wi] = (int8_t *)malloc((size_t)RC * N);
            if (!snap[wi]) return ORC_ENOMEM;
            memcpy(snap[wi], s, (size_t)RC * N);
        }
        int32_t ui = index_of(tm, n_tm, tau);
        if (ui >= 0) {
            for (int32_t rl = 0; rl < RC; ++rl) {
                const int8_t *sc = s + (size_t)rl * N;
                for (int32_t w = 0; w < n_tw; ++w) {
                    if (tw[w] > tau || !snap[w] || !C_out) continue;
                    const int8_t *sw = snap[w] + (size_t)rl * N;
                    int64_t acc = 0;
                    for (int32_t i = 0; i < N; ++i) acc += (int64_t)sc[i] * sw[i];
                    C_out[((size_t)rl * n_tw + w) * n_tm + ui] = acc;
                }
                if (E_out) {
                    int64_t acc = 0;
                    for (int32_t i = 0; i < N; ++i) acc += (int64_t)sc[i] * h[(size_t)rl * N + i];
                    E_out[(size_t)rl * n_tm + ui] = acc / 2;
                }
            }
            if (q_out)
                for (int32_t p = 0; p < RC / 2; ++p) {
                    const int8_t *sa = s + (size_t)(2 * p) * N;
                    const int8_t *sb = s + (size_t)(2 * p + 1) * N;
                    int64_t acc = 0;
                    for (int32_t i = 0; i < N; ++i) acc += (int64_t)sa[i] * sb[i];
                    q_out[(size_t)p * n_tm + ui] = acc;
                }
        }
        if (tau == n_sweeps) break;

        const uint32_t t = (uint32_t)tau;
        for (int32_t i = 0; i < N; ++i)
            for (int32_t rl = 0; rl < RC; ++rl) {
                int32_t r = r_first + rl;
                int8_t *sr = s + (size_t)rl * N;
                int32_t *hr = h + (size_t)rl * N;
                int32_t k = sr[i] * hr[i]; /* dE = 2k / sqrt(N) */
                uint32_t r32 = draw_word(seed, (uint32_t)i, t, (uint32_t)(r / 4), 0, r % 4);
                int flip = (k <= 0) || (r32 < thr[(size_t)rl * N + k]);
                if (flip) {
                    sr[i] = (int8_t)(-sr[i]);
                    for (int32_t j = 0; j < N; ++j) hr[j] += 2 * (int32_t)J[(size_t)j * N + i] * sr[i];
                }
            }
    }

    if (spins_out) memcpy(spins_out, s, (size_t)RC * N);
    for (int32_t w = 0; w < n_tw; ++w) free(snap[w]);
    free(snap);
    free(thr);
    free(h);
    free(s);
    return ORC_OK;
}
