// sk_internal.cuh -- Sherrington-Kirkpatrick device layout and launch wrappers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sg_internal.cuh"

namespace sg {

// One SK sample, spins padded to Np (a multiple of 128 and of the block size).
struct SkDev {
    const uint32_t* JbT;      // [Np/32][Np] bit j%32 of word j/32 of row i, at (j/32)*Np + i: J_ij = -1
    const uint8_t* J8;        // [Np][Np] e4m3: +1 = 0x38, -1 = 0xB8, 0 on the diagonal/padding
    const uint32_t* thr;      // [n_temps][N] thresholds (entry k)
    const int32_t* temp_index;// [R] row of thr used by replica r
    const float* coef;        // [R] sqrt(N) * T / 2 (start of the K* search)
    uint32_t* S;              // [R][Np/32] spins, bit = 1 means s = -1
    uint8_t* D;               // [R][Np] e4m3 spin changes (s' - s)/2 of the current block
    int32_t* H;               // [R][Np] local fields sum_j J_ij s_j
    int32_t* kst;             // [R][Np] K* of the current sweep (largest accepted k)
    uint32_t* flips;          // [R][Np/32] flip masks written by the latest in-block update
    uint32_t* snap;           // [n_tw][R][Np/32]
    int* err;                 // device status word
    uint64_t seed;
    int32_t N, Np, R;
    int32_t inblock_warps;    // replica warps per in-block CTA (2, 4 or 8)
    int32_t test_nowait;      // nonzero only in tests of the timeout path: every bounded wait
                              // of a sweep becomes a single test (drains keep the full bound)
};

// --------------------------------------------------------------------------------------------
// TMA tile load and tcgen05 descriptors (inline PTX); mbarrier helpers are in sg_internal.cuh
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// shared-memory matrix descriptor, K-major operand in the 128B (kw = 128) or 64B (kw = 64)
// swizzled layout written by TMA: 8-row groups are kw*8 bytes apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, int kw) {
    const uint64_t sbo = (uint64_t)(kw * 8) >> 4;
    const uint64_t layout = kw == 128 ? 2ull : 4ull;
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | (sbo << 32) | (1ull << 46) |
           (layout << 61);
}

constexpr int kSkPersistSlots = 8;  // spin-change ring slots of the persistent sweeps (Q)

// Persistent sweeps (sk_persist.cu): one cooperative launch runs n_sweeps sweeps; field CTAs
// hold row tiles of H in tensor memory, chain CTAs run the sequential decisions (block = 128
// spins).  Blocks of 32 * (2W + 2) threads: a chain CTA uses all (W replica warps, W fold warps,
// a staging warp and a release warp); a field CTA uses warps 0..3 (tensor-memory epilogue,
// thread 0 issues the MMAs) and warp W (operand loads).
constexpr int kSkPersistMaxSweeps = 64;  // sweeps of one launch (the K* buffer holds them)
struct SkPersistArgs {
    uint8_t* Dring;   // [Q][R][128] e4m3 spin changes 2 D = s' - s of the last Q blocks
    int32_t* Hpub;    // [R][Np] fields of a tile's rows, published for its chain block
    uint32_t* sync;   // [2Q + nb] D_count[Q], D_free[Q], H_ready[nb]; zeroed before each launch
    int16_t* kst16;   // [kSkPersistMaxSweeps][R][Np] K* of the launch's sweeps
    const uint32_t* clock;  // device sweep clock: the launch runs sweeps *clock + t_off + s
    uint32_t t_off;
    int n_sweeps;     // sweeps in this launch, 1..kSkPersistMaxSweeps
    int nb;           // blocks = row tiles, Np / 128
    int nG;           // field CTAs; CTA j owns tiles j, j + nG, ...
    int TPC;          // tiles per field CTA (TPC * R <= 512 tensor-memory columns)
    int nC;           // chain CTAs, R / W
    int W;            // replica warps per chain CTA (4 or 8)
    int L;            // blocks of flips a chain warp folds in itself (lookahead), L < nb
    int Q;            // spin-change ring slots: kSkPersistSlots
    int nst;          // shared-memory stages of a field CTA (2..4)
};
// 2-D tensor maps (no swizzle) of the chain CTAs' staging, boxes of 128 rows: jb: JbT as
// [Np/32 column words][Np rows] of 32-bit words, box 128 x 4 (one block's column words);
// kst: kst16 as [kSkPersistMaxSweeps R][Np] 16-bit words, box 128 x W; h, hpub: [R][Np] of
// 32-bit words, box 128 x W
struct SkPersistMaps {
    CUtensorMap jb, kst, h, hpub;
};
size_t sk_persist_smem_bytes(const SkDev& d, const SkPersistArgs& a);
// 1 if the configuration can be launched with every CTA resident on num_sms SMs
int sk_persist_fits(const SkDev& d, const SkPersistArgs& a, int num_sms);
// the lookaheads L the persistent kernel is compiled for
int sk_persist_lookahead_supported(int L);
// queue a.n_sweeps sweeps: K* of all of them (k_sk_kstar16), counter reset, one cooperative
// launch; mapJ: J8 boxes of 128 x 128, mapD: Dring as [Q R rows][128] with boxes of 128 x R.
// Returns the kernel launches queued (2) or -1.
int sk_persist_sweeps(const SkDev& d, const SkPersistArgs& a, const CUtensorMap& mapJ,
                      const CUtensorMap& mapD, const SkPersistMaps& maps, cudaStream_t st);
// K* of n consecutive sweeps from index *clock + t_off, int16, into dst[(s R + r) Np + i]
int sk_kstar16_sweeps(const SkDev& d, const uint32_t* clock, uint32_t t_off, int n, int16_t* dst,
                      cudaStream_t st);

// --------------------------------------------------------------------------------------------
// K* for a replica: largest k in [0, N-1] with k == 0 or r32 < thr[k].  A logarithmic estimate
// (thr[k] ~ 2^32 exp(-k / coef), coef = sqrt(N) T / 2) is corrected exactly on the table.
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ int sk_kstar(uint32_t r32, const uint32_t* __restrict__ thr, int n,
                                        float coef) {
    const float u = ((float)r32 + 0.5f) * 2.3283064365386963e-10f;
    const float est = -__logf(u) * coef;
    int k;
    if (!(est < (float)(n - 1))) k = n - 1;
    else if (!(est > 0.f)) k = 0;
    else k = (int)est;
    while (k + 1 <= n - 1 && r32 < __ldg(thr + k + 1)) ++k;
    while (k >= 1 && !(r32 < __ldg(thr + k))) --k;
    return k;
}

int sk_init(const SkDev& d, cudaStream_t st);
int sk_kstar_sweep(const SkDev& d, const uint32_t* clock, uint32_t t_off, cudaStream_t st);

// One operation of a blocked sweep's schedule (sk_blocked_schedule in sg_sk.cu): stream 0 is the
// handle's stream, 1 the side stream; events 0, 1 are "in-block done" (block parity), 2, 3
// "side done"; a field update of rows leaves the row tiles [skip0, skip1) out.
enum { kSchedKstar = 0, kSchedInblock = 1, kSchedFieldAll = 2, kSchedFieldRows = 3,
       kSchedRecord = 4, kSchedWait = 5 };
struct SkSchedOp {
    int32_t op, stream, block, skip0, skip1, event;
};
// the same into even[] or odd[] by the parity of the sweep index
int sk_kstar_sweep_into(const SkDev& d, const uint32_t* clock, uint32_t t_off, int32_t* even,
                        int32_t* odd, cudaStream_t st);
// prev_b0 < 0: no previous-block update folded in (the caller's field GEMM covered those rows)
// after_inblock: the launch directly follows the previous block's in-block kernel in stream
// order (programmatic dependent launch); otherwise a plain launch
int sk_inblock(const SkDev& d, int b0, int prev_b0, int B, bool after_inblock, cudaStream_t st);
int sk_inblock_prepare();
size_t sk_field_smem_bytes(int B, int kw, int NT);
int sk_field_prepare(int B, int kw, int NT);
int sk_field_update(const SkDev& d, const CUtensorMap& mapJ, const CUtensorMap& mapD, int b0,
                    int B, int kw, int NT, int scale, cudaStream_t st);
// same on every row tile except [skip0, skip1); atomic_add = 1 when another launch may update
// the same rows concurrently
int sk_field_update_rows(const SkDev& d, const CUtensorMap& mapJ, const CUtensorMap& mapD, int b0,
                         int B, int kw, int NT, int scale, int skip0, int skip1, int atomic_add,
                         cudaStream_t st);
size_t sk_plain_smem_bytes(int Np);
int sk_plain_prepare(int Np);
int sk_plain_sweep(const SkDev& d, const uint32_t* clock, uint32_t t_off, cudaStream_t st);
// adds the raw counts (C and q differences, E = 1/2 sum s h) into the destinations
int sk_measure(const SkDev& d, int n_active, int64_t* cdst, int64_t c_stride_r,
               int64_t c_stride_w, int64_t* qdst, int64_t q_stride_p, int64_t* edst,
               int64_t e_stride_r, cudaStream_t st);
int sk_snapshot(const SkDev& d, int w, cudaStream_t st);

}  // namespace sg
