// sk_internal.cuh -- Sherrington-Kirkpatrick device layout and launch wrappers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

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

int sk_init(const SkDev& d, cudaStream_t st);
int sk_kstar_sweep(const SkDev& d, const uint32_t* clock, uint32_t t_off, cudaStream_t st);
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
