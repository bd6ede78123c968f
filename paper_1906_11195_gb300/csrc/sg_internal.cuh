// sg_internal.cuh -- declarations shared by the host API (sg_api.cu) and the kernel files:
// device layouts, the device-side Philox, and the launch wrappers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sg {

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; in each, counter words 0 and 2
// are multiplied by the two round multipliers, the high halves are mixed into words 1 and 3
// with the round key, and the key advances by the two Weyl increments.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t uint4_word(const uint4& v, int w) {
    return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// --------------------------------------------------------------------------------------------
// shared-memory barriers (mbarrier) and bulk asynchronous copies (inline PTX)
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// bounded wait: false if the barrier phase did not complete within max_iter polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, uint32_t max_iter) {
    for (uint32_t it = 0; it < max_iter; ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// try_wait with a suspend-time hint: an incomplete phase suspends the thread in hardware until
// the phase completes or about hint_ns pass, instead of spinning on the issue slots
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t phase, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// non-blocking test of a phase
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// wait bounded in time: false if the phase did not complete within budget_ns (global timer);
// a zero budget only tests the phase once, without waiting
__device__ __forceinline__ bool mbar_wait_timed(uint64_t* bar, uint32_t phase, uint64_t budget_ns) {
    if (budget_ns == 0) return mbar_test_wait(bar, phase);
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    const uint32_t hint = budget_ns < 1000000ull ? (uint32_t)budget_ns : 1000000u;
    for (;;) {
        if (mbar_try_wait_sleep(bar, phase, hint)) return true;
        if (global_ns() - t0 > budget_ns) return false;
    }
}

// 1-D bulk copy global -> shared (TMA engine), completion counted on an mbarrier in bytes.
// Both addresses must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Same, with an L2 cache-policy operand (createpolicy) attached to the copy.
__device__ __forceinline__ void bulk_copy_g2s_hint(void* dst, const void* src, uint32_t bytes,
                                                   uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// L2 eviction-priority policies: streamed data goes first, the spin array stays
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

constexpr int kVbThrStride = 64;      // thresholds per (graph, replica): m = 0..63
constexpr uint32_t kInactive = 0xFFFFFFFFu;
constexpr int kDegShift = 26;         // vinfo = orig | deg << 26
constexpr uint32_t kOrigMask = (1u << kDegShift) - 1u;

// ---------------------------------------------------------------------------------------------
// Viana-Bray packed layout (sliced ELL over colour-major slots).
// Slots are ordered by (colour, graph, degree descending, original label); every (colour, graph) group is
// padded to a multiple of 32 slots, so a warp-sized slice has one colour and one graph.
// ---------------------------------------------------------------------------------------------
struct VbPackedDev {
    const uint32_t* vinfo;       // [n_slots] orig | deg << 26, kInactive for padding slots
    const uint32_t* slice_base;  // [n_slices+1] first entry of each slice (entries of 32 lanes)
    const uint32_t* slice_graph; // [n_slices] graph index
    const uint32_t* col;         // [n_entries] neighbour slot (self for padding entries)
    const uint64_t* jb;          // [n_entries] coupling word (0 for padding entries)
    const uint64_t* seeds;       // [n_graphs]
    const uint32_t* thr;         // [n_graphs][R][64]
    const uint4* groups;         // [n_groups] {first slice, slices, first entry, entries}
    const uint4* slice_meta;     // [n_slices] {first entry, width, graph, upper}: upper =
                                 // max entries to later colour classes | kind << 16
    const uint32_t* group_graph; // [n_groups] graph of each group (groups never mix graphs)
    const uint8_t* gtab;         // [n_graphs] {uint32 thr[R][64]; uint64 seed; uint64 pad}
    const uint32_t* colour_groups;  // [n_colours+1] first group of each colour class
    int* err;                    // device status word (bounded waits)
    uint32_t* gbar;              // [2] grid-barrier arrivals and exits of a fused sweep (zeroed)
    uint64_t* S;                 // [n_slots][R]
    uint64_t* snap;              // [n_tw][n_slots][R]
    // upper entries for the energy: per slice, each lane's neighbours in later colour classes
    // (higher slots), sliced-ELL like col/jb; every edge appears once
    const uint32_t* up_slice_base;  // [n_slices+1] (null: count over every directed entry)
    const uint32_t* up_col;
    const uint64_t* up_jb;
    int64_t n_slots;
    int32_t n_slices;
    int32_t R;
    int32_t n_colours;
    uint64_t stage_wait_ns;      // bound of one pipeline wait in the colour kernel
};

constexpr int kVbMaxColours = 64;  // greedy colouring with degree <= 63

// Viana-Bray plain layout (one graph, colour-major CSR, int8 spins per lane).
struct VbPlainDev {
    const int32_t* row_ptr;  // [N+1] in colour-major labels
    const int32_t* col;      // [2M]
    const uint64_t* jb;      // [2M]
    const uint32_t* orig;    // [N] original label of each new label
    const uint32_t* thr;     // [R][64]
    int8_t* s;               // [R][L][N]
    int8_t* snap;            // [n_tw][R][L][N]
    uint64_t seed;
    int32_t N, R, L;
};

// A measurement: per-lane counts of differences, accumulated with atomics into
// dst[g * stride_g + r * stride_r + k * stride_k] (g graph, r replica or pair, k lane).
//   kind 0: Hamming distance between the spins and snapshot w (all replicas)
//   kind 1: Hamming distance between replicas 2p and 2p+1 (all pairs)
//   kind 2: number of unsatisfied directed entries, J_ij s_i s_j = -1 (all replicas)
// kind 0: C against snapshot w; 1: q; 2: E; 3 (packed only): C against snapshots 0 .. w-1 in
// one pass (snapshot k adds at dst + k * stride_w), reading the current spins once
struct VbCountJob {
    int kind;
    int w;
    int64_t* dst;
    int64_t stride_g, stride_r, stride_k;
    int64_t stride_w;
    int shift;  // counts are added times 2^shift (the energy over upper entries counts each
                // edge once and reports the number of unsatisfied directed entries, twice that)
};

// slice_meta.w >> 16: how a slice's entries lie relative to its colour class (every entry of
// every vertex goes to a later class / none does / some do)
constexpr uint32_t kUpAll = 1u, kUpNone = 0u, kUpMixed = 2u;

// The energy a measuring sweep takes of the state it starts from (one instance): per-lane
// unsatisfied directed entries added at e_dst[r * stride_r + k * stride_k] (r replica, k lane).
struct VbSweepMeas {
    int64_t* e_dst;
    int64_t stride_r, stride_k;
};

// launch wrappers (vb_kernels.cu); each returns the number of kernel launches queued
int vb_packed_init(const VbPackedDev& d, cudaStream_t st);
// sweep index t = *clock + t_off (the clock lives in device memory so that captured CUDA graphs
// can be replayed at any time)
// One sweep of every colour class in colour order.  variant (0 .. kVbColourVariants - 1)
// selects the pipeline shape (stream stages, gather buffers, gather lookahead, CTAs per SM);
// fused runs the classes in one cooperative launch with grid-wide barriers between them
// (R = 2, 4), else one launch per class.  colour_groups is the host copy of d.colour_groups.
// No choice changes the results.  Returns the launches queued, or -1.
int vb_packed_sweep(const VbPackedDev& d, const uint32_t* colour_groups, const uint32_t* clock,
                    uint32_t t_off, int variant, bool fused, cudaStream_t st);
constexpr int kVbColourVariants = 3;
// The same sweep (same spins, same random numbers) that also adds the energy of the state it
// starts from (vb_colour_meas.cu); single-instance layouts only.
int vb_packed_sweep_meas(const VbPackedDev& d, const uint32_t* colour_groups,
                         const uint32_t* clock, uint32_t t_off, int variant, bool fused,
                         const VbSweepMeas& meas, cudaStream_t st);
int vb_packed_snapshot(const VbPackedDev& d, int w, cudaStream_t st);
// the upper entries (each vertex's neighbours in later colour classes, padded with the vertex
// itself and J = 0) from col and jb, given up_slice_base
int vb_packed_build_upper(const VbPackedDev& d, cudaStream_t st);
// also_q (kind 1, with job of kind 0 or 3): the replica overlaps in the same launch, one more
// pass over the warp's slices (whose current spins are still in L1)
int vb_packed_count(const VbPackedDev& d, const VbCountJob& job, cudaStream_t st,
                    const VbCountJob* also_q = nullptr);

int vb_plain_init(const VbPlainDev& d, cudaStream_t st);
int vb_plain_colour(const VbPlainDev& d, int32_t v_begin, int32_t v_end, const uint32_t* clock,
                    uint32_t t_off, cudaStream_t st);
int vb_plain_snapshot(const VbPlainDev& d, int w, cudaStream_t st);
int vb_plain_count(const VbPlainDev& d, const VbCountJob& job, cudaStream_t st);

}  // namespace sg
