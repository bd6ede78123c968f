// vb_colour.cuh -- the packed VB colour-class sweep (multispin coding, SI section 2; one colour
// class, an independent set, at a time: the generalisation of the bipartite half-updates of SI
// section 3).  Included by vb_kernels.cu (plain sweeps) and vb_colour_meas.cu (sweeps that also
// measure the energy of the state they start from), so that the two sets of instantiations
// compile in parallel.
#pragma once

#include "../../include/sg.h"
#include "sg_internal.cuh"

namespace sg {

// ---------------------------------------------------------------------------------------------
// packed: one colour class
// ---------------------------------------------------------------------------------------------
template <int R>
struct SpinWords { uint64_t v[R]; };

template <int R>
__device__ __forceinline__ SpinWords<R> load_words(const uint64_t* p) {
    SpinWords<R> s;
    if constexpr (R == 1) {
        s.v[0] = p[0];
    } else if constexpr (R == 2) {
        const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(p);
        s.v[0] = a.x; s.v[1] = a.y;
    } else {
        const ulonglong2 a = reinterpret_cast<const ulonglong2*>(p)[0];
        const ulonglong2 b = reinterpret_cast<const ulonglong2*>(p)[1];
        s.v[0] = a.x; s.v[1] = a.y; s.v[2] = b.x; s.v[3] = b.y;
    }
    return s;
}

template <int R>
__device__ __forceinline__ SpinWords<R> gather_words(const uint64_t* p) {
    SpinWords<R> s;
    if constexpr (R == 1) {
        s.v[0] = __ldg(p);
    } else if constexpr (R == 2) {
        const ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2*>(p));
        s.v[0] = a.x; s.v[1] = a.y;
    } else {
        const ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2*>(p));
        const ulonglong2 b = __ldcg(reinterpret_cast<const ulonglong2*>(p) + 1);
        s.v[0] = a.x; s.v[1] = a.y; s.v[2] = b.x; s.v[3] = b.y;
    }
    return s;
}

template <int R>
__device__ __forceinline__ void store_words_keep(uint64_t* p, const SpinWords<R>& s, uint64_t pol) {
    if constexpr (R == 1) {
        asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(s.v[0]), "l"(pol)
                     : "memory");
    } else {
#pragma unroll
        for (int h = 0; h < R / 2; ++h)
            asm volatile("st.global.L2::cache_hint.v2.u64 [%0], {%1, %2}, %3;" ::"l"(p + 2 * h),
                         "l"(s.v[2 * h]), "l"(s.v[2 * h + 1]), "l"(pol)
                         : "memory");
    }
}

constexpr int kGroupSlices = 8;       // slices (warps) per staged group
constexpr int kGroupEntries = 1024;   // staged sliced-ELL entries per group

// add one 64-lane word into a P-plane bit-sliced counter (the count never exceeds 2^P - 1)
template <int P>
__device__ __forceinline__ void bitslice_add(uint64_t (&p)[P], uint64_t x) {
#pragma unroll
    for (int b = 0; b < P; ++b) {
        const uint64_t c = p[b] & x;
        p[b] ^= x;
        x = c;
    }
}

// lanes whose counter value is >= k (k a per-thread scalar, 0 <= k <= 2^P - 1)
template <int P>
__device__ __forceinline__ uint64_t bitslice_ge(const uint64_t (&p)[P], int k) {
    uint64_t gt = 0ull, eq = ~0ull;
#pragma unroll
    for (int b = P - 1; b >= 0; --b) {
        const uint64_t kb = ((k >> b) & 1) ? ~0ull : 0ull;
        gt |= eq & p[b] & ~kb;
        eq &= ~(p[b] ^ kb);
    }
    return gt | eq;
}

// Pipelined colour-class kernel.  The slices of a colour class are cut into groups of at most
// kGroupSlices slices (one warp each) and kGroupEntries sliced-ELL entries.  Per group, two kinds
// of data move into shared memory:
//   * the stream part (group descriptor, vinfo, own spin words, slice metadata, neighbour slots,
//     coupling words, the graph's thresholds and key), which depends on nothing the sweep
//     writes, is staged by bulk asynchronous copies (completion on the stage's mbarrier) several
//     groups ahead, to cover the DRAM latency;
//   * the neighbours' spin words, which must be read after the previous colour class finished,
//     are gathered with 16-byte cp.async copies into a separate, smaller ring of gather buffers,
//     L groups ahead of the computation, to cover the L2 latency.
// The computation of a group then reads everything from shared memory.  Keeping the two rings
// apart lets the stream ring run deep without reserving gather space for groups whose copies
// are still in flight.  A group holding one slice wider than the stage (degree > 32, flagged by
// the host) is computed straight from global memory.
constexpr uint32_t kWideGroup = 0x80000000u;

template <int R>
struct VbStream {
    uint64_t J[kGroupEntries];
    uint32_t col[kGroupEntries];
    uint64_t S[kGroupSlices * 32 * R];
    uint32_t vinfo[kGroupSlices * 32];
    uint4 meta[kGroupSlices];        // per slice: first entry, width, graph, 0
    uint32_t thr[R * kVbThrStride];  // the group's graph: thresholds of its replicas ...
    uint64_t seed[2];                // ... and its Philox key
    uint4 gi;                        // group descriptor: first slice, slices (| wide), entry, entries
};

template <int R>
struct VbGath {
    uint64_t v[kGroupEntries * R];
};

// Energy taken by a measuring sweep from the state it starts from: per vertex, the
// unsatisfied edges to neighbours in later colour classes (slot > own slot; the classes are
// laid out in colour order), which the sweep has not updated yet when it updates the vertex, so
// both ends still hold their start values; each edge is counted once, at its earlier-class end.
// Per-lane counts accumulate in kMeasPlanes-plane bit-sliced counters per thread (at most
// kMeasMax between two flushes through the CTA-shared accumulator; with 8 planes a warp rarely
// flushes before the end of the launch).
constexpr int kMeasPlanes = 8;
constexpr uint32_t kMeasMax = (1u << kMeasPlanes) - 1u;  // >= SG_VB_MAX_DEGREE
static_assert(kMeasMax >= SG_VB_MAX_DEGREE, "one slice's entries fit an empty counter");

template <int R>
struct MeasAcc { uint64_t e[R][kMeasPlanes]; };

// a += x (a P-plane count, P <= kMeasPlanes); the caller keeps the sum below 2^kMeasPlanes
template <int P>
__device__ __forceinline__ void meas_add(uint64_t (&a)[kMeasPlanes], const uint64_t (&x)[P]) {
    static_assert(P <= kMeasPlanes, "count wider than the accumulator");
    uint64_t c = 0ull;
#pragma unroll
    for (int b = 0; b < kMeasPlanes; ++b) {
        if (b < P) {
            const uint64_t s = a[b] ^ x[b] ^ c;
            c = (a[b] & x[b]) | (c & (a[b] ^ x[b]));
            a[b] = s;
        } else {
            const uint64_t s = a[b] ^ c;
            c = a[b] & c;
            a[b] = s;
        }
    }
}

// Count the unsatisfied edges of one vertex (all lanes, all replicas) with a P-plane counter
// and flip the lanes whose count reaches kmin.  Neighbour words come from the gather buffer, or
// straight from global memory for a wide slice (J == nullptr).  MEAS: the entries to later
// classes are counted again into the energy accumulator, before the flip.
template <int R, int P, bool MEAS>
__device__ __forceinline__ void count_and_flip(SpinWords<R>& si, const uint64_t* J,
                                               const uint32_t* col, const uint64_t* gath,
                                               uint32_t loc, uint32_t width, const VbPackedDev& d,
                                               uint32_t idx, uint32_t slot, const int (&kmin)[R],
                                               MeasAcc<R>& acc, uint32_t kind) {
    if constexpr (!MEAS) {
        uint64_t planes[R][P];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int b = 0; b < P; ++b) planes[r][b] = 0ull;
        if (J) {
            for (uint32_t e = 0; e < width; ++e, loc += 32) {
                const uint64_t Je = J[loc];
#pragma unroll
                for (int r = 0; r < R; ++r) bitslice_add<P>(planes[r], si.v[r] ^ gath[loc * R + r] ^ Je);
            }
        } else {
            for (uint32_t e = 0; e < width; ++e, idx += 32) {
                const uint32_t j = __ldg(d.col + idx);
                const uint64_t Je = __ldg(d.jb + idx);
                const SpinWords<R> sj = gather_words<R>(d.S + (int64_t)j * R);
#pragma unroll
                for (int r = 0; r < R; ++r) bitslice_add<P>(planes[r], si.v[r] ^ sj.v[r] ^ Je);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) si.v[r] ^= bitslice_ge<P>(planes[r], kmin[r]);
    } else {
        // one replica at a time (the entries are read again per replica), so that only two
        // counters are live beside the accumulator; a slice whose entries all go to later
        // classes adds the flip count itself
        const bool mixed = kind == kUpMixed;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            uint64_t planes[P], up[P];
#pragma unroll
            for (int b = 0; b < P; ++b) planes[b] = up[b] = 0ull;
            if (J) {
                uint32_t l = loc;
                for (uint32_t e = 0; e < width; ++e, l += 32) {
                    const uint64_t x = si.v[r] ^ gath[l * R + r] ^ J[l];
                    bitslice_add<P>(planes, x);
                    if (mixed) bitslice_add<P>(up, col[l] > slot ? x : 0ull);
                }
            } else {
                uint32_t ix = idx;
                for (uint32_t e = 0; e < width; ++e, ix += 32) {
                    const uint32_t j = __ldg(d.col + ix);
                    const uint64_t x = si.v[r] ^ __ldcg(d.S + (int64_t)j * R + r) ^ __ldg(d.jb + ix);
                    bitslice_add<P>(planes, x);
                    if (mixed) bitslice_add<P>(up, j > slot ? x : 0ull);
                }
            }
            if (mixed) meas_add<P>(acc.e[r], up);
            else if (kind == kUpAll) meas_add<P>(acc.e[r], planes);
            si.v[r] ^= bitslice_ge<P>(planes, kmin[r]);
        }
    }
}

// --- narrow slices (width <= 8): unrolled carry-save counting --------------------------------
// full adder and half adder on 64 lanes at once (each lowers to 3-input logic operations)
__device__ __forceinline__ void full_add(uint64_t a, uint64_t b, uint64_t c, uint64_t& s,
                                         uint64_t& cy) {
    s = a ^ b ^ c;
    cy = (a & b) | (c & (a ^ b));
}

__device__ __forceinline__ void half_add(uint64_t a, uint64_t b, uint64_t& s, uint64_t& cy) {
    s = a ^ b;
    cy = a & b;
}

// planes needed to count W one-bit inputs
template <int W>
struct CountBits { static constexpr int P = W <= 1 ? 1 : W <= 3 ? 2 : W <= 7 ? 3 : 4; };

// p = bit-sliced number of set inputs among x[0..W-1], per lane (carry-save adder trees)
template <int W>
__device__ __forceinline__ void count_bits(const uint64_t (&x)[W], uint64_t (&p)[CountBits<W>::P]) {
    if constexpr (W == 1) {
        p[0] = x[0];
    } else if constexpr (W == 2) {
        half_add(x[0], x[1], p[0], p[1]);
    } else if constexpr (W == 3) {
        full_add(x[0], x[1], x[2], p[0], p[1]);
    } else if constexpr (W == 4 || W == 5) {
        uint64_t s1, c1, c2;
        full_add(x[0], x[1], x[2], s1, c1);
        if constexpr (W == 4) half_add(s1, x[3], p[0], c2);
        else full_add(s1, x[3], x[4], p[0], c2);
        half_add(c1, c2, p[1], p[2]);
    } else if constexpr (W == 6 || W == 7) {
        uint64_t s1, c1, s2, c2, c3;
        full_add(x[0], x[1], x[2], s1, c1);
        full_add(x[3], x[4], x[5], s2, c2);
        if constexpr (W == 6) half_add(s1, s2, p[0], c3);
        else full_add(s1, s2, x[6], p[0], c3);
        full_add(c1, c2, c3, p[1], p[2]);
    } else {
        static_assert(W == 8, "narrow path covers widths 1..8");
        uint64_t s1, c1, s2, c2, s3, c3, c4;
        full_add(x[0], x[1], x[2], s1, c1);
        full_add(x[3], x[4], x[5], s2, c2);
        full_add(s1, s2, x[6], s3, c3);
        half_add(s3, x[7], p[0], c4);
        // the four weight-2 carries
        uint64_t t1, d1, d2;
        full_add(c1, c2, c3, t1, d1);
        half_add(t1, c4, p[1], d2);
        half_add(d1, d2, p[2], p[3]);
    }
}

// lanes whose P-plane count u is >= k (0 <= k <= 2^P - 1): the carry out of u + (2^P - k)
template <int P>
__device__ __forceinline__ uint64_t at_least(const uint64_t (&p)[P], int k) {
    const uint32_t c = (1u << P) - (uint32_t)k;
    uint64_t carry = 0ull;
#pragma unroll
    for (int b = 0; b < P; ++b) {
        const uint64_t cb = ((c >> b) & 1u) ? ~0ull : 0ull;
        carry = (p[b] & carry) | (cb & (p[b] | carry));
    }
    return k == 0 ? ~0ull : carry;
}

template <int R, int W, bool MEAS>
__device__ __forceinline__ void count_and_flip_narrow(SpinWords<R>& si, const uint64_t* J,
                                                      const uint32_t* col, const uint64_t* gath,
                                                      uint32_t loc, uint32_t slot,
                                                      const int (&kmin)[R], MeasAcc<R>& acc,
                                                      uint32_t kind) {
    if constexpr (!MEAS) {
        uint64_t x[R][W];
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const uint64_t Je = J[loc + 32 * e];
#pragma unroll
            for (int r = 0; r < R; ++r) x[r][e] = si.v[r] ^ gath[(loc + 32 * e) * R + r] ^ Je;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            uint64_t p[CountBits<W>::P];
            count_bits<W>(x[r], p);
            si.v[r] ^= at_least<CountBits<W>::P>(p, kmin[r]);
        }
    } else {
        // one replica at a time: the energy count over the entries to later classes (a slice
        // whose entries all go there reuses the flip count), then the flip count over all
#pragma unroll
        for (int r = 0; r < R; ++r) {
            uint64_t x[W];
#pragma unroll
            for (int e = 0; e < W; ++e) x[e] = si.v[r] ^ gath[(loc + 32 * e) * R + r] ^ J[loc + 32 * e];
            uint64_t p[CountBits<W>::P];
            if (kind == kUpMixed) {
                uint64_t xu[W];
#pragma unroll
                for (int e = 0; e < W; ++e) xu[e] = col[loc + 32 * e] > slot ? x[e] : 0ull;
                count_bits<W>(xu, p);
                meas_add<CountBits<W>::P>(acc.e[r], p);
            }
            count_bits<W>(x, p);
            if (kind == kUpAll) meas_add<CountBits<W>::P>(acc.e[r], p);
            si.v[r] ^= at_least<CountBits<W>::P>(p, kmin[r]);
        }
    }
}

// 2 s: a stage is late only if something broke.  The pipeline waits use the handle's
// d.stage_wait_ns (this value unless a test shortens it); the drains before a CTA exits always
// use this one, so no copy can still be landing when the CTA is gone.
constexpr uint64_t kStageWaitNs = 2000000000ull;

template <int R>
__device__ __forceinline__ void gather_async(uint64_t* dst, const uint64_t* src, uint64_t pol) {
    if constexpr (R == 1) {
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;" ::"r"(
                         smem_addr(dst)), "l"(src), "l"(pol)
                     : "memory");
    } else {
#pragma unroll
        for (int h = 0; h < R / 2; ++h)
            asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                             smem_addr(dst + 2 * h)), "l"(src + 2 * h), "l"(pol)
                         : "memory");
    }
}

// the W neighbour gathers of one lane of a narrow slice: slots first, then the copies
template <int R, int W>
__device__ __forceinline__ void gather_n(uint64_t* gath, const uint32_t* col, uint32_t loc,
                                         const uint64_t* S, uint64_t pol) {
    uint32_t j[W];
#pragma unroll
    for (int e = 0; e < W; ++e) j[e] = col[loc + 32 * e];
#pragma unroll
    for (int e = 0; e < W; ++e) gather_async<R>(&gath[(loc + 32 * e) * R], S + (int64_t)j[e] * R, pol);
}

// Acceptance constants of one vertex (all replicas): one Philox block per (vertex, sweep) serves
// replicas 0..3; the accepted m form a prefix 1..m*, so a lane flips iff its unsatisfied count u
// reaches kmin = ceil((d - m*) / 2).  Independent of the neighbours, so a consumer warp computes
// it for the next group while the current group's gathers are still in flight.
template <int R>
__device__ __forceinline__ void acceptance(const VbStream<R>& st, uint32_t warp, uint32_t lane,
                                           uint32_t t, int (&kmin)[R]) {
    const uint32_t vi = st.vinfo[warp * 32 + lane];
    const int deg = vi == kInactive ? 0 : (int)(vi >> kDegShift);
    const uint32_t orig = vi & kOrigMask;
    const uint64_t seed = st.seed[0];
    const uint4 rnd =
        philox4x32_10(make_uint4(orig, t, 0u, 0u), (uint32_t)seed, (uint32_t)(seed >> 32));
    // thr is non-increasing, so most draws stop at m = 1: read that entry for every replica
    // at once, and walk on only where it is accepted
    uint32_t t1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) t1[r] = st.thr[r * kVbThrStride + 1];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t r32 = uint4_word(rnd, r);
        int ms = 0;
        if (deg > 0 && r32 < t1[r]) {
            ms = 1;
            while (ms < deg && r32 < st.thr[r * kVbThrStride + ms + 1]) ++ms;
        }
        kmin[r] = (deg - ms + 1) >> 1;
    }
}

// One consumer warp's work on one slice of a staged group (neighbour words already gathered).
template <int R, bool MEAS>
__device__ __forceinline__ void update_slice(const VbPackedDev& d, const VbStream<R>& st,
                                             const uint64_t* gath, const uint4& gi, uint32_t warp,
                                             uint32_t lane, const int (&kmin)[R],
                                             uint64_t pol_keep, MeasAcc<R>& acc) {
    const bool wide = (gi.y & kWideGroup) != 0u;
    const uint32_t slice = gi.x + warp;
    const uint32_t vi = st.vinfo[warp * 32 + lane];
    if (vi == kInactive) return;
    const uint4 m = st.meta[warp];  // first entry, width, graph, upper entries
    const uint32_t width = m.y;
    const uint32_t kind = m.w >> 16;
    SpinWords<R> si;
#pragma unroll
    for (int r = 0; r < R; ++r) si.v[r] = st.S[(warp * 32 + lane) * R + r];
    const uint64_t* J = wide ? nullptr : st.J;
    const uint32_t loc = m.x - gi.z + lane, idx = m.x + lane;
    const uint32_t slot32 = slice * 32u + lane;  // this vertex's slot (slots < 2^32)
    // the slice's width (warp-uniform) selects the code: unrolled carry-save counting for the
    // common narrow slices of a staged group, a ripple counter sized by the width otherwise
    if (J && width <= 8) {
        switch (width) {
            case 0:  // isolated vertices: dE = 0, every lane flips (kmin = 0)
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (kmin[r] == 0) si.v[r] = ~si.v[r];
                break;
            case 1: count_and_flip_narrow<R, 1, MEAS>(si, J, st.col, gath, loc, slot32, kmin, acc, kind); break;
            case 2: count_and_flip_narrow<R, 2, MEAS>(si, J, st.col, gath, loc, slot32, kmin, acc, kind); break;
            case 3: count_and_flip_narrow<R, 3, MEAS>(si, J, st.col, gath, loc, slot32, kmin, acc, kind); break;
            case 4: count_and_flip_narrow<R, 4, MEAS>(si, J, st.col, gath, loc, slot32, kmin, acc, kind); break;
            case 5: count_and_flip_narrow<R, 5, MEAS>(si, J, st.col, gath, loc, slot32, kmin, acc, kind); break;
            case 6: count_and_flip_narrow<R, 6, MEAS>(si, J, st.col, gath, loc, slot32, kmin, acc, kind); break;
            case 7: count_and_flip_narrow<R, 7, MEAS>(si, J, st.col, gath, loc, slot32, kmin, acc, kind); break;
            default: count_and_flip_narrow<R, 8, MEAS>(si, J, st.col, gath, loc, slot32, kmin, acc, kind); break;
        }
    } else if (width <= 1) count_and_flip<R, 1, MEAS>(si, J, st.col, gath, loc, width, d, idx, slot32, kmin, acc, kind);
    else if (width <= 3) count_and_flip<R, 2, MEAS>(si, J, st.col, gath, loc, width, d, idx, slot32, kmin, acc, kind);
    else if (width <= 7) count_and_flip<R, 3, MEAS>(si, J, st.col, gath, loc, width, d, idx, slot32, kmin, acc, kind);
    else if (width <= 15) count_and_flip<R, 4, MEAS>(si, J, st.col, gath, loc, width, d, idx, slot32, kmin, acc, kind);
    else if (width <= 31) count_and_flip<R, 5, MEAS>(si, J, st.col, gath, loc, width, d, idx, slot32, kmin, acc, kind);
    else count_and_flip<R, 6, MEAS>(si, J, st.col, gath, loc, width, d, idx, slot32, kmin, acc, kind);
    store_words_keep<R>(d.S + ((int64_t)slice * 32 + lane) * R, si, pol_keep);
}

// Grid-wide barrier between colour classes of one launch, taken by the 256 consumer threads of
// every CTA (the producer warp keeps staging).  `alive` is this thread's health; the CTA joins
// the grid barrier only if every consumer thread is alive, so a CTA that gave up makes the
// others time out (bounded) instead of hanging.  Returns the same value to all consumers.
constexpr uint32_t kGridPolls = 1u << 22;

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool consumers_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 256, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0u;
}

__device__ __forceinline__ bool grid_barrier(uint32_t* count, uint32_t target, int* err,
                                             uint32_t tid, bool alive) {
    __shared__ int passed;
    if (!consumers_all(alive)) return false;  // also orders this CTA's spin stores before the fence
    if (tid == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        int ok = 1;
        for (uint32_t polls = 0; ld_acquire_gpu(count) < target; ++polls) {
            if (polls >= kGridPolls) {
                atomicOr(err, 8);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        passed = ok;
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    return passed != 0;
}

// Add the warp's energy counters into the CTA-shared accumulator ([R][64] per-lane counts) and
// clear them: a butterfly of bit-sliced additions sums the 32 threads (the total of one lane is
// at most 32 kMeasMax, kMeasPlanes + 5 planes), then lane l adds the totals of spin lanes l and
// l + 32.  Warp-wide: every lane of the warp calls it.  Kept out of line: the call sites sit in
// the update loop, whose registers it would otherwise crowd.
template <int R>
__device__ __noinline__ void meas_flush(MeasAcc<R>& acc, unsigned long long* s_meas,
                                           uint32_t lane) {
    constexpr int PW = kMeasPlanes + 5;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        uint64_t p[PW];
#pragma unroll
        for (int b = 0; b < PW; ++b) p[b] = b < kMeasPlanes ? acc.e[r][b] : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            uint64_t carry = 0ull;
#pragma unroll
            for (int b = 0; b < PW; ++b) {
                const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, p[b], off);
                const uint64_t x = p[b] ^ o;
                const uint64_t sum = x ^ carry;
                carry = (p[b] & o) | (carry & x);
                p[b] = sum;
            }
        }
        uint32_t c0 = 0, c1 = 0;
#pragma unroll
        for (int b = 0; b < PW; ++b) {
            c0 |= (uint32_t)((p[b] >> lane) & 1ull) << b;
            c1 |= (uint32_t)((p[b] >> (lane + 32)) & 1ull) << b;
        }
        if (c0) atomicAdd(s_meas + r * 64 + lane, (unsigned long long)c0);
        if (c1) atomicAdd(s_meas + r * 64 + lane + 32, (unsigned long long)c1);
#pragma unroll
        for (int b = 0; b < kMeasPlanes; ++b) acc.e[r][b] = 0ull;
    }
}

// Warp-specialised, persistent colour-class kernel over the colour classes [c_begin, c_end) of
// one sweep.  Warp kGroupSlices (the producer) stages the stream part of the CTA's groups, in
// colour order, into a ring of NSS stages ("full" mbarrier: bytes landed; "empty": released by
// the 8 consumer warps); it runs ahead across colour boundaries, which is safe because the
// stream part holds nothing a colour class writes (a class writes only its own vertices' words,
// staged when that class is reached).  Consumer warp w owns slice w of every group: it starts
// the cp.async gathers of its neighbours' words for the group L ahead (within the class) into
// gather buffer (k + L) mod NG once every warp has released it ("gfree" mbarrier), waits for the
// gathers of the current group, updates its 32 vertices and releases both.  Between two classes
// the consumers of all CTAs meet at a grid-wide barrier, so no gather of class c + 1 is issued
// before every word of class c is written; such launches are cooperative (all CTAs resident).
// MEAS (a graph of one instance): the sweep also adds the energy of the state it starts from
// into meas.e_dst, two per unsatisfied edge (the directed count), flushed once per CTA.
template <int R, int NSS, int NG, int L, bool MEAS>
__device__ __forceinline__ void colour_sweep(const VbPackedDev& d, uint32_t c_begin, uint32_t c_end,
                                             const uint32_t* __restrict__ clock, uint32_t t_off,
                                             const VbSweepMeas& meas) {
    static_assert(L >= 1 && L < NG && L < NSS, "gathers run L groups ahead inside both rings");
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ uint32_t s_kc[kVbMaxColours + 1];  // first ring index of each class (this CTA)
    __shared__ uint32_t s_cg[kVbMaxColours];      // first group of each class
    __shared__ unsigned long long s_meas[MEAS ? R * 64 : 1];
    VbStream<R>* stream = reinterpret_cast<VbStream<R>*>(smem_raw);
    VbGath<R>* gath = reinterpret_cast<VbGath<R>*>(stream + NSS);
    uint64_t* full = reinterpret_cast<uint64_t*>(gath + NG);
    uint64_t* empty = full + NSS;
    uint64_t* gfree = empty + NSS;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t t = __ldg(clock) + t_off;
    const uint64_t* __restrict__ S = d.S;
    const uint64_t pol_stream = l2_evict_first(), pol_keep = l2_evict_last();
    const uint32_t nc = c_end - c_begin;

    if (tid == 0) {
        for (int s = 0; s < NSS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kGroupSlices);
        }
        for (int b = 0; b < NG; ++b) mbar_init(&gfree[b], kGroupSlices);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        uint32_t acc = 0;
        for (uint32_t j = 0; j < nc; ++j) {
            const uint32_t a = __ldg(&d.colour_groups[c_begin + j]);
            const uint32_t b = __ldg(&d.colour_groups[c_begin + j + 1]);
            s_cg[j] = a;
            s_kc[j] = acc;
            acc += a + blockIdx.x < b ? (b - a - blockIdx.x + gridDim.x - 1) / gridDim.x : 0u;
        }
        s_kc[nc] = acc;
    }
    if constexpr (MEAS)
        for (uint32_t i = tid; i < (uint32_t)R * 64u; i += blockDim.x) s_meas[i] = 0ull;
    __syncthreads();
    const uint32_t n_mine = s_kc[nc];

    if (warp == kGroupSlices) {
        // ------------------------------------------------------------------ producer
        if (lane == 0 && n_mine) {
            const uint32_t gtab_bytes = R * kVbThrStride * 4u + 16u;
            auto group_of = [&](uint32_t k, uint32_t& j) -> uint32_t {
                while (k >= s_kc[j + 1]) ++j;
                return s_cg[j] + blockIdx.x + (k - s_kc[j]) * gridDim.x;
            };
            uint32_t jn = 0;
            uint32_t g_next = group_of(0, jn);
            uint4 gi_next = __ldg(&d.groups[g_next]);
            uint32_t graph_next = __ldg(&d.group_graph[g_next]);
            uint32_t issued = 0;
            for (uint32_t k = 0; k < n_mine; ++k) {
                const uint4 gi = gi_next;
                const uint32_t graph = graph_next;
                if (k + 1 < n_mine) {  // the next descriptor's load overlaps this group's issue
                    g_next = group_of(k + 1, jn);
                    gi_next = __ldg(&d.groups[g_next]);
                    graph_next = __ldg(&d.group_graph[g_next]);
                }
                const int s = (int)(k % NSS);
                if (k >= (uint32_t)NSS &&
                    !mbar_wait_timed(&empty[s], ((k / NSS) - 1) & 1u, d.stage_wait_ns)) {
                    atomicOr(d.err, 4);
                    break;
                }
                const uint32_t nsl = gi.y & ~kWideGroup;
                const bool wide = (gi.y & kWideGroup) != 0u;
                const uint32_t nslot = nsl * 32u;
                const uint32_t bytes = nslot * 4u + nslot * R * 8u + nsl * 16u + gtab_bytes +
                                       (wide ? 0u : gi.w * 12u);
                stream[s].gi = gi;  // published by the arrive below (release semantics)
                mbar_expect_tx(&full[s], bytes);
                bulk_copy_g2s_hint(stream[s].meta, d.slice_meta + gi.x, nsl * 16u, &full[s],
                                   pol_stream);
                bulk_copy_g2s(stream[s].thr, d.gtab + (size_t)graph * gtab_bytes, gtab_bytes,
                              &full[s]);
                bulk_copy_g2s_hint(stream[s].vinfo, d.vinfo + (int64_t)gi.x * 32, nslot * 4u,
                                   &full[s], pol_stream);
                bulk_copy_g2s_hint(stream[s].S, S + (int64_t)gi.x * 32 * R, nslot * R * 8u,
                                   &full[s], pol_keep);
                if (gi.w && !wide) {
                    bulk_copy_g2s_hint(stream[s].col, d.col + gi.z, gi.w * 4u, &full[s],
                                       pol_stream);
                    bulk_copy_g2s_hint(stream[s].J, d.jb + gi.z, gi.w * 8u, &full[s], pol_stream);
                }
                issued = k + 1;
            }
            // no copy may still be landing in shared memory when the CTA exits (the consumers
            // wait for every stage they use; this matters only after a timeout)
            for (uint32_t k = issued > (uint32_t)NSS ? issued - NSS : 0u; k < issued; ++k)
                if (!mbar_wait_timed(&full[k % NSS], (k / NSS) & 1u, kStageWaitNs)) atomicOr(d.err, 4);
        }
        return;
    }

    // ---------------------------------------------------------------------- consumers
    // start the gathers of this warp's slice of group k if k < k_end (its stream stage has
    // landed and every warp has released the gather buffer's previous group)
    auto gathers = [&](uint32_t k, uint32_t k_end) -> bool {
        if (k < k_end) {
            const int s = (int)(k % NSS), b = (int)(k % NG);
            if (!mbar_wait_timed(&full[s], (k / NSS) & 1u, d.stage_wait_ns)) return false;
            if (k >= (uint32_t)NG && !mbar_wait_timed(&gfree[b], ((k / NG) - 1) & 1u, d.stage_wait_ns))
                return false;
            const uint4 gi = stream[s].gi;
            const uint32_t nsl = gi.y & ~kWideGroup;
            if (warp < nsl && !(gi.y & kWideGroup) &&
                stream[s].vinfo[warp * 32 + lane] != kInactive) {
                const uint4 m = stream[s].meta[warp];
                const uint32_t loc = m.x - gi.z + lane;
                switch (m.y) {  // narrow slices: every slot read before the first copy is issued
                    case 1: gather_n<R, 1>(gath[b].v, stream[s].col, loc, S, pol_keep); break;
                    case 2: gather_n<R, 2>(gath[b].v, stream[s].col, loc, S, pol_keep); break;
                    case 3: gather_n<R, 3>(gath[b].v, stream[s].col, loc, S, pol_keep); break;
                    case 4: gather_n<R, 4>(gath[b].v, stream[s].col, loc, S, pol_keep); break;
                    case 5: gather_n<R, 5>(gath[b].v, stream[s].col, loc, S, pol_keep); break;
                    case 6: gather_n<R, 6>(gath[b].v, stream[s].col, loc, S, pol_keep); break;
                    case 7: gather_n<R, 7>(gath[b].v, stream[s].col, loc, S, pol_keep); break;
                    case 8: gather_n<R, 8>(gath[b].v, stream[s].col, loc, S, pol_keep); break;
                    default:
                        for (uint32_t e = 0, l = loc; e < m.y; ++e, l += 32)
                            gather_async<R>(&gath[b].v[l * R], S + (int64_t)stream[s].col[l] * R,
                                            pol_keep);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        return true;
    };
    // every give-up decision is taken by the whole warp (the loop holds __syncwarp)
    bool ok = true;
    MeasAcc<R> macc;
    uint32_t mbound = 0;  // entries added to macc since its last flush (warp-uniform)
    if constexpr (MEAS) {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int b = 0; b < kMeasPlanes; ++b) macc.e[r][b] = 0ull;
    }
    int kmin_next[R];
    if (n_mine) {
        ok = __all_sync(0xFFFFFFFFu, mbar_wait_timed(&full[0], 0u, d.stage_wait_ns));
        if (ok) acceptance<R>(stream[0], warp, lane, t, kmin_next);
    }
    for (uint32_t j = 0; j < nc; ++j) {
        const uint32_t kb = s_kc[j], ke = s_kc[j + 1];
        if (j > 0) {
            ok = grid_barrier(d.gbar, j * gridDim.x, d.err, tid, ok);
            if (!ok) break;
        }
        for (uint32_t k = kb; ok && k < kb + L; ++k) ok = __all_sync(0xFFFFFFFFu, gathers(k, ke));
        for (uint32_t k = kb; ok && k < ke; ++k) {
            if (!__all_sync(0xFFFFFFFFu, gathers(k + L, ke))) {
                ok = false;
                break;
            }
            int kmin[R];
#pragma unroll
            for (int r = 0; r < R; ++r) kmin[r] = kmin_next[r];
            // the next group's random numbers and thresholds; inside the class its stage has
            // landed (k + 1 <= k + L), across a class boundary it is waited for here
            if (k + 1 < n_mine) {
                const uint32_t kn = k + 1;
                if (kn >= ke)
                    ok = __all_sync(0xFFFFFFFFu, mbar_wait_timed(&full[kn % NSS], (kn / NSS) & 1u,
                                                           d.stage_wait_ns));
                if (ok) acceptance<R>(stream[kn % NSS], warp, lane, t, kmin_next);
            }
            asm volatile("cp.async.wait_group %0;" ::"n"(L) : "memory");
            if (!ok) break;
            const int s = (int)(k % NSS), b = (int)(k % NG);
            const uint4 gi = stream[s].gi;
            if (warp < (gi.y & ~kWideGroup)) {
                if constexpr (MEAS) {
                    const uint32_t w = stream[s].meta[warp].w & 0xFFFFu;  // entries to later classes
                    if (mbound + w > kMeasMax) {
                        meas_flush<R>(macc, s_meas, lane);
                        mbound = 0;
                    }
                    mbound += w;
                }
                update_slice<R, MEAS>(d, stream[s], gath[b].v, gi, warp, lane, kmin, pol_keep, macc);
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[s]);
                mbar_arrive(&gfree[b]);
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!ok && lane == 0) atomicOr(d.err, 4);
    if constexpr (MEAS) {
        meas_flush<R>(macc, s_meas, lane);
        asm volatile("bar.sync 1, 256;" ::: "memory");  // the consumers' shared adds are done
        for (uint32_t i = tid; i < (uint32_t)R * 64u; i += 256u) {
            const unsigned long long v = s_meas[i];
            if (v)
                atomicAdd((unsigned long long*)(meas.e_dst + (int64_t)(i >> 6) * meas.stride_r +
                                                (int64_t)(i & 63u) * meas.stride_k),
                          v << 1);
        }
    }
    if (nc > 1) {
        // the last CTA past every barrier of this launch rearms the counters for the next one
        if (consumers_all(ok) && tid == 0) {
            if (atomicAdd(&d.gbar[1], 1u) == gridDim.x - 1) {
                atomicExch(&d.gbar[0], 0u);
                atomicExch(&d.gbar[1], 0u);
            }
        }
    }
}

// the kernels: plain sweeps, and the sweep after a measurement (its energy taken on the way;
// two CTAs per SM for R <= 2 as for the plain sweep, the registers capped to that)
template <int R, int NSS, int NG, int L>
__global__ void __launch_bounds__(32 * (kGroupSlices + 1))
    k_vb_packed_colour(VbPackedDev d, uint32_t c_begin, uint32_t c_end,
                       const uint32_t* __restrict__ clock, uint32_t t_off, VbSweepMeas meas) {
    colour_sweep<R, NSS, NG, L, false>(d, c_begin, c_end, clock, t_off, meas);
}

template <int R, int NSS, int NG, int L>
__global__ void __launch_bounds__(32 * (kGroupSlices + 1), R <= 2 ? 2 : 1)
    k_vb_packed_colour_meas(VbPackedDev d, uint32_t c_begin, uint32_t c_end,
                            const uint32_t* __restrict__ clock, uint32_t t_off, VbSweepMeas meas) {
    colour_sweep<R, NSS, NG, L, true>(d, c_begin, c_end, clock, t_off, meas);
}

template <int R, int NSS, int NG>
static constexpr size_t colour_smem() {
    return NSS * sizeof(VbStream<R>) + NG * sizeof(VbGath<R>) + (2 * NSS + NG) * sizeof(uint64_t);
}

static int g_num_sms = 0;

static int num_sms() {
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms;
}

// one launch per colour class (c_end = c_begin + 1), or one cooperative launch for the classes
// [c_begin, c_end) with every CTA resident
template <int R, int NSS, int NG, int L, bool MEAS>
static int colour_launch_v(const VbPackedDev& d, uint32_t c_begin, uint32_t c_end, uint32_t ng,
                           const uint32_t* clock, uint32_t t_off, const VbSweepMeas& meas,
                           int per_sm, cudaStream_t st) {
    constexpr size_t smem = colour_smem<R, NSS, NG>();
    static_assert(smem <= 227 * 1024, "pipeline shape exceeds the shared memory of one CTA");
    auto kern = [] {
        if constexpr (MEAS) return k_vb_packed_colour_meas<R, NSS, NG, L>;
        else return k_vb_packed_colour<R, NSS, NG, L>;
    }();
    static int resident = -1;
    if (resident < 0) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 32 * (kGroupSlices + 1), smem) !=
            cudaSuccess)
            n = 0;
        resident = n;
    }
    const int cps = per_sm < resident ? per_sm : resident;
    if (cps <= 0) return -1;
    const uint32_t cap = (uint32_t)num_sms() * (uint32_t)cps;
    if (c_end == c_begin + 1) {
        if (!ng) return 0;
        const uint32_t grid = ng < cap ? ng : cap;
        kern<<<grid, 32 * (kGroupSlices + 1), smem, st>>>(d, c_begin, c_end, clock, t_off, meas);
        return 1;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cap);
    cfg.blockDim = dim3(32 * (kGroupSlices + 1));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, d, c_begin, c_end, clock, t_off, meas) == cudaSuccess ? 1 : -1;
}

// pipeline shapes (the handle's autotuner picks one; none changes the results), as
// (stream stages, gather buffers, gather lookahead, CTAs per SM):
//   R = 1, 2: variant 0 (3, 3, 1, 2), variant 1 (4, 2, 1, 2), variant 2 (2, 2, 1, 3)
//   R = 4:    variant 0 (4, 2, 1, 1), variant 1 (2, 2, 1, 2), variant 2 (3, 3, 1, 1)
// With three gather buffers and gathers one group ahead, the buffer a warp fills for group
// k + 1 was last read for group k - 2, which every warp finished an iteration earlier: no warp
// waits for the slowest warp of the previous group before starting its gathers.
template <int R, bool MEAS>
static int colour_launch(const VbPackedDev& d, uint32_t c_begin, uint32_t c_end, uint32_t ng,
                         const uint32_t* clock, uint32_t t_off, int variant,
                         const VbSweepMeas& meas, cudaStream_t st) {
    if constexpr (R == 4) {
        if (variant == 0) return colour_launch_v<R, 4, 2, 1, MEAS>(d, c_begin, c_end, ng, clock, t_off, meas, 1, st);
        if (variant == 1) return colour_launch_v<R, 2, 2, 1, MEAS>(d, c_begin, c_end, ng, clock, t_off, meas, 2, st);
        return colour_launch_v<R, 3, 3, 1, MEAS>(d, c_begin, c_end, ng, clock, t_off, meas, 1, st);
    } else {
        if (variant == 0) return colour_launch_v<R, 3, 3, 1, MEAS>(d, c_begin, c_end, ng, clock, t_off, meas, 2, st);
        if (variant == 1) return colour_launch_v<R, 4, 2, 1, MEAS>(d, c_begin, c_end, ng, clock, t_off, meas, 2, st);
        return colour_launch_v<R, 2, 2, 1, MEAS>(d, c_begin, c_end, ng, clock, t_off, meas, 3, st);
    }
}

// One sweep (fused: one cooperative launch over all colour classes; else one launch per class).
// The fused form needs coherent gathers across classes inside a launch, which the 16-byte
// L2-only copies give for R = 2 and 4; R = 1 (8-byte copies through L1) uses one launch per class.
template <bool MEAS>
static int packed_sweep(const VbPackedDev& d, const uint32_t* colour_groups, const uint32_t* clock,
                        uint32_t t_off, int variant, bool fused, const VbSweepMeas& meas,
                        cudaStream_t st) {
    const uint32_t nc = (uint32_t)d.n_colours;
    if (!nc) return 0;
    if (fused && nc > 1 && d.R != 1) {
        int r = -1;
        if (d.R == 2) r = colour_launch<2, MEAS>(d, 0, nc, 0, clock, t_off, variant, meas, st);
        else if (d.R == 4) r = colour_launch<4, MEAS>(d, 0, nc, 0, clock, t_off, variant, meas, st);
        return r;
    }
    int n = 0;
    for (uint32_t c = 0; c < nc; ++c) {
        const uint32_t ng = colour_groups[c + 1] - colour_groups[c];
        int r = -1;
        switch (d.R) {
            case 1: r = colour_launch<1, MEAS>(d, c, c + 1, ng, clock, t_off, variant, meas, st); break;
            case 2: r = colour_launch<2, MEAS>(d, c, c + 1, ng, clock, t_off, variant, meas, st); break;
            case 4: r = colour_launch<4, MEAS>(d, c, c + 1, ng, clock, t_off, variant, meas, st); break;
            default: return -1;
        }
        if (r < 0) return -1;
        n += r;
    }
    return n;
}

}  // namespace sg
