// vb_kernels.cu -- Viana-Bray Metropolis kernels for sm_103a.
//
// Model (Eq. 3): H = -sum_{(ij) in E} J_ij s_i s_j, J_ij = +-1.  Flipping s_i changes the
// energy by dE = 2m with m = s_i sum_j J_ij s_j = d_i - 2u_i, u_i the number of unsatisfied
// edges at i (J_ij s_i s_j = -1).  Metropolis (Methods): flip iff m <= 0 or r32 < thr[m].
// A sweep updates one colour class (an independent set) at a time, the generalisation of the
// bipartite half-updates of SI section 3.
//
// Packed kernel (multispin coding, SI section 2): bit k of a uint64 spin word is lane k (an
// independent disorder sample); one thread updates one vertex for all 64 lanes and all R
// replicas.  Per neighbour, x = S_i ^ S_j ^ J marks the unsatisfied lanes; the x words are
// summed into a bit-sliced count (an unrolled carry-save adder tree for slices of width <= 8,
// a ripple counter of up to 6 planes, degree <= 63, otherwise).  Because thr[m] is
// non-increasing in m and the random number is shared by the 64 lanes, the accepted set
// {m <= m*} is a prefix: with m* = #{m in 1..d : r32 < thr[m]}, a lane flips iff d - 2u <= m*,
// i.e. u >= ceil((d - m*)/2): one bit-sliced compare against a per-thread constant.
#include "sg_internal.cuh"

namespace sg {

// ---------------------------------------------------------------------------------------------
// packed: initial spins (quench from a random configuration)
// ---------------------------------------------------------------------------------------------
__global__ void k_vb_packed_init(VbPackedDev d) {
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= d.n_slots) return;
    const uint32_t vi = d.vinfo[slot];
    const int R = d.R;
    if (vi == kInactive) {
        for (int r = 0; r < R; ++r) d.S[slot * R + r] = 0ull;
        return;
    }
    const uint32_t g = d.slice_graph[slot >> 5];
    const uint64_t seed = d.seeds[g];
    const uint32_t orig = vi & kOrigMask;
    for (int r = 0; r < R; ++r) {
        const uint4 w = philox4x32_10(make_uint4(orig, 0u, (uint32_t)r, 1u), (uint32_t)seed,
                                      (uint32_t)(seed >> 32));
        d.S[slot * R + r] = (uint64_t)w.x | ((uint64_t)w.y << 32);
    }
}

int vb_packed_init(const VbPackedDev& d, cudaStream_t st) {
    const int bs = 256;
    const int64_t nb = (d.n_slots + bs - 1) / bs;
    k_vb_packed_init<<<(unsigned)nb, bs, 0, st>>>(d);
    return 1;
}

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

// Count the unsatisfied edges of one vertex (all lanes, all replicas) with a P-plane counter
// and flip the lanes whose count reaches kmin.  Neighbour words come from the gather buffer, or
// straight from global memory for a wide slice (J == nullptr).
template <int R, int P>
__device__ __forceinline__ void count_and_flip(SpinWords<R>& si, const uint64_t* J,
                                               const uint64_t* gath, uint32_t loc, uint32_t width,
                                               const VbPackedDev& d, uint32_t idx,
                                               const int (&kmin)[R]) {
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

template <int R, int W>
__device__ __forceinline__ void count_and_flip_narrow(SpinWords<R>& si, const uint64_t* J,
                                                      const uint64_t* gath, uint32_t loc,
                                                      const int (&kmin)[R]) {
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
template <int R>
__device__ __forceinline__ void update_slice(const VbPackedDev& d, const VbStream<R>& st,
                                             const uint64_t* gath, const uint4& gi, uint32_t warp,
                                             uint32_t lane, const int (&kmin)[R],
                                             uint64_t pol_keep) {
    const bool wide = (gi.y & kWideGroup) != 0u;
    const uint32_t slice = gi.x + warp;
    const uint32_t vi = st.vinfo[warp * 32 + lane];
    if (vi == kInactive) return;
    const uint4 m = st.meta[warp];  // first entry, width
    const uint32_t width = m.y;
    SpinWords<R> si;
#pragma unroll
    for (int r = 0; r < R; ++r) si.v[r] = st.S[(warp * 32 + lane) * R + r];
    const uint64_t* J = wide ? nullptr : st.J;
    const uint32_t loc = m.x - gi.z + lane, idx = m.x + lane;
    // the slice's width (warp-uniform) selects the code: unrolled carry-save counting for the
    // common narrow slices of a staged group, a ripple counter sized by the width otherwise
    if (J && width <= 8) {
        switch (width) {
            case 0:  // isolated vertices: dE = 0, every lane flips (kmin = 0)
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (kmin[r] == 0) si.v[r] = ~si.v[r];
                break;
            case 1: count_and_flip_narrow<R, 1>(si, J, gath, loc, kmin); break;
            case 2: count_and_flip_narrow<R, 2>(si, J, gath, loc, kmin); break;
            case 3: count_and_flip_narrow<R, 3>(si, J, gath, loc, kmin); break;
            case 4: count_and_flip_narrow<R, 4>(si, J, gath, loc, kmin); break;
            case 5: count_and_flip_narrow<R, 5>(si, J, gath, loc, kmin); break;
            case 6: count_and_flip_narrow<R, 6>(si, J, gath, loc, kmin); break;
            case 7: count_and_flip_narrow<R, 7>(si, J, gath, loc, kmin); break;
            default: count_and_flip_narrow<R, 8>(si, J, gath, loc, kmin); break;
        }
    } else if (width <= 1) count_and_flip<R, 1>(si, J, gath, loc, width, d, idx, kmin);
    else if (width <= 3) count_and_flip<R, 2>(si, J, gath, loc, width, d, idx, kmin);
    else if (width <= 7) count_and_flip<R, 3>(si, J, gath, loc, width, d, idx, kmin);
    else if (width <= 15) count_and_flip<R, 4>(si, J, gath, loc, width, d, idx, kmin);
    else if (width <= 31) count_and_flip<R, 5>(si, J, gath, loc, width, d, idx, kmin);
    else count_and_flip<R, 6>(si, J, gath, loc, width, d, idx, kmin);
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
template <int R, int NSS, int NG, int L>
__global__ void __launch_bounds__(32 * (kGroupSlices + 1))
    k_vb_packed_colour(VbPackedDev d, uint32_t c_begin, uint32_t c_end,
                       const uint32_t* __restrict__ clock, uint32_t t_off) {
    static_assert(L >= 1 && L < NG && L < NSS, "gathers run L groups ahead inside both rings");
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ uint32_t s_kc[kVbMaxColours + 1];  // first ring index of each class (this CTA)
    __shared__ uint32_t s_cg[kVbMaxColours];      // first group of each class
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
            if (warp < (gi.y & ~kWideGroup))
                update_slice<R>(d, stream[s], gath[b].v, gi, warp, lane, kmin, pol_keep);
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[s]);
                mbar_arrive(&gfree[b]);
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!ok && lane == 0) atomicOr(d.err, 4);
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
template <int R, int NSS, int NG, int L>
static int colour_launch_v(const VbPackedDev& d, uint32_t c_begin, uint32_t c_end, uint32_t ng,
                           const uint32_t* clock, uint32_t t_off, int per_sm, cudaStream_t st) {
    constexpr size_t smem = colour_smem<R, NSS, NG>();
    static_assert(smem <= 227 * 1024, "pipeline shape exceeds the shared memory of one CTA");
    auto kern = k_vb_packed_colour<R, NSS, NG, L>;
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
        kern<<<grid, 32 * (kGroupSlices + 1), smem, st>>>(d, c_begin, c_end, clock, t_off);
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
    return cudaLaunchKernelEx(&cfg, kern, d, c_begin, c_end, clock, t_off) == cudaSuccess ? 1 : -1;
}

// pipeline shapes (the handle's autotuner picks one; none changes the results), as
// (stream stages, gather buffers, gather lookahead, CTAs per SM):
//   R = 1, 2: variant 0 (3, 3, 1, 2), variant 1 (4, 2, 1, 2), variant 2 (2, 2, 1, 3)
//   R = 4:    variant 0 (4, 2, 1, 1), variant 1 (2, 2, 1, 2), variant 2 (3, 3, 1, 1)
// With three gather buffers and gathers one group ahead, the buffer a warp fills for group
// k + 1 was last read for group k - 2, which every warp finished an iteration earlier: no warp
// waits for the slowest warp of the previous group before starting its gathers.
template <int R>
static int colour_launch(const VbPackedDev& d, uint32_t c_begin, uint32_t c_end, uint32_t ng,
                         const uint32_t* clock, uint32_t t_off, int variant, cudaStream_t st) {
    if constexpr (R == 4) {
        if (variant == 0) return colour_launch_v<R, 4, 2, 1>(d, c_begin, c_end, ng, clock, t_off, 1, st);
        if (variant == 1) return colour_launch_v<R, 2, 2, 1>(d, c_begin, c_end, ng, clock, t_off, 2, st);
        return colour_launch_v<R, 3, 3, 1>(d, c_begin, c_end, ng, clock, t_off, 1, st);
    } else {
        if (variant == 0) return colour_launch_v<R, 3, 3, 1>(d, c_begin, c_end, ng, clock, t_off, 2, st);
        if (variant == 1) return colour_launch_v<R, 4, 2, 1>(d, c_begin, c_end, ng, clock, t_off, 2, st);
        return colour_launch_v<R, 2, 2, 1>(d, c_begin, c_end, ng, clock, t_off, 3, st);
    }
}

// One sweep (fused: one cooperative launch over all colour classes; else one launch per class).
// The fused form needs coherent gathers across classes inside a launch, which the 16-byte
// L2-only copies give for R = 2 and 4; R = 1 (8-byte copies through L1) uses one launch per class.
int vb_packed_sweep(const VbPackedDev& d, const uint32_t* colour_groups, const uint32_t* clock,
                    uint32_t t_off, int variant, bool fused, cudaStream_t st) {
    const uint32_t nc = (uint32_t)d.n_colours;
    if (!nc) return 0;
    if (fused && nc > 1 && d.R != 1) {
        int r = -1;
        if (d.R == 2) r = colour_launch<2>(d, 0, nc, 0, clock, t_off, variant, st);
        else if (d.R == 4) r = colour_launch<4>(d, 0, nc, 0, clock, t_off, variant, st);
        return r;
    }
    int n = 0;
    for (uint32_t c = 0; c < nc; ++c) {
        const uint32_t ng = colour_groups[c + 1] - colour_groups[c];
        int r = -1;
        switch (d.R) {
            case 1: r = colour_launch<1>(d, c, c + 1, ng, clock, t_off, variant, st); break;
            case 2: r = colour_launch<2>(d, c, c + 1, ng, clock, t_off, variant, st); break;
            case 4: r = colour_launch<4>(d, c, c + 1, ng, clock, t_off, variant, st); break;
            default: return -1;
        }
        if (r < 0) return -1;
        n += r;
    }
    return n;
}


// ---------------------------------------------------------------------------------------------
// snapshot copy (16-byte vectors; the regions are 256-byte aligned and a multiple of 16 bytes)
// ---------------------------------------------------------------------------------------------
__global__ void k_copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t n16) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

static int copy_bytes(const void* src, void* dst, int64_t bytes, cudaStream_t st) {
    const int64_t n16 = bytes / 16;
    const int bs = 256;
    int64_t nb = (n16 + bs - 1) / bs;
    if (nb > 152 * 16) nb = 152 * 16;
    if (nb < 1) nb = 1;
    k_copy16<<<(unsigned)nb, bs, 0, st>>>((const uint4*)src, (uint4*)dst, n16);
    return 1;
}

int vb_packed_snapshot(const VbPackedDev& d, int w, cudaStream_t st) {
    const int64_t words = d.n_slots * d.R;
    return copy_bytes(d.S, d.snap + (int64_t)w * words, words * 8, st);
}

// ---------------------------------------------------------------------------------------------
// packed: per-lane difference counts (C, q, E).  Each warp walks a contiguous run of slices,
// accumulates bit-sliced per-lane counters (16 planes) and flushes them to global memory when
// the graph changes and at the end of its run.
// ---------------------------------------------------------------------------------------------
// A lane adds at most one word per slot (C, q: 16 slices, so 5 planes hold up to 31) or one per
// entry (E: 16 slices x width <= 63 = 1008 words: 10 planes, up to 1023), so PL planes cannot
// overflow before the flush at the end of a run; the 32-lane butterfly needs PL + 5 planes.
constexpr int kCountSlicesPerWarp = 16;

template <int NQ, int PW>
__device__ __forceinline__ void count_add(uint64_t (&p)[NQ][PW], int q, uint64_t x) {
#pragma unroll
    for (int b = 0; b < PW - 5; ++b) {
        const uint64_t c = p[q][b] & x;
        p[q][b] ^= x;
        x = c;
    }
}

// Sum the bit-sliced counters of the 32 lanes with a butterfly of bit-sliced additions, then
// lane l adds the totals of spin lanes l and l + 32.  With a CTA-shared accumulator (cta_acc,
// [NQ][64], one graph per CTA run) the warp adds there and the CTA flushes once; otherwise
// straight into global memory.
template <int NQ, int PW>
__device__ __forceinline__ void count_flush(uint64_t (&p)[NQ][PW], const VbCountJob& job,
                                            uint32_t g, int nq, uint32_t lane,
                                            unsigned long long* cta_acc = nullptr) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (q >= nq) break;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            uint64_t carry = 0ull;
#pragma unroll
            for (int b = 0; b < PW; ++b) {
                const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, p[q][b], off);
                const uint64_t x = p[q][b] ^ o;
                const uint64_t sum = x ^ carry;
                carry = (p[q][b] & o) | (carry & x);
                p[q][b] = sum;
            }
        }
        uint32_t c0 = 0, c1 = 0;
#pragma unroll
        for (int b = 0; b < PW; ++b) {
            c0 |= (uint32_t)((p[q][b] >> lane) & 1ull) << b;
            c1 |= (uint32_t)((p[q][b] >> (lane + 32)) & 1ull) << b;
        }
        if (cta_acc) {
            if (c0) atomicAdd(cta_acc + q * 64 + lane, (unsigned long long)c0);
            if (c1) atomicAdd(cta_acc + q * 64 + lane + 32, (unsigned long long)c1);
        } else {
            int64_t* base = job.dst + g * job.stride_g + q * job.stride_r;
            if (c0)
                atomicAdd((unsigned long long*)(base + lane * job.stride_k),
                          (unsigned long long)c0 << job.shift);
            if (c1)
                atomicAdd((unsigned long long*)(base + (lane + 32) * job.stride_k),
                          (unsigned long long)c1 << job.shift);
        }
#pragma unroll
        for (int b = 0; b < PW; ++b) p[q][b] = 0ull;
    }
}

// EN: the energy job (kind 2, PW = 15); otherwise C and q jobs (kinds 0, 1, 3, PW = 10)
template <int R, bool EN>
__global__ void __launch_bounds__(256, EN ? (R <= 2 ? 2 : 1) : (R <= 2 ? 3 : 2))
    k_vb_packed_count(VbPackedDev d, VbCountJob job) {
    constexpr int NQ = R;
    constexpr int PW = EN ? 15 : 10;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t s_lo = (int64_t)warp * kCountSlicesPerWarp;
    int64_t s_hi = s_lo + kCountSlicesPerWarp;
    if (s_hi > d.n_slices) s_hi = d.n_slices;
    const int64_t words = d.n_slots * R;
    // kind 3: one pass per snapshot over this warp's slices; the current spins of the slices
    // (a few KB) stay in L1 after the first pass
    const int passes = job.kind == 3 ? job.w : 1;
    // The CTA's slices belong to one graph (the common case: a single instance, or slices of
    // one graph in a batch): the warps add into a shared accumulator and the CTA flushes it once,
    // so the global counters see one atomic per CTA instead of one per warp.
    __shared__ unsigned long long acc[NQ * 64];
    __shared__ int one_graph;
    const int64_t cta_lo = (int64_t)blockIdx.x * (blockDim.x / 32) * kCountSlicesPerWarp;
    int64_t cta_hi = cta_lo + (int64_t)(blockDim.x / 32) * kCountSlicesPerWarp;
    if (cta_hi > d.n_slices) cta_hi = d.n_slices;
    if (threadIdx.x == 0)
        one_graph = cta_lo < cta_hi && __ldg(d.slice_graph + cta_lo) == __ldg(d.slice_graph + cta_hi - 1);
    for (int pass = 0; pass < passes; ++pass) {
        VbCountJob jb = job;
        if (job.kind == 3) {
            jb.kind = 0;
            jb.w = pass;
            jb.dst = job.dst + pass * job.stride_w;
        }
        const int kind = jb.kind;
        const int nq = kind == 1 ? R / 2 : R;
        uint64_t p[NQ][PW];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int b = 0; b < PW; ++b) p[q][b] = 0ull;
        const uint64_t* snap = d.snap + (int64_t)(kind == 0 ? jb.w : 0) * words;
        int64_t cur_g = -1;
        for (int q = threadIdx.x; q < NQ * 64; q += blockDim.x) acc[q] = 0ull;
        __syncthreads();
        unsigned long long* cta_acc = one_graph ? acc : nullptr;
        if (cta_acc && s_lo < s_hi) {
            // every slice of the CTA belongs to one graph: no per-slice graph test, so nothing
            // but the loads and the counting sits in the loop and the loads of several slices
            // (or entries) can be in flight together
            cur_g = __ldg(d.slice_graph + s_lo);
            if constexpr (!EN) {
#pragma unroll 4
                for (int64_t s = s_lo; s < s_hi; ++s) {
                    const int64_t slot = s * 32 + lane;
                    const SpinWords<R> si = load_words<R>(d.S + slot * R);
                    if (kind == 0) {
                        const SpinWords<R> sw = load_words<R>(snap + slot * R);
#pragma unroll
                        for (int r = 0; r < R; ++r) count_add<NQ, PW>(p, r, si.v[r] ^ sw.v[r]);
                    } else {
#pragma unroll
                        for (int q = 0; q < R / 2; ++q)
                            count_add<NQ, PW>(p, q, si.v[2 * q] ^ si.v[2 * q + 1]);
                    }
                }
            } else {
                uint32_t base = __ldg(d.slice_base + s_lo);
                for (int64_t s = s_lo; s < s_hi; ++s) {
                    const uint32_t next = __ldg(d.slice_base + s + 1);
                    const SpinWords<R> si = load_words<R>(d.S + (s * 32 + lane) * R);
                    const uint32_t width = (next - base) >> 5;
                    uint32_t idx = base + lane;
#pragma unroll 4
                    for (uint32_t e = 0; e < width; ++e, idx += 32) {
                        const uint32_t j = __ldg(d.col + idx);
                        const uint64_t J = __ldg(d.jb + idx);
                        const SpinWords<R> sj = gather_words<R>(d.S + (int64_t)j * R);
#pragma unroll
                        for (int r = 0; r < R; ++r) count_add<NQ, PW>(p, r, si.v[r] ^ sj.v[r] ^ J);
                    }
                    base = next;
                }
            }
        } else
        // padding slots hold zero words and zero couplings, so they add nothing: no vinfo test,
        // and the loads of several slices can be in flight together
#pragma unroll 4
        for (int64_t s = s_lo; s < s_hi; ++s) {
            const uint32_t g = __ldg(d.slice_graph + s);  // warp-uniform
            if ((int64_t)g != cur_g) {
                if (cur_g >= 0) count_flush<NQ, PW>(p, jb, (uint32_t)cur_g, nq, lane, cta_acc);
                cur_g = g;
            }
            const int64_t slot = s * 32 + lane;
            const SpinWords<R> si = load_words<R>(d.S + slot * R);
            if constexpr (!EN) {
                if (kind == 0) {
                    const SpinWords<R> sw = load_words<R>(snap + slot * R);
#pragma unroll
                    for (int r = 0; r < R; ++r) count_add<NQ, PW>(p, r, si.v[r] ^ sw.v[r]);
                } else {
#pragma unroll
                    for (int q = 0; q < R / 2; ++q)
                        count_add<NQ, PW>(p, q, si.v[2 * q] ^ si.v[2 * q + 1]);
                }
            } else {
                const uint32_t base = __ldg(d.slice_base + s);
                const uint32_t width = (__ldg(d.slice_base + s + 1) - base) >> 5;
                uint32_t idx = base + lane;
#pragma unroll 4
                for (uint32_t e = 0; e < width; ++e, idx += 32) {
                    const uint32_t j = __ldg(d.col + idx);
                    const uint64_t J = __ldg(d.jb + idx);
                    const SpinWords<R> sj = gather_words<R>(d.S + (int64_t)j * R);
#pragma unroll
                    for (int r = 0; r < R; ++r) count_add<NQ, PW>(p, r, si.v[r] ^ sj.v[r] ^ J);
                }
            }
        }
        if (cur_g >= 0) count_flush<NQ, PW>(p, jb, (uint32_t)cur_g, nq, lane, cta_acc);
        if (cta_acc) {
            __syncthreads();
            const int64_t g = (int64_t)__ldg(d.slice_graph + cta_lo);
            for (int q = threadIdx.x; q < nq * 64; q += blockDim.x) {
                const unsigned long long v = acc[q];
                if (v)
                    atomicAdd((unsigned long long*)(jb.dst + g * jb.stride_g + (q >> 6) * jb.stride_r +
                                                    (q & 63) * jb.stride_k),
                              v << jb.shift);
            }
            __syncthreads();
        }
    }
}

// The energy job (kind 2) runs over the upper entries when the layout has them: each edge once,
// from its lower-colour endpoint (the higher slot), counted twice (shift 1).
int vb_packed_count(const VbPackedDev& d, const VbCountJob& job_in, cudaStream_t st) {
    VbCountJob job = job_in;
    VbPackedDev dd = d;
    if (job.kind == 2 && d.up_slice_base) {
        dd.slice_base = d.up_slice_base;
        dd.col = d.up_col;
        dd.jb = d.up_jb;
        job.shift = 1;
    }
    const int bs = 256;
    const int64_t warps = (d.n_slices + kCountSlicesPerWarp - 1) / kCountSlicesPerWarp;
    const unsigned nb = (unsigned)((warps + (bs / 32) - 1) / (bs / 32));
    const bool en = job.kind == 2;
    switch (d.R) {
        case 1:
            if (en) k_vb_packed_count<1, true><<<nb, bs, 0, st>>>(dd, job);
            else k_vb_packed_count<1, false><<<nb, bs, 0, st>>>(dd, job);
            break;
        case 2:
            if (en) k_vb_packed_count<2, true><<<nb, bs, 0, st>>>(dd, job);
            else k_vb_packed_count<2, false><<<nb, bs, 0, st>>>(dd, job);
            break;
        case 4:
            if (en) k_vb_packed_count<4, true><<<nb, bs, 0, st>>>(dd, job);
            else k_vb_packed_count<4, false><<<nb, bs, 0, st>>>(dd, job);
            break;
        default: return -1;
    }
    return 1;
}

// ---------------------------------------------------------------------------------------------
// plain kernel: one thread per (vertex, lane, replica), int8 spins, CSR in colour-major labels
// ---------------------------------------------------------------------------------------------
__global__ void k_vb_plain_init(VbPlainDev d) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)d.N * d.R) return;
    const int32_t v = (int32_t)(idx % d.N);
    const int32_t r = (int32_t)(idx / d.N);
    const uint4 w = philox4x32_10(make_uint4(d.orig[v], 0u, (uint32_t)r, 1u), (uint32_t)d.seed,
                                  (uint32_t)(d.seed >> 32));
    const uint64_t bits = (uint64_t)w.x | ((uint64_t)w.y << 32);
    for (int k = 0; k < d.L; ++k)
        d.s[((int64_t)r * d.L + k) * d.N + v] = ((bits >> k) & 1ull) ? (int8_t)-1 : (int8_t)1;
}

int vb_plain_init(const VbPlainDev& d, cudaStream_t st) {
    const int bs = 256;
    const int64_t n = (int64_t)d.N * d.R;
    k_vb_plain_init<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(d);
    return 1;
}

__global__ void k_vb_plain_colour(VbPlainDev d, int32_t v0, int32_t nv, const uint32_t* clock,
                                  uint32_t t_off) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nv * d.R * d.L) return;
    const uint32_t t = *clock + t_off;
    const int32_t v = v0 + (int32_t)(idx % nv);
    const int32_t rk = (int32_t)(idx / nv);
    const int32_t r = rk / d.L, k = rk % d.L;
    const uint4 rnd = philox4x32_10(make_uint4(d.orig[v], t, (uint32_t)(r >> 2), 0u),
                                    (uint32_t)d.seed, (uint32_t)(d.seed >> 32));
    const uint32_t r32 = uint4_word(rnd, r & 3);
    int8_t* s = d.s + (int64_t)rk * d.N;
    int field = 0;
    for (int32_t e = d.row_ptr[v]; e < d.row_ptr[v + 1]; ++e) {
        const int J = ((d.jb[e] >> k) & 1ull) ? -1 : 1;
        field += J * s[d.col[e]];
    }
    const int m = s[v] * field;
    const bool flip = (m <= 0) || (r32 < d.thr[r * kVbThrStride + m]);
    if (flip) s[v] = (int8_t)(-s[v]);
}

int vb_plain_colour(const VbPlainDev& d, int32_t v_begin, int32_t v_end, const uint32_t* clock,
                    uint32_t t_off, cudaStream_t st) {
    const int32_t nv = v_end - v_begin;
    if (nv <= 0) return 0;
    const int bs = 256;
    const int64_t n = (int64_t)nv * d.R * d.L;
    k_vb_plain_colour<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(d, v_begin, nv, clock, t_off);
    return 1;
}

int vb_plain_snapshot(const VbPlainDev& d, int w, cudaStream_t st) {
    const int64_t bytes = (int64_t)d.R * d.L * d.N;
    // int8 snapshots are not 16-byte multiples in general: use a byte copy
    return cudaMemcpyAsync(d.snap + (int64_t)w * bytes, d.s, (size_t)bytes,
                           cudaMemcpyDeviceToDevice, st) == cudaSuccess ? 0 : -1;
}

// per-(replica or pair, lane) difference counts over the vertices; blockIdx.y = rq * L + k
__global__ void k_vb_plain_count(VbPlainDev d, VbCountJob job) {
    const int32_t rk = blockIdx.y;
    const int32_t rq = rk / d.L, k = rk % d.L;
    const int64_t plane = (int64_t)d.R * d.L * d.N;
    unsigned long long acc = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < d.N; v += gridDim.x * blockDim.x) {
        if (job.kind == 0) {
            const int64_t o = ((int64_t)rq * d.L + k) * d.N + v;
            acc += d.s[o] != d.snap[(int64_t)job.w * plane + o];
        } else if (job.kind == 1) {
            const int64_t a = ((int64_t)(2 * rq) * d.L + k) * d.N + v;
            const int64_t b = ((int64_t)(2 * rq + 1) * d.L + k) * d.N + v;
            acc += d.s[a] != d.s[b];
        } else {
            const int8_t* s = d.s + ((int64_t)rq * d.L + k) * d.N;
            for (int32_t e = d.row_ptr[v]; e < d.row_ptr[v + 1]; ++e) {
                const int J = ((d.jb[e] >> k) & 1ull) ? -1 : 1;
                acc += (J * s[v] * s[d.col[e]]) < 0;
            }
        }
    }
    // block reduction
    __shared__ unsigned long long red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ull;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
        if (threadIdx.x == 0 && acc)
            atomicAdd((unsigned long long*)(job.dst + rq * job.stride_r + k * job.stride_k), acc);
    }
}

int vb_plain_count(const VbPlainDev& d, const VbCountJob& job, cudaStream_t st) {
    const int nq = job.kind == 1 ? d.R / 2 : d.R;
    if (nq <= 0) return 0;
    const int bs = 256;
    int nb = (d.N + bs - 1) / bs;
    if (nb > 64) nb = 64;
    dim3 grid((unsigned)nb, (unsigned)(nq * d.L));
    k_vb_plain_count<<<grid, bs, 0, st>>>(d, job);
    return 1;
}

}  // namespace sg
