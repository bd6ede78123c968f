// vb_kernels.cu -- Viana-Bray Metropolis kernels for sm_103a (the colour-class sweep itself is
// in vb_colour.cuh).
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
#include "vb_colour.cuh"

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

int vb_packed_sweep(const VbPackedDev& d, const uint32_t* colour_groups, const uint32_t* clock,
                    uint32_t t_off, int variant, bool fused, cudaStream_t st) {
    return packed_sweep<false>(d, colour_groups, clock, t_off, variant, fused, VbSweepMeas{}, st);
}

// ---------------------------------------------------------------------------------------------
// upper entries: one thread per slot keeps, in order, the entries whose neighbour lies in a
// later colour class (a higher slot), and pads the rest of its upper width with itself
// ---------------------------------------------------------------------------------------------
__global__ void k_vb_build_upper(VbPackedDev d) {
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= d.n_slots) return;
    const int64_t s = slot >> 5;
    const uint32_t l = (uint32_t)(slot & 31);
    const uint32_t base = d.slice_base[s], width = (d.slice_base[s + 1] - base) >> 5;
    const uint32_t ub = d.up_slice_base[s], uw = (d.up_slice_base[s + 1] - ub) >> 5;
    uint32_t* up_col = const_cast<uint32_t*>(d.up_col);
    uint64_t* up_jb = const_cast<uint64_t*>(d.up_jb);
    uint32_t e2 = 0;
    for (uint32_t e = 0; e < width; ++e) {
        const uint32_t idx = base + 32 * e + l;
        const uint32_t c = d.col[idx];
        if ((int64_t)c > slot && e2 < uw) {
            up_col[ub + 32 * e2 + l] = c;
            up_jb[ub + 32 * e2 + l] = d.jb[idx];
            ++e2;
        }
    }
    for (; e2 < uw; ++e2) {
        up_col[ub + 32 * e2 + l] = (uint32_t)slot;
        up_jb[ub + 32 * e2 + l] = 0ull;
    }
}

int vb_packed_build_upper(const VbPackedDev& d, cudaStream_t st) {
    if (!d.up_slice_base || d.n_slots == 0) return 0;
    const int bs = 256;
    k_vb_build_upper<<<(unsigned)((d.n_slots + bs - 1) / bs), bs, 0, st>>>(d);
    return 1;
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
    k_vb_packed_count(VbPackedDev d, VbCountJob job, VbCountJob qjob) {
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
    const int main_passes = job.kind == 3 ? job.w : 1;
    const int passes = main_passes + (!EN && qjob.kind == 1 ? 1 : 0);
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
        if (pass >= main_passes) {
            jb = qjob;
        } else if (job.kind == 3) {
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
int vb_packed_count(const VbPackedDev& d, const VbCountJob& job_in, cudaStream_t st,
                    const VbCountJob* also_q) {
    VbCountJob job = job_in;
    VbCountJob qjob{};
    qjob.kind = -1;
    if (also_q && job.kind != 2 && job.kind != 1 && also_q->kind == 1) qjob = *also_q;
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
            if (en) k_vb_packed_count<1, true><<<nb, bs, 0, st>>>(dd, job, qjob);
            else k_vb_packed_count<1, false><<<nb, bs, 0, st>>>(dd, job, qjob);
            break;
        case 2:
            if (en) k_vb_packed_count<2, true><<<nb, bs, 0, st>>>(dd, job, qjob);
            else k_vb_packed_count<2, false><<<nb, bs, 0, st>>>(dd, job, qjob);
            break;
        case 4:
            if (en) k_vb_packed_count<4, true><<<nb, bs, 0, st>>>(dd, job, qjob);
            else k_vb_packed_count<4, false><<<nb, bs, 0, st>>>(dd, job, qjob);
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
