// sk_kernels.cu -- Sherrington-Kirkpatrick Metropolis kernels for sm_103a.
//
// Model (Eq. 1 with the binary couplings of SI section 1): H = -sum_{i<j} J_ij s_i s_j / sqrt(N),
// J_ij = +-1.  With the local field h_i = sum_j J_ij s_j, flipping s_i costs dE = 2k/sqrt(N),
// k = s_i h_i; Metropolis accepts iff k <= 0 or r32 < thr[k].  Spins are visited in the fixed
// order i = 0..N-1 (SI section 1).  Because thr[k] is non-increasing, the accepted set for one
// random number is a prefix {k <= K*}, K* = max{k : k = 0 or r32 < thr[k]}.
//
// Blocked sweep (exact reformulation of the sequential order): the spins are cut into blocks
// of B.  For block b:
//   1. in-block kernel: every replica (one warp each) first adds the previous block's flips to
//      the fields of its own rows (popcounts over the bit-packed couplings), then runs the B
//      sequential decisions of the block and records the changes D_j = (s_j' - s_j)/2 in
//      {-1, 0, +1}.  Inside a 32-spin chunk the warp finds the next flip with a ballot: lanes
//      past the last accepted flip evaluate their decision with the fields as they stand; the
//      lowest tentative flip is final, moves every later lane's k by +-2 (its coupling bit),
//      and the rest is re-evaluated.  The number of rounds is the number of flips in the chunk
//      plus one; after the chunk, popcounts update the fields of the block's later chunks.
//   2. field kernel: H[rows, R] += 2 J[rows, block] D[block, R] for every row but those of the
//      next block (which the next in-block kernel folds in itself), as a tcgen05 tensor-core
//      GEMM with e4m3 operands (J = +-1, 0 on the diagonal and in padding; D in {-1,0,1}: all
//      exact) and an FP32 accumulator in tensor memory that starts from zero for every block,
//      so partial sums stay below B in magnitude and are exact; the epilogue adds 2*acc to the
//      int32 fields.  It runs on a parallel branch and is needed only two blocks later.
//      Integer arithmetic makes the result identical to the sequential order.
#include <cuda.h>

#include <mutex>

#include "sg_internal.cuh"
#include "sk_internal.cuh"

namespace sg {

__device__ __forceinline__ uint8_t e4m3_of_sign(int v) {  // v in {-1, 0, 1}
    return v > 0 ? (uint8_t)0x38 : (v < 0 ? (uint8_t)0xB8 : (uint8_t)0x00);
}

// --------------------------------------------------------------------------------------------
// initial spins (quench) and D = s for the initial field computation
// --------------------------------------------------------------------------------------------
__global__ void k_sk_init(SkDev d) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over R * Np
    const int64_t total = (int64_t)d.R * d.Np;
    if (idx >= total) return;  // total is a multiple of 32: whole warps exit together
    const int r = (int)(idx / d.Np);
    const int i = (int)(idx % d.Np);
    int s = 1;
    if (i < d.N) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)i, 0u, (uint32_t)r, 1u),
                                      (uint32_t)d.seed, (uint32_t)(d.seed >> 32));
        s = (w.x & 1u) ? -1 : 1;
    }
    d.D[(int64_t)r * d.Np + i] = i < d.N ? e4m3_of_sign(s) : (uint8_t)0;
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, s < 0);
    if ((threadIdx.x & 31) == 0) d.S[(int64_t)r * (d.Np / 32) + i / 32] = bits;
}

int sk_init(const SkDev& d, cudaStream_t st) {
    const int64_t total = (int64_t)d.R * d.Np;
    k_sk_init<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(d);
    return 1;
}

// --------------------------------------------------------------------------------------------
// K* of every (replica, spin) for one sweep: depends only on the random numbers and the tables,
// so it is computed for the whole sweep at once, off the sequential chain.
// --------------------------------------------------------------------------------------------
// dst: even[] for an even sweep index t, odd[] for an odd one (the same array for the
// launch-per-block sequence; the persistent sweep double-buffers)
__global__ void k_sk_kstar(SkDev d, const uint32_t* __restrict__ clock, uint32_t t_off,
                           int32_t* even, int32_t* odd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over R * Np
    if (idx >= (int64_t)d.R * d.Np) return;
    const int r = (int)(idx / d.Np);
    const int i = (int)(idx % d.Np);
    const uint32_t t = __ldg(clock) + t_off;
    int k = -0x7FFFFFFF;  // padding never flips
    if (i < d.N) {
        const uint4 rnd = philox4x32_10(make_uint4((uint32_t)i, t, (uint32_t)(r >> 2), 0u),
                                        (uint32_t)d.seed, (uint32_t)(d.seed >> 32));
        k = sk_kstar(uint4_word(rnd, r & 3), d.thr + (int64_t)d.temp_index[r] * d.N, d.N,
                     d.coef[r]);
    }
    ((t & 1u) ? odd : even)[idx] = k;
}

int sk_kstar_sweep_into(const SkDev& d, const uint32_t* clock, uint32_t t_off, int32_t* even,
                        int32_t* odd, cudaStream_t st) {
    const int64_t total = (int64_t)d.R * d.Np;
    k_sk_kstar<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(d, clock, t_off, even, odd);
    return 1;
}

int sk_kstar_sweep(const SkDev& d, const uint32_t* clock, uint32_t t_off, cudaStream_t st) {
    return sk_kstar_sweep_into(d, clock, t_off, d.kst, d.kst, st);
}

// K* of n consecutive sweeps as int16 (|K*| < N <= 32768; padding gets -32768, which no k
// reaches): one thread per (sweep, replica group of 4, spin), one Philox block per thread for
// the group's four replicas.  dst[(s R + r) Np + i].
__global__ void k_sk_kstar16(SkDev d, const uint32_t* __restrict__ clock, uint32_t t_off, int n,
                             int16_t* __restrict__ dst) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int groups = d.R / 4;
    const int64_t per_sweep = (int64_t)groups * d.Np;
    if (idx >= per_sweep * n) return;
    const int s = (int)(idx / per_sweep);
    const int64_t rem = idx - (int64_t)s * per_sweep;
    const int g = (int)(rem / d.Np);
    const int i = (int)(rem - (int64_t)g * d.Np);
    int16_t* out = dst + ((int64_t)s * d.R + 4 * g) * d.Np + i;
    if (i >= d.N) {
#pragma unroll
        for (int w = 0; w < 4; ++w) out[(int64_t)w * d.Np] = (int16_t)-32768;
        return;
    }
    const uint32_t t = __ldg(clock) + t_off + (uint32_t)s;
    const uint4 rnd = philox4x32_10(make_uint4((uint32_t)i, t, (uint32_t)g, 0u), (uint32_t)d.seed,
                                    (uint32_t)(d.seed >> 32));
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int r = 4 * g + w;
        out[(int64_t)w * d.Np] = (int16_t)sk_kstar(uint4_word(rnd, w),
                                                   d.thr + (int64_t)__ldg(d.temp_index + r) * d.N,
                                                   d.N, __ldg(d.coef + r));
    }
}

int sk_kstar16_sweeps(const SkDev& d, const uint32_t* clock, uint32_t t_off, int n, int16_t* dst,
                      cudaStream_t st) {
    const int64_t total = (int64_t)(d.R / 4) * d.Np * n;
    k_sk_kstar16<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(d, clock, t_off, n, dst);
    return 1;
}

// --------------------------------------------------------------------------------------------
// in-block sequential update, one warp per replica.  The CTA stages the couplings of the
// block's rows with the block's own columns (and, when prev_b0 >= 0, with the previous block's
// columns) in shared memory; its replicas (2, 4 or 8 warps) share them.  The couplings are
// stored column-word major (JbT[w][i] = word w of row i), so the block's rows of one column
// word are one contiguous run: a single thread stages them with one bulk copy per word, and in
// shared memory ([word][row]) the 32 lanes of a warp (32 consecutive rows) read 32 consecutive
// words, one per bank.
// When prev_b0 >= 0 the kernel first adds the previous block's flips to the fields of its own
// rows (popcounts over bit-packed couplings, written back to H): that update is on the
// sequential critical path, while the tensor-core update of every other row runs elsewhere.
// --------------------------------------------------------------------------------------------
// 2 s: the coupling copies of a launch are late only if something broke
constexpr uint64_t kSkStageWaitNs = 2000000000ull;

template <int NC>
__global__ void __launch_bounds__(256) k_sk_inblock(SkDev d, int b0, int prev_b0) {
    static_assert(NC == 2 || NC == 4 || NC == 8 || NC == 16, "B = 64, 128, 256 or 512");
    // [2 * NC words][B rows]: own column words 0..NC-1, then the previous block's
    extern __shared__ __align__(128) uint32_t jblk[];
    __shared__ __align__(8) uint64_t jbar;
    constexpr int B = 32 * NC;
    const int lane = threadIdx.x & 31;
    const int words = d.Np / 32;
    const int wb = b0 / 32;
    const int pwb = prev_b0 >= 0 ? prev_b0 / 32 : 0;
    const int nw = prev_b0 >= 0 ? 2 * NC : NC;  // column words staged
    // A programmatic launch after the previous block's in-block kernel: let the next block's
    // kernel start its own prologue now (it reads nothing of ours before its dependency wait).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const bool active = r < d.R;
    // Prologue on data no in-block kernel writes (couplings, the sweep's K* table): may run
    // while the previous block is still being updated.
    if (threadIdx.x == 0) {
        mbar_init(&jbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_tx(&jbar, (uint32_t)(nw * B * 4));
        for (int w = 0; w < nw; ++w) {
            const int cw = w < NC ? wb + w : pwb + (w - NC);
            bulk_copy_g2s(jblk + w * B, d.JbT + (int64_t)cw * d.Np + b0, B * 4, &jbar);
        }
    }
    int kst[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) kst[c] = active ? d.kst[(int64_t)r * d.Np + b0 + 32 * c + lane] : 0;
    // Everything below depends on the previous block (spins, flips, fields): wait until that
    // kernel has completed and its writes are visible (immediate for a plain launch).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int h[NC];
    uint32_t sw[NC], pF[NC], psn[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int i = b0 + 32 * c + lane;
        h[c] = active ? d.H[(int64_t)r * d.Np + i] : 0;
        sw[c] = active ? d.S[(int64_t)r * words + wb + c] : 0u;
        const bool pv = active && prev_b0 >= 0;
        pF[c] = pv ? d.flips[(int64_t)r * words + pwb + c] : 0u;
        psn[c] = pv ? d.S[(int64_t)r * words + pwb + c] : 0u;
    }
    __syncthreads();  // the barrier's initialisation is visible to every thread
    if (!mbar_wait_timed(&jbar, 0u, d.test_nowait ? 0ull : kSkStageWaitNs)) {
        // no thread leaves while a copy may still be landing in shared memory
        mbar_wait_timed(&jbar, 0u, kSkStageWaitNs);
        atomicOr(d.err, 4);
        return;
    }
    if (!active) return;
    if (prev_b0 >= 0) {
        // fields += 2 sum_{j flipped in the previous block} J_ij s_j'
        int dh[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) dh[c] = 0;
#pragma unroll
        for (int cp = 0; cp < NC; ++cp) {
            const uint32_t F = pF[cp];
            if (!F) continue;
            const uint32_t sn = psn[cp];
            const int pf = __popc(F);
#pragma unroll
            for (int c = 0; c < NC; ++c)
                dh[c] += 2 * (pf - 2 * __popc(F & (jblk[(NC + cp) * B + 32 * c + lane] ^ sn)));
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (dh[c]) d.H[(int64_t)r * d.Np + b0 + 32 * c + lane] = h[c] + dh[c];
            h[c] += dh[c];
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int i = b0 + 32 * c + lane;
        const uint32_t sbit = (sw[c] >> lane) & 1u;
        const int x = sbit ? -h[c] : h[c];
        const uint32_t neg = jblk[c * B + 32 * c + lane] ^ sw[c] ^ (sbit ? 0xFFFFFFFFu : 0u);
        // Resolve the chunk's 32 sequential decisions: every lane past the last accepted flip
        // decides with the fields as they stand; the lowest lane that flips is accepted (the
        // lanes below it keep their decision), its flip moves every later lane's k by +2 or -2 (by
        // that lane's coupling bit), and the rest is decided again.  Only ALU work and a ballot per accepted flip.
        uint32_t F = 0, last = 0;  // accepted flips; lowest-bit mask of the last one (0: none)
        const uint32_t lane_bit = 1u << lane;
        int cur = x;
        for (;;) {
            const bool tent = lane_bit > last && cur <= kst[c];
            const uint32_t bm = __ballot_sync(0xFFFFFFFFu, tent);
            if (bm == 0u) break;
            last = bm & (0u - bm);
            F |= last;
            cur += (neg & last) ? 2 : -2;
        }
        const uint32_t nsw = sw[c] ^ F;
        // changes D_i = (s' - s)/2 for the field GEMM: -s_old where flipped
        const int dval = ((F >> lane) & 1u) ? (sbit ? 1 : -1) : 0;
        d.D[(int64_t)r * d.Np + i] = e4m3_of_sign(dval);
        if (lane == 0) {
            d.S[(int64_t)r * words + wb + c] = nsw;
            d.flips[(int64_t)r * words + wb + c] = F;
        }
        // fields of the later rows of this block: h += 2 sum_{j in F} J_ij s_j'
        if (F) {
            const int pf = __popc(F);
#pragma unroll
            for (int c2 = c + 1; c2 < NC; ++c2) {
                const uint32_t m = jblk[c * B + 32 * c2 + lane] ^ nsw;
                h[c2] += 2 * (pf - 2 * __popc(F & m));
            }
        }
        sw[c] = nsw;
    }
}

int sk_inblock(const SkDev& d, int b0, int prev_b0, int B, bool after_inblock, cudaStream_t st) {
    const int wpc = d.inblock_warps > 0 ? d.inblock_warps : 4;
    const unsigned nb = (unsigned)((d.R + wpc - 1) / wpc);
    const int nc = B / 32;
    void (*kern)(SkDev, int, int) = nullptr;
    switch (nc) {
        case 2: kern = k_sk_inblock<2>; break;
        case 4: kern = k_sk_inblock<4>; break;
        case 8: kern = k_sk_inblock<8>; break;
        case 16: kern = k_sk_inblock<16>; break;
        default: return -1;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb);
    cfg.blockDim = dim3(32 * wpc);
    cfg.dynamicSmemBytes = (size_t)32 * nc * (2 * nc) * 4;
    cfg.stream = st;
    // directly after the previous block's in-block kernel: programmatic dependent launch, so
    // the launch and the prologue overlap that kernel
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = after_inblock ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, d, b0, prev_b0) == cudaSuccess ? 1 : -1;
}

int sk_inblock_prepare() {
    const cudaError_t e = cudaFuncSetAttribute(k_sk_inblock<16>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               32 * 16 * 32 * 4);
    return e == cudaSuccess ? 0 : -1;
}

// --------------------------------------------------------------------------------------------
// field update GEMM: H[n0.., m0..m0+127] += scale * (J[m0.., b0..b0+B) . D[n0.., b0..b0+B)^T)
// One CTA (4 warps) per 128-row x NT-replica tile; one elected thread issues TMA and MMA.
// --------------------------------------------------------------------------------------------
constexpr uint32_t kWaitPolls = 1u << 24;

// NTC: the replica tile NT fixed at compile time (64 or 128: the epilogue is then straight-line
// code), or 0 to take it from the argument nt
template <int NTC>
__global__ void __launch_bounds__(128, 1) k_sk_field_mma(const __grid_constant__ CUtensorMap mapJ,
                                                      const __grid_constant__ CUtensorMap mapD,
                                                      SkDev d, int b0, int B, int kw, int nt,
                                                      int scale, int skip0, int skip1,
                                                      int atomic_add) {
    const int NT = NTC ? NTC : nt;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned operand area
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nchunks = B / kw;
    uint8_t* sA = smem;                                  // nchunks x [128][kw]
    uint8_t* sB = smem + (size_t)nchunks * 128 * kw;     // nchunks x [NT][kw]
    uint64_t* bars = (uint64_t*)(sB + (size_t)nchunks * NT * kw);
    uint32_t* tslot = (uint32_t*)(bars + 2);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // row tiles [0, ntiles) without [skip0, skip1)
    const int tile = (int)blockIdx.x < skip0 ? (int)blockIdx.x : (int)blockIdx.x + (skip1 - skip0);
    const int m0 = tile * 128;
    if (threadIdx.x == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapJ)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapD)) : "memory");
    }
    const int n0 = blockIdx.y * NT;
    const uint32_t ncols = NT <= 32 ? 32u : (NT <= 64 ? 64u : (NT <= 128 ? 128u : 256u));

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint64_t pol_keep = l2_evict_last();

    // Prefetch this thread's fields (row m0 + 32 warp + lane, up to 128 replica columns) while
    // the operands land and the MMAs run: no other launch writes these rows meanwhile.
    const int row = m0 + 32 * warp + lane;
    int hv[4][32];
    if (!atomic_add) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (32 * c + j < NT) hv[c][j] = __ldcg(d.H + (int64_t)(n0 + 32 * c + j) * d.Np + row);
    }

    // polls of one wait (a test of the timeout path shortens them to one; drains keep the bound)
    const uint32_t polls = d.test_nowait ? 1u : kWaitPolls;
    __shared__ int mma_issued;
    bool ok = true;
    if (tid == 0) {
        mma_issued = 0;
        const uint32_t bytes = (uint32_t)(nchunks * (128 + NT) * kw);
        mbar_expect_tx(&bars[0], bytes);
        for (int kc = 0; kc < nchunks; ++kc) {
            // the couplings are read every sweep: keep them in L2
            tma_load_2d(sA + (size_t)kc * 128 * kw, &mapJ, b0 + kc * kw, m0, &bars[0], pol_keep);
            tma_load_2d(sB + (size_t)kc * NT * kw, &mapD, b0 + kc * kw, n0, &bars[0], pol_keep);
        }
        ok = mbar_wait(&bars[0], 0, polls);
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // instruction descriptor: D = F32, A = B = E4M3, both K-major, M = 128, N = NT
            const uint32_t idesc = (1u << 4) | ((uint32_t)(NT >> 3) << 17) | ((128u >> 4) << 24);
            int first = 1;
            for (int kc = 0; kc < nchunks; ++kc)
                for (int ks = 0; ks < kw / 32; ++ks) {
                    const uint64_t ad = smem_desc(smem_addr(sA + (size_t)kc * 128 * kw) + ks * 32, kw);
                    const uint64_t bd = smem_desc(smem_addr(sB + (size_t)kc * NT * kw) + ks * 32, kw);
                    const uint32_t acc = first ? 0u : 1u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                    first = 0;
                }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&bars[1]))
                : "memory");
            mma_issued = 1;
        } else {
            atomicOr(d.err, 1);
        }
    }
    ok = __syncthreads_and(ok);
    if (ok) {
        ok = mbar_wait(&bars[1], 0, polls);
        if (!ok) atomicOr(d.err, 2);
    }
    ok = __syncthreads_and(ok);
    // an MMA that was issued must have finished with tensor memory before it is released
    if (!ok && mma_issued && tid == 0) mbar_wait(&bars[1], 0, kWaitPolls);
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (32 * c >= NT) break;
            uint32_t v[32];
            const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * c);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                  "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                  "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
                  "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                  "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
                  "=r"(v[30]), "=r"(v[31])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            int* hbase = d.H + (int64_t)(n0 + 32 * c) * d.Np + row;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (32 * c + j >= NT) break;
                const int dv = __float2int_rn(__uint_as_float(v[j]));
                if (atomic_add) {
                    // concurrent updates of the same rows (split across streams) commute
                    if (dv) atomicAdd(hbase + (int64_t)j * d.Np, scale * dv);
                } else {
                    hbase[(int64_t)j * d.Np] = hv[c][j] + scale * dv;
                }
            }
        }
    } else if (tid == 0) {
        // give any copies still in flight a bounded chance to land before the CTA exits
        mbar_wait(&bars[0], 0, kWaitPolls);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                     : "memory");
}

size_t sk_field_smem_bytes(int B, int kw, int NT) {
    const int nchunks = B / kw;
    return 1024 + (size_t)nchunks * (128 + NT) * kw + 64;
}

int sk_field_update_rows(const SkDev& d, const CUtensorMap& mapJ, const CUtensorMap& mapD, int b0,
                         int B, int kw, int NT, int scale, int skip0, int skip1, int atomic_add,
                         cudaStream_t st) {
    const int ntiles = d.Np / 128;
    const int n = ntiles - (skip1 - skip0);
    if (n <= 0) return 0;
    const size_t smem = sk_field_smem_bytes(B, kw, NT);
    dim3 grid((unsigned)n, (unsigned)(d.R / NT));
    if (NT == 64)
        k_sk_field_mma<64><<<grid, 128, smem, st>>>(mapJ, mapD, d, b0, B, kw, NT, scale, skip0,
                                                    skip1, atomic_add);
    else if (NT == 128)
        k_sk_field_mma<128><<<grid, 128, smem, st>>>(mapJ, mapD, d, b0, B, kw, NT, scale, skip0,
                                                     skip1, atomic_add);
    else
        k_sk_field_mma<0><<<grid, 128, smem, st>>>(mapJ, mapD, d, b0, B, kw, NT, scale, skip0,
                                                   skip1, atomic_add);
    return 1;
}

int sk_field_update(const SkDev& d, const CUtensorMap& mapJ, const CUtensorMap& mapD, int b0,
                    int B, int kw, int NT, int scale, cudaStream_t st) {
    return sk_field_update_rows(d, mapJ, mapD, b0, B, kw, NT, scale, 0, 0, 0, st);
}

// The limit is a property of the kernel, shared by every handle and every host thread: it only
// ever grows, under a lock.
static int g_field_smem_limit = 0;
static std::mutex g_field_smem_mutex;

int sk_field_prepare(int B, int kw, int NT) {
    const int need = (int)sk_field_smem_bytes(B, kw, NT);
    std::lock_guard<std::mutex> lock(g_field_smem_mutex);
    if (need <= g_field_smem_limit) return 0;
    for (auto kern : {k_sk_field_mma<0>, k_sk_field_mma<64>, k_sk_field_mma<128>})
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, need) !=
            cudaSuccess)
            return -1;
    g_field_smem_limit = need;
    return 0;
}

// --------------------------------------------------------------------------------------------
// plain kernel: one thread block per replica, spins in the fixed order, fields in shared memory
// --------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sk_plain_sweep(SkDev d, const uint32_t* clock,
                                                        uint32_t t_off) {
    const uint32_t t = *clock + t_off;
    extern __shared__ int sh[];
    int* h = sh;                          // [Np]
    int* kst = sh + d.Np;                 // [Np]
    uint32_t* sb = (uint32_t*)(kst + d.Np);  // [Np/32]
    __shared__ int flip_sign;
    const int r = blockIdx.x;
    const int words = d.Np / 32;
    const uint32_t* thr = d.thr + (int64_t)d.temp_index[r] * d.N;
    for (int i = threadIdx.x; i < d.Np; i += blockDim.x) {
        h[i] = d.H[(int64_t)r * d.Np + i];
        if (i < d.N) {
            const uint4 rnd = philox4x32_10(make_uint4((uint32_t)i, t, (uint32_t)(r >> 2), 0u),
                                            (uint32_t)d.seed, (uint32_t)(d.seed >> 32));
            kst[i] = sk_kstar(uint4_word(rnd, r & 3), thr, d.N, d.coef[r]);
        }
    }
    for (int w = threadIdx.x; w < words; w += blockDim.x) sb[w] = d.S[(int64_t)r * words + w];
    __syncthreads();
    for (int i = 0; i < d.N; ++i) {
        if (threadIdx.x == 0) {
            const int s = ((sb[i >> 5] >> (i & 31)) & 1u) ? -1 : 1;
            const bool flip = s * h[i] <= kst[i];
            if (flip) sb[i >> 5] ^= 1u << (i & 31);
            flip_sign = flip ? -s : 0;  // new spin value, or 0 for no flip
        }
        __syncthreads();
        const int sn = flip_sign;
        if (sn) {
            const uint8_t* row = d.J8 + (int64_t)i * d.Np;
            for (int j = threadIdx.x; j < d.Np; j += blockDim.x) {
                const uint8_t b = row[j];
                const int J = b == 0x38 ? 1 : (b == 0xB8 ? -1 : 0);
                h[j] += 2 * J * sn;
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < d.Np; i += blockDim.x) d.H[(int64_t)r * d.Np + i] = h[i];
    for (int w = threadIdx.x; w < words; w += blockDim.x) d.S[(int64_t)r * words + w] = sb[w];
}

size_t sk_plain_smem_bytes(int Np) { return (size_t)Np * 8 + (size_t)Np / 8; }

static int g_plain_smem_limit = 0;

int sk_plain_prepare(int Np) {
    const int need = (int)sk_plain_smem_bytes(Np);
    if (need <= g_plain_smem_limit) return 0;
    const cudaError_t e = cudaFuncSetAttribute(k_sk_plain_sweep,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    if (e != cudaSuccess) return -1;
    g_plain_smem_limit = need;
    return 0;
}

int sk_plain_sweep(const SkDev& d, const uint32_t* clock, uint32_t t_off, cudaStream_t st) {
    k_sk_plain_sweep<<<(unsigned)d.R, 256, sk_plain_smem_bytes(d.Np), st>>>(d, clock, t_off);
    return 1;
}

// --------------------------------------------------------------------------------------------
// measurements: per replica, Hamming distances to snapshots, the pair overlap, and the energy
//   diff_C[r][w] (w < n_active), diff_q[r/2] (even r), E[r] = sum_{i<j} J_ij s_i s_j
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ long long block_sum(long long v, long long* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    long long tot = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    return tot;  // valid in thread 0
}

__global__ void k_sk_measure(SkDev d, int n_active, int64_t* cdst, int64_t c_stride_r,
                             int64_t c_stride_w, int64_t* qdst, int64_t q_stride_p, int64_t* edst,
                             int64_t e_stride_r) {
    __shared__ long long red[32];
    const int r = blockIdx.x;
    const int words = d.Np / 32;
    const uint32_t* S = d.S + (int64_t)r * words;
    for (int w = 0; w < n_active; ++w) {
        const uint32_t* P = d.snap + ((int64_t)w * d.R + r) * words;
        long long acc = 0;
        for (int k = threadIdx.x; k < words; k += blockDim.x) acc += __popc(S[k] ^ P[k]);
        const long long tot = block_sum(acc, red);
        if (threadIdx.x == 0) cdst[r * c_stride_r + w * c_stride_w] += tot;
    }
    if ((r & 1) == 0 && r + 1 < d.R && qdst) {
        const uint32_t* S2 = S + words;
        long long acc = 0;
        for (int k = threadIdx.x; k < words; k += blockDim.x) acc += __popc(S[k] ^ S2[k]);
        const long long tot = block_sum(acc, red);
        if (threadIdx.x == 0) qdst[(r >> 1) * q_stride_p] += tot;
    }
    long long acc = 0;
    for (int i = threadIdx.x; i < d.N; i += blockDim.x) {
        const int s = ((S[i >> 5] >> (i & 31)) & 1u) ? -1 : 1;
        acc += (long long)s * d.H[(int64_t)r * d.Np + i];
    }
    const long long tot = block_sum(acc, red);
    if (threadIdx.x == 0) edst[r * e_stride_r] += tot / 2;
}

int sk_measure(const SkDev& d, int n_active, int64_t* cdst, int64_t c_stride_r,
               int64_t c_stride_w, int64_t* qdst, int64_t q_stride_p, int64_t* edst,
               int64_t e_stride_r, cudaStream_t st) {
    k_sk_measure<<<(unsigned)d.R, 256, 0, st>>>(d, n_active, cdst, c_stride_r, c_stride_w, qdst,
                                               q_stride_p, edst, e_stride_r);
    return 1;
}

__global__ void k_copy_words(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t n16) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

int sk_snapshot(const SkDev& d, int w, cudaStream_t st) {
    const int64_t words = (int64_t)d.R * (d.Np / 32);
    const int64_t n16 = words / 4;
    int64_t nb = (n16 + 255) / 256;
    if (nb > 1024) nb = 1024;
    if (nb < 1) nb = 1;
    k_copy_words<<<(unsigned)nb, 256, 0, st>>>((const uint4*)d.S, (uint4*)(d.snap + w * words), n16);
    return 1;
}

}  // namespace sg
