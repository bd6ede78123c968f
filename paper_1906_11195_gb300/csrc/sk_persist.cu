// sk_persist.cu -- persistent Sherrington-Kirkpatrick sweeps with the local fields resident in
// tensor memory (sm_103a): one cooperative launch runs several consecutive sweeps.
//
// Every sweep visits i = 0..N-1 in order (SI section 1).  The spins are cut into blocks of 128,
// and the fields H[i][r] = sum_j J_ij s_j^r into the same 128-row tiles.  Blocks are numbered
// k = s nb + b over the sweeps s of the launch (nb blocks per sweep).  Two kinds of CTA share
// the launch (all CTAs resident):
//
//   field CTAs (the first nG): CTA j owns the row tiles t = j, j + nG, ... (TPC of them).  Their
//     fields live in tensor memory as FP32 accumulators for the whole launch (loaded from H at
//     the start, written back at the end).  For every block k, once the spin changes
//     D_k = (s' - s)/2 of all replicas are published (stored as 2 D_k), the CTA loads
//     J[tile rows][block b] and 2 D_k with TMA and adds J (2 D_k) to each of its tiles with
//     tcgen05.mma (kind::f8f6f4, e4m3 operands: J = +-1 and 2 D in {-2, 0, +2} are exact, and so
//     is every partial sum, because |H| < N <= 2^15 stays far below 2^24).  When block k has
//     been applied, the tile of chain block k + L + 1 (if the CTA owns it) is copied to Hpub and
//     H_ready of that tile is raised to k + L + 2.
//
//   chain CTAs (the next nC): CTA c owns replicas W c .. W c + W - 1, one warp per replica, plus
//     a staging warp.  For block k the staging warp loads (TMA, into a ring of shared-memory
//     stages) the couplings of block b's rows with the columns of blocks k - L .. k (as bits),
//     the replicas' K* (the largest accepted k of each spin's random number, computed for all
//     sweeps of the launch before it starts) and the fields of block b's rows: from H itself
//     for k <= L (nothing of
//     this launch has reached them through the tensor cores yet), else from Hpub once H_ready
//     says it holds every block before k - L.  The replica warp adds the flips of blocks
//     k - L .. k - 1 of this launch (its own, kept in shared memory) with popcounts over the
//     coupling bits, then takes the 128 sequential decisions (ballot per accepted flip, as in
//     the in-block kernel) and writes 2 D_k into ring slot k mod Q.  The staging warp raises
//     D_count[slot] once every replica warp of the CTA is done with the block.
//
// So the sequential chain of a replica never waits for a launch or for the tensor cores, as
// long as the field CTAs publish a tile within L chain blocks; it needs L < nb so that a fold
// window never holds a block twice.  Ring slots are reused only after every field CTA has read
// them (D_free).  Every wait is bounded (global timer); a CTA that gives up flags d.err, drains
// its copies and tensor-core work in flight with the normal bound, releases its tensor memory
// and exits, and the other CTAs notice the flag and do the same.  The counters are zero at the
// start of every launch.
#include <cuda.h>

#include "sg_internal.cuh"
#include "sk_internal.cuh"

namespace sg {

namespace {

constexpr uint64_t kPersistWaitNs = 2000000000ull;  // 2 s: only a broken launch waits that long
constexpr uint32_t kTileBytes = 128 * 128;          // one e4m3 128 x 128 coupling tile
constexpr int kChainStages = 3;  // staged blocks ahead of the chain

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}


__device__ __forceinline__ int err_raised(const int* err) {
    return *reinterpret_cast<const volatile int*>(err);
}

// Wait until *p >= target.  False when the bound passes, when another CTA has flagged an error,
// or at once if the test hook asks for single checks.
__device__ bool wait_at_least(const uint32_t* p, uint32_t target, const int* err, bool nowait) {
    if (ld_acquire(p) >= target) return true;
    if (nowait) return false;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (it > 256) __nanosleep(64);
        if (ld_acquire(p) >= target) return true;
        if ((it & 31) == 0 && (err_raised(err) || global_ns() - t0 > kPersistWaitNs)) return false;
    }
}

// the same on a counter in this CTA's shared memory
__device__ bool wait_smem_at_least(const uint32_t* p, uint32_t target, const int* err, bool nowait,
                                   const volatile int* abort_flag) {
    auto load = [&] {
        uint32_t v;
        asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
        return v;
    };
    if (load() >= target) return true;
    if (nowait) return false;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (load() >= target) return true;
        if ((it & 63) == 0 && (err_raised(err) || *abort_flag || global_ns() - t0 > kPersistWaitNs))
            return false;
    }
}

// mbarrier wait bounded by the global timer that also gives up when an error is flagged; it
// spins on try_wait (no suspend hint: the waits sit on the sequential chain's critical path)
__device__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t phase, const int* err, bool nowait,
                                   const volatile int* abort_flag) {
    if (mbar_try_wait(bar, phase)) return true;
    if (nowait) return false;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, phase)) return true;
        if ((it & 63) == 0 &&
            (err_raised(err) || *abort_flag || global_ns() - t0 > kPersistWaitNs))
            return false;
    }
}

// 2 D in e4m3 for D in {-1, 0, 1}: +-2.0 (0x40, 0xC0) or 0, so that one MMA adds the whole field
// change 2 J D (the accumulators hold the fields themselves; there is no epilogue to scale)
__device__ __forceinline__ uint8_t e4m3_twice(int v) {
    return v > 0 ? (uint8_t)0x40 : (v < 0 ? (uint8_t)0xC0 : (uint8_t)0x00);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
        "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
        "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
        "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

// shared memory of a field CTA: nst stages of {TPC coupling tiles, the D tile}
__host__ __device__ __forceinline__ size_t field_stage_bytes(int TPC, int R) {
    return (size_t)TPC * kTileBytes + (size_t)R * 128;
}

// shared memory of a chain CTA: spin and flip words of its replicas, the fold warps' fields
// for two blocks, then the staged ring
__host__ __device__ __forceinline__ size_t chain_words_bytes(int W, int Np) {
    return (size_t)2 * W * (Np / 32) * 4 + (size_t)2 * W * 128 * 4;
}
__host__ __device__ __forceinline__ size_t chain_stage_bytes(int W, int L) {
    return (size_t)(L + 1) * 4 * 128 * 4 + (size_t)W * 128 * (2 + 4);  // coupling words, K*, fields
}

}  // namespace

// ------------------------------------------------------------------------------------------
// field CTA: warp W (lane 0) loads the operands, thread 0 issues the MMAs, warps 0..3 (128
// threads, one per tensor-memory lane) move fields between tensor memory and global memory
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void bar_epilogue() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// barrier of the 128 epilogue threads that also returns whether all of them passed v: every
// decision that leads into or around a barrier is taken uniformly
__device__ __forceinline__ bool epilogue_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0u;
}

template <int W>
__device__ void persist_field_cta(const CUtensorMap* mapJ, const CUtensorMap* mapD,
                                  const SkPersistMaps& m, const SkDev& d, const SkPersistArgs& a,
                                  uint8_t* smem, uint64_t* bars, uint32_t* tslot,
                                  volatile int* abort_flag) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int j = blockIdx.x;
    const int R = d.R, Np = d.Np, nb = a.nb, nst = a.nst, L = a.L;
    constexpr int Q = kSkPersistSlots;
    const int nk = a.n_sweeps * nb;  // blocks of the launch
    const bool nowait = d.test_nowait != 0;
    int ntl = 0;  // tiles owned
    for (int u = 0; u < a.TPC; ++u)
        if (j + u * a.nG < nb) ++ntl;
    uint64_t* full = bars;           // [nst]: operands landed (A and B arrivals + bytes)
    uint64_t* mdone = bars + nst;    // [nst]: the block's MMAs finished
    const size_t sbytes = field_stage_bytes(a.TPC, R);
    uint32_t* D_count = a.sync;
    uint32_t* D_free = a.sync + Q;
    uint32_t* H_ready = a.sync + 2 * Q;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(a.TPC * R)) ncols <<= 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 2);
            mbar_init(&mdone[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    // the fields of the owned tiles into tensor memory: warp w holds rows 32 w .. 32 w + 31
    if (warp < 4) {
        for (int u = 0; u < ntl; ++u) {
            const int row = (j + u * a.nG) * 128 + 32 * warp + lane;
            for (int c = 0; c < R / 32; ++c) {
                uint32_t v[32];
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    v[q] = __float_as_uint((float)__ldcg(d.H + (int64_t)(32 * c + q) * Np + row));
                tmem_st32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(u * R + 32 * c), v);
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (warp == W) {
        // ---------------- operand producer ----------------
        if (lane == 0) {
            const uint64_t pol = l2_evict_last();
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(mapJ)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(mapD)) : "memory");
            int blk[4] = {-1, -1, -1, -1};     // latest block issued into each stage
            bool b_in[4] = {false, false, false, false};
            for (int k = 0; k < nk; ++k) {
                const int s = k % nst;
                const int b = k % nb;
                if (k >= nst && !mbar_wait_or_abort(&mdone[s], (uint32_t)(k / nst - 1) & 1u, d.err, nowait,
                                                    abort_flag)) {
                    atomicOr(d.err, 64);
                    *abort_flag = 1;
                    break;
                }
                uint8_t* st = smem + (size_t)s * sbytes;
                // the couplings depend on nothing of the sweep: issued before the wait below
                mbar_expect_tx(&full[s], (uint32_t)ntl * kTileBytes);
                for (int u = 0; u < ntl; ++u)
                    tma_load_2d(st + (size_t)u * kTileBytes, mapJ, b * 128, (j + u * a.nG) * 128, &full[s], pol);
                blk[s] = k;
                b_in[s] = false;
                if (!wait_at_least(&D_count[k % Q], (uint32_t)(k / Q + 1) * (uint32_t)a.nC, d.err, nowait)) {
                    atomicOr(d.err, 16);
                    *abort_flag = 1;
                    break;
                }
                fence_proxy_async_global();
                mbar_expect_tx(&full[s], (uint32_t)R * 128u);
                tma_load_2d(st + (size_t)a.TPC * kTileBytes, mapD, 0, (k % Q) * R, &full[s], pol);
                b_in[s] = true;
            }
            if (*abort_flag) {
                // every copy that was issued lands before the CTA releases its shared memory
                for (int s = 0; s < nst; ++s) {
                    if (blk[s] < 0) continue;
                    if (!b_in[s]) mbar_arrive(&full[s]);  // the spin changes were never requested
                    mbar_wait_timed(&full[s], (uint32_t)(blk[s] / nst) & 1u, kPersistWaitNs);
                }
            }
        }
    } else if (warp < 4) {
        // ---------------- MMA issue (thread 0) and epilogue (warps 0..3) ----------------
        const uint32_t idesc = (1u << 4) | ((uint32_t)(R >> 3) << 17) | ((128u >> 4) << 24);
        int last_commit = -1;
        for (int k = 0; k < nk; ++k) {
            const int s = k % nst;
            const uint32_t ph = (uint32_t)(k / nst) & 1u;
            if (tid == 0 && !*abort_flag) {
                if (!mbar_wait_or_abort(&full[s], ph, d.err, nowait, abort_flag)) {
                    atomicOr(d.err, 32);
                    *abort_flag = 1;
                } else {
                    // every field CTA has its copy once all have arrived here: slot reusable
                    red_release_add(&D_free[k % Q], 1u);
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint8_t* st = smem + (size_t)s * sbytes;
                    const uint8_t* sb = st + (size_t)a.TPC * kTileBytes;
                    for (int u = 0; u < ntl; ++u)
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = smem_desc(smem_addr(st + (size_t)u * kTileBytes) + ks * 32, 128);
                            const uint64_t bd = smem_desc(smem_addr(sb) + ks * 32, 128);
                            asm volatile(
                                "{\n\t.reg .pred p;\n\t"
                                "setp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                    tmem + (uint32_t)(u * R)),
                                "l"(ad), "l"(bd), "r"(idesc), "r"(1u)
                                : "memory");
                        }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_addr(&mdone[s]))
                        : "memory");
                    last_commit = k;
                }
            }
            // publish the tile of chain block kc = k + L + 1 once block k is in it (its chain
            // block needs exactly that)
            const int kc = k + L + 1;
            int pub_u = -1;
            if (kc < nk)
                for (int u = 0; u < ntl; ++u)
                    if (j + u * a.nG == kc % nb) pub_u = u;
            if (pub_u >= 0) {
                bool ok = epilogue_all(!*abort_flag);
                if (ok) ok = mbar_wait_or_abort(&mdone[s], ph, d.err, nowait, abort_flag);
                ok = epilogue_all(ok);
                if (ok) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // Hpub is [replica][row]: a warp's 32 rows of one replica are 128 contiguous
                    // bytes
                    const int row = (kc % nb) * 128 + 32 * warp + lane;
                    for (int c = 0; c < R / 32; ++c) {
                        uint32_t v[32];
                        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(pub_u * R + 32 * c), v);
#pragma unroll
                        for (int q = 0; q < 32; ++q)
                            __stcg(a.Hpub + (int64_t)(32 * c + q) * Np + row, __float2int_rn(__uint_as_float(v[q])));
                    }
                    fence_proxy_async_global();  // read by the chains' TMA copies
                } else if (tid == 0) {
                    atomicOr(d.err, 128);
                    *abort_flag = 1;
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                bar_epilogue();
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // H_ready[tile] = kc + 1: the tile holds every block before kc - L
                if (tid == 0 && ok)
                    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&H_ready[kc % nb]),
                                 "r"((uint32_t)(kc + 1))
                                 : "memory");
            }
        }
        bar_epilogue();
        // final fields back to H once the last MMAs are done
        if (!*abort_flag) {
            const int kl = nk - 1;
            if (mbar_wait_or_abort(&mdone[kl % nst], (uint32_t)(kl / nst) & 1u, d.err, nowait, abort_flag)) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int u = 0; u < ntl; ++u) {
                    const int row = (j + u * a.nG) * 128 + 32 * warp + lane;
                    for (int c = 0; c < R / 32; ++c) {
                        uint32_t v[32];
                        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(u * R + 32 * c), v);
#pragma unroll
                        for (int q = 0; q < 32; ++q)
                            d.H[(int64_t)(32 * c + q) * Np + row] = __float2int_rn(__uint_as_float(v[q]));
                    }
                }
            } else {
                atomicOr(d.err, 256);
                *abort_flag = 1;
            }
        }
        // issued MMAs finish before the tensor memory is released (full bound)
        if (tid == 0 && *abort_flag && last_commit >= 0)
            mbar_wait_timed(&mdone[last_commit % nst], (uint32_t)(last_commit / nst) & 1u, kPersistWaitNs);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                     : "memory");
}

// ------------------------------------------------------------------------------------------
// chain CTA: warps 0..W-1 are the replicas' chains, warps W..2W-1 their fold warps, warp 2W
// (lane 0) stages the blocks, warp 2W + 1 (lane 0) tells the field CTAs (D_count) when every
// replica warp has written a block's spin changes.  For block k the fold warp of replica w adds to the staged fields
// the flips of blocks k - L .. k - 2 (complete while the chain runs block k - 1) and hands the
// result over in shared memory; the chain warp adds block k - 1's flips itself (16 popcounts
// per lane) and takes the decisions.  So only one block's fold sits on the chain.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void fold_block(int (&h)[4], const uint32_t* Jp, const uint32_t* Fw,
                                           const uint32_t* Sw, int bp, bool live, uint32_t lane) {
    uint32_t Fv[4], sv[4], jv[4][4];
#pragma unroll
    for (int cp = 0; cp < 4; ++cp) {
        Fv[cp] = live ? Fw[bp * 4 + cp] : 0u;
        sv[cp] = Sw[bp * 4 + cp];
#pragma unroll
        for (int q = 0; q < 4; ++q) jv[cp][q] = Jp[cp * 128 + 32 * q + lane];
    }
#pragma unroll
    for (int cp = 0; cp < 4; ++cp) {
        const int pf = __popc(Fv[cp]);
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] += 2 * (pf - 2 * __popc(Fv[cp] & (jv[cp][q] ^ sv[cp])));
    }
}

template <int W, int L>
__device__ void persist_chain_cta(const SkDev& d, const SkPersistArgs& a, const SkPersistMaps& m,
                                  uint8_t* smem, uint64_t* bars, uint32_t* done_cnt,
                                  volatile int* abort_flag) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = blockIdx.x - a.nG;
    const int r0 = c * W;
    const int Np = d.Np, R = d.R, nb = a.nb;
    constexpr int Q = kSkPersistSlots;
    const int nk = a.n_sweeps * nb;
    const int words = Np / 32;
    const bool nowait = d.test_nowait != 0;
    uint32_t* Ssm = reinterpret_cast<uint32_t*>(smem);          // [W][words] spin words
    uint32_t* Fsm = Ssm + (size_t)W * words;                     // [W][words] latest flips
    int32_t* hb = reinterpret_cast<int32_t*>(Fsm + (size_t)W * words);  // [2][W][128] folded fields
    uint8_t* ring = smem + chain_words_bytes(W, Np);
    const size_t stb = chain_stage_bytes(W, L);
    uint64_t* fullc = bars;                   // [kChainStages]: the stage's copies landed
    uint64_t* emptyc = bars + kChainStages;   // [kChainStages]: chain and fold warps done
    uint64_t* cdone = bars + 2 * kChainStages;    // [W][2]: the chain finished block k (k & 1)
    uint64_t* hrdy = cdone + 2 * W;               // [W][2]: folded fields of block k (k & 1)
    uint32_t* D_count = a.sync;
    uint32_t* D_free = a.sync + Q;
    uint32_t* H_ready = a.sync + 2 * Q;

    if (tid == 0) {
        for (int s = 0; s < kChainStages; ++s) {
            mbar_init(&fullc[s], 1);
            mbar_init(&emptyc[s], 2 * W);
        }
        for (int i = 0; i < 4 * W; ++i) mbar_init(&cdone[i], 1);  // cdone and hrdy
        for (int w = 0; w < W; ++w) done_cnt[w] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp < W) {
        const uint32_t* Sg = d.S + (int64_t)(r0 + warp) * words;
        for (int k = lane; k < words; k += 32) {
            Ssm[warp * words + k] = Sg[k];
            Fsm[warp * words + k] = 0u;
        }
    }
    __syncthreads();

    if (warp == 2 * W) {
        // ---------------- staging warp: block k (couplings, K*, fields) ----------------
        if (lane == 0) {
            const uint32_t stage_tx = (uint32_t)chain_stage_bytes(W, L);
            const uint64_t pol = l2_evict_last();
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&m.jb)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&m.hpub)) : "memory");
            int last_fill[kChainStages];
            for (int s = 0; s < kChainStages; ++s) last_fill[s] = -1;
            auto prefetch = [&](int k) -> bool {
                const int s = k % kChainStages;
                const int b = k % nb, sw = k / nb;
                // ring slot k mod Q: its previous contents (block k - Q) read by every field CTA
                if (k >= Q && !wait_at_least(&D_free[k % Q], (uint32_t)(k / Q) * (uint32_t)a.nG, d.err, nowait)) {
                    atomicOr(d.err, 512);
                    return false;
                }
                const bool pub = k > L;
                if (pub && !wait_at_least(&H_ready[b], (uint32_t)(k + 1), d.err, nowait)) {
                    atomicOr(d.err, 1024);
                    return false;
                }
                if (pub) fence_proxy_async_global();  // the fields were written by generic stores
                uint8_t* st = ring + (size_t)s * stb;
                uint32_t* Jw = reinterpret_cast<uint32_t*>(st);                    // [(L+1)*4][128]
                int16_t* ks = reinterpret_cast<int16_t*>(Jw + (L + 1) * 4 * 128);  // [W][128]
                int32_t* hs = reinterpret_cast<int32_t*>(ks + W * 128);           // [W][128]
                mbar_expect_tx(&fullc[s], stage_tx);
                // couplings of block b's rows with the columns of blocks k - L .. k (cyclic in
                // the sweep; a block before the launch's first is never folded, any rows do)
                for (int i = 0; i <= L; ++i) {
                    int bi = b - L + i;
                    if (bi < 0) bi += nb;  // L < nb
                    tma_load_2d(Jw + i * 4 * 128, &m.jb, b * 128, bi * 4, &fullc[s], pol);
                }
                tma_load_2d(ks, &m.kst, b * 128, sw * R + r0, &fullc[s], pol);
                tma_load_2d(hs, pub ? &m.hpub : &m.h, b * 128, r0, &fullc[s], pol);
                last_fill[s] = k;
                return true;
            };
            bool ok = true;
            for (int k = 0; k < kChainStages && k < nk && ok; ++k) ok = prefetch(k);
            for (int k = 0; k < nk && ok; ++k) {
                const int s = k % kChainStages;
                if (!mbar_wait_or_abort(&emptyc[s], (uint32_t)(k / kChainStages) & 1u, d.err, nowait,
                                        abort_flag)) {
                    atomicOr(d.err, 2048);
                    ok = false;
                    break;
                }
                if (k + kChainStages < nk) ok = prefetch(k + kChainStages);
            }
            if (!ok) {
                *abort_flag = 1;
                // copies that were issued land before the CTA exits
                for (int s = 0; s < kChainStages; ++s)
                    if (last_fill[s] >= 0)
                        mbar_wait_timed(&fullc[s], (uint32_t)(last_fill[s] / kChainStages) & 1u, kPersistWaitNs);
            }
        }
    } else if (warp == 2 * W + 1) {
        // ---------------- release warp: D_count of block k once every replica wrote D_k ------
        // (apart from the staging warp, whose next stage does not wait for this gpu-scope
        // release, about a microsecond)
        if (lane == 0) {
            for (int k = 0; k < nk; ++k) {
                bool ok = true;
                for (int w = 0; w < W && ok; ++w)
                    ok = wait_smem_at_least(&done_cnt[w], (uint32_t)(k + 1), d.err, nowait, abort_flag);
                if (!ok) {
                    atomicOr(d.err, 65536);
                    *abort_flag = 1;
                    break;
                }
                red_release_add(&D_count[k % Q], 1u);
            }
        }
    } else if (warp >= W) {
        // ---------------- fold warp of replica w ----------------
        const int w = warp - W;
        const uint32_t* Sw = Ssm + w * words;
        const uint32_t* Fw = Fsm + w * words;
        for (int k = 0, b = 0; k < nk; ++k, b = (b + 1 == nb) ? 0 : b + 1) {
            const int s = k % kChainStages;
            bool ok = mbar_wait_or_abort(&fullc[s], (uint32_t)(k / kChainStages) & 1u, d.err, nowait,
                                         abort_flag);
            // the chain has finished block k - 2 (its flips and spins are in shared memory)
            if (ok && k >= 2)
                ok = mbar_wait_or_abort(&cdone[w * 2 + (k & 1)], (uint32_t)((k - 2) >> 1) & 1u, d.err,
                                        nowait, abort_flag);
            if (!ok) {
                if (lane == 0) atomicOr(d.err, 32768);
                *abort_flag = 1;
                break;
            }
            const uint32_t* Jw = reinterpret_cast<const uint32_t*>(ring + (size_t)s * stb);
            const int16_t* ks16 = reinterpret_cast<const int16_t*>(Jw + (L + 1) * 4 * 128);
            const int32_t* hs = reinterpret_cast<const int32_t*>(ks16 + W * 128) + w * 128;
            int h[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) h[q] = hs[32 * q + lane];
#pragma unroll
            for (int i = 0; i < L - 1; ++i) {
                int bp = b - L + i;
                if (bp < 0) bp += nb;  // L < nb
                fold_block(h, Jw + i * 4 * 128, Fw, Sw, bp, k - L + i >= 0, lane);
            }
            int32_t* hd = hb + ((k & 1) * W + w) * 128;
#pragma unroll
            for (int q = 0; q < 4; ++q) hd[32 * q + lane] = h[q];
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&hrdy[w * 2 + (k & 1)]);
                mbar_arrive(&emptyc[s]);
            }
        }
    } else {
        // ---------------- replica warp ----------------
        const int r = r0 + warp;
        uint32_t* Sw = Ssm + warp * words;
        uint32_t* Fw = Fsm + warp * words;
        const uint32_t lane_bit = 1u << lane;
        for (int k = 0, b = 0; k < nk; ++k, b = (b + 1 == nb) ? 0 : b + 1) {
            const int s = k % kChainStages;
            bool ok = mbar_wait_or_abort(&fullc[s], (uint32_t)(k / kChainStages) & 1u, d.err, nowait,
                                         abort_flag);
            if (ok)
                ok = mbar_wait_or_abort(&hrdy[warp * 2 + (k & 1)], (uint32_t)(k >> 1) & 1u, d.err,
                                        nowait, abort_flag);
            if (!ok) {
                if (lane == 0) atomicOr(d.err, 4096);
                *abort_flag = 1;
                break;
            }
            const uint8_t* st = ring + (size_t)s * stb;
            const uint32_t* Jw = reinterpret_cast<const uint32_t*>(st);
            const int16_t* ks = reinterpret_cast<const int16_t*>(Jw + (L + 1) * 4 * 128) + warp * 128;
            const uint32_t* Jown = Jw + L * 4 * 128;  // [4 column words][128 rows] of block b
            const int32_t* hd = hb + ((k & 1) * W + warp) * 128;
            int h[4], kst[4];
            uint32_t sw[4], jd[4], jl[6];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                h[q] = hd[32 * q + lane];
                kst[q] = ks[32 * q + lane];
                sw[q] = Sw[b * 4 + q];
                jd[q] = Jown[q * 128 + 32 * q + lane];  // couplings inside chunk q
            }
            // couplings of chunk q's columns with the rows of a later chunk q2
            jl[0] = Jown[0 * 128 + 32 * 1 + lane];
            jl[1] = Jown[0 * 128 + 32 * 2 + lane];
            jl[2] = Jown[0 * 128 + 32 * 3 + lane];
            jl[3] = Jown[1 * 128 + 32 * 2 + lane];
            jl[4] = Jown[1 * 128 + 32 * 3 + lane];
            jl[5] = Jown[2 * 128 + 32 * 3 + lane];
            // the flips of block k - 1, just taken: the one fold left on the chain
            {
                int bp = b - 1;
                if (bp < 0) bp += nb;
                fold_block(h, Jw + (L - 1) * 4 * 128, Fw, Sw, bp, k >= 1, lane);
            }
            uint8_t* Dslot = a.Dring + ((int64_t)(k % Q) * R + r) * 128;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t sbit = (sw[q] >> lane) & 1u;
                const int x = sbit ? -h[q] : h[q];
                const uint32_t neg = jd[q] ^ sw[q] ^ (sbit ? 0xFFFFFFFFu : 0u);
                uint32_t F = 0, last = 0;
                int cur = x;
                for (;;) {
                    const bool tent = lane_bit > last && cur <= kst[q];
                    const uint32_t bm = __ballot_sync(0xFFFFFFFFu, tent);
                    if (bm == 0u) break;
                    last = bm & (0u - bm);
                    F |= last;
                    cur += (neg & last) ? 2 : -2;
                }
                const uint32_t nsw = sw[q] ^ F;
                const int dval = ((F >> lane) & 1u) ? (sbit ? 1 : -1) : 0;
                Dslot[32 * q + lane] = e4m3_twice(dval);
                if (lane == 0) {
                    Sw[b * 4 + q] = nsw;
                    Fw[b * 4 + q] = F;
                }
                {
                    const int pf = __popc(F);
#pragma unroll
                    for (int q2 = q + 1; q2 < 4; ++q2) {
                        const uint32_t jw = jl[q == 0 ? q2 - 1 : (q == 1 ? q2 + 1 : 5)];
                        h[q2] += 2 * (pf - 2 * __popc(F & (jw ^ nsw)));
                    }
                }
                sw[q] = nsw;
            }
            // D_k of this replica is written: order it for the tensor-core readers; tell the
            // fold warp that block k is done; release the stage (the staging warp publishes
            // the block once every warp is done)
            fence_proxy_async_global();
            __syncwarp();
            if (lane == 0) {
                asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(&done_cnt[warp])),
                             "r"((uint32_t)(k + 1))
                             : "memory");
                mbar_arrive(&cdone[warp * 2 + (k & 1)]);
                mbar_arrive(&emptyc[s]);
            }
        }
    }
    __syncthreads();
    if (warp < W && !*abort_flag) {
        uint32_t* Sg = d.S + (int64_t)(r0 + warp) * words;
        for (int k = lane; k < words; k += 32) Sg[k] = Ssm[warp * words + k];
    }
}

template <int W, int L>
__global__ void __launch_bounds__(32 * (2 * W + 2), 1)
    k_sk_persist(const __grid_constant__ CUtensorMap mapJ, const __grid_constant__ CUtensorMap mapD,
                 const __grid_constant__ SkPersistMaps maps, SkDev d, SkPersistArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bars[2 * kChainStages + 4 * 8];  // chain CTA: W <= 8
    __shared__ uint32_t tslot;
    __shared__ uint32_t done_cnt[8];  // chain CTA: blocks each replica warp has written D for
    __shared__ int abort_flag;
    if (threadIdx.x == 0) abort_flag = 0;
    __syncthreads();
    if ((int)blockIdx.x < a.nG)
        persist_field_cta<W>(&mapJ, &mapD, maps, d, a, smem, bars, &tslot, &abort_flag);
    else
        persist_chain_cta<W, L>(d, a, maps, smem, bars, done_cnt, &abort_flag);
}

size_t sk_persist_smem_bytes(const SkDev& d, const SkPersistArgs& a) {
    const size_t f = (size_t)a.nst * field_stage_bytes(a.TPC, d.R);
    const size_t c = chain_words_bytes(a.W, d.Np) + kChainStages * chain_stage_bytes(a.W, a.L);
    const size_t need = 1024 + (f > c ? f : c);
    const size_t floor_one_per_sm = 116 * 1024;
    return need > floor_one_per_sm ? need : floor_one_per_sm;
}

// lookaheads compiled in (the fold of L blocks is unrolled)
#define SG_PERSIST_KERNELS(X) X(4, 4) X(4, 6) X(4, 8) X(8, 4) X(8, 6) X(8, 8)

static void* persist_kernel(int W, int L) {
#define SG_PERSIST_PICK(w, l) if (W == w && L == l) return (void*)k_sk_persist<w, l>;
    SG_PERSIST_KERNELS(SG_PERSIST_PICK)
#undef SG_PERSIST_PICK
    return nullptr;
}

int sk_persist_lookahead_supported(int L) { return L == 4 || L == 6 || L == 8; }

int sk_persist_fits(const SkDev& d, const SkPersistArgs& a, int num_sms) {
    void* kern = persist_kernel(a.W, a.L);
    // R: whole 32-column chunks of tensor memory, at most one TMA box of spin changes; the
    // staging warp, kChainStages blocks ahead, needs L >= kChainStages - 1 (fields published in
    // time) and a ring of at least kChainStages slots (slots freed in time)
    if (!kern || d.R < 32 || d.R > 256 || d.R % 32 || a.nst < 2 || a.nst > 4 || a.Q != kSkPersistSlots ||
        a.L < kChainStages - 1 || a.L >= a.nb || a.TPC * d.R > 512 || a.nC * a.W != d.R ||
        a.n_sweeps < 1 || kSkPersistSlots < kChainStages ||
        a.n_sweeps > kSkPersistMaxSweeps)
        return 0;
    const size_t smem = sk_persist_smem_bytes(d, a);
    if (smem > 227 * 1024) return 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * (2 * a.W + 2), smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm >= 1 && a.nG + a.nC <= per_sm * num_sms;
}

int sk_persist_sweeps(const SkDev& d, const SkPersistArgs& a, const CUtensorMap& mapJ,
                      const CUtensorMap& mapD, const SkPersistMaps& maps, cudaStream_t st) {
    if (!persist_kernel(a.W, a.L) || a.n_sweeps < 1 || a.n_sweeps > kSkPersistMaxSweeps) return -1;
    // K* of every sweep of the launch, with the whole GPU
    sk_kstar16_sweeps(d, a.clock, a.t_off, a.n_sweeps, a.kst16, st);
    if (cudaMemsetAsync(a.sync, 0, (size_t)(2 * kSkPersistSlots + a.nb) * 4, st) != cudaSuccess)
        return -1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.nG + a.nC));
    cfg.blockDim = dim3((unsigned)(32 * (2 * a.W + 2)));
    cfg.dynamicSmemBytes = sk_persist_smem_bytes(d, a);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaErrorInvalidValue;
#define SG_PERSIST_LAUNCH(w, l) \
    if (a.W == w && a.L == l) e = cudaLaunchKernelEx(&cfg, k_sk_persist<w, l>, mapJ, mapD, maps, d, a);
    SG_PERSIST_KERNELS(SG_PERSIST_LAUNCH)
#undef SG_PERSIST_LAUNCH
    return e == cudaSuccess ? 2 : -1;
}

}  // namespace sg
