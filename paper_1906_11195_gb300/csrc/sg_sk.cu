// sg_sk.cu -- Sherrington-Kirkpatrick model, host side: validation, padding, threshold tables,
// tensor maps for the tensor-core field update, launch sequence and measurement bookkeeping.
//
// Eq. 1 with the binary couplings of SI section 1: J_ij = +-1 symmetric, J_ii = 0, energy scale
// 1/sqrt(N) folded into the acceptance table.  Spins are updated in the fixed order i = 0..N-1
// (SI section 1); the blocked kernel reproduces that order exactly (see sk_kernels.cu).
#include <cudaTypedefs.h>
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sg.h"
#include "sg_internal.cuh"
#include "sg_model.h"
#include "sk_internal.cuh"

namespace sg {

// One blocked sweep as the operations SkModel::sweep issues, in host issue order.  B < 128 (a
// row tile spans two blocks): in-block(b) then the update of every row by block b, on the
// handle's stream.  B >= 128: in-block(b) on the handle's stream folds block b - 1's flips into
// its own rows; the tensor-core update of every other row by block b (all rows for the last
// block, those of block b + 1 left to in-block(b + 1)) runs on the side stream, after in-block(b)
// (event b & 1 of "in-block done"), and in-block(b + 2), the first to need it, waits for it
// (event b & 1 of "side done"); the sweep ends by joining both.  The two branches write disjoint
// rows and the side stream runs its updates in order, so the integers are exact.
std::vector<SkSchedOp> sk_blocked_schedule(int n, int B, int Np) {
    std::vector<SkSchedOp> ops;
    const int ntiles = Np / 128;
    const int nblocks = (n + B - 1) / B;
    ops.push_back({kSchedKstar, 0, 0, 0, 0, 0});
    if (B < 128) {
        for (int b = 0; b < nblocks; ++b) {
            ops.push_back({kSchedInblock, 0, b, 0, 0, 0});
            ops.push_back({kSchedFieldAll, 0, b, 0, 0, 0});
        }
        return ops;
    }
    bool pending[2] = {false, false};
    for (int b = 0; b < nblocks; ++b) {
        const int b0 = b * B;
        if (pending[b & 1]) {
            ops.push_back({kSchedWait, 0, b, 0, 0, 2 + (b & 1)});
            pending[b & 1] = false;
        }
        ops.push_back({kSchedInblock, 0, b, 0, 0, 0});
        int skip0 = 0, skip1 = 0;
        if (b + 1 < nblocks) {
            skip0 = (b0 + B) / 128;
            skip1 = std::min(ntiles, (b0 + 2 * B) / 128);
        }
        ops.push_back({kSchedRecord, 0, b, 0, 0, b & 1});
        ops.push_back({kSchedWait, 1, b, 0, 0, b & 1});
        ops.push_back({kSchedFieldRows, 1, b, skip0, skip1, 0});
        ops.push_back({kSchedRecord, 1, b, 0, 0, 2 + (b & 1)});
        pending[b & 1] = true;
    }
    for (int k = 0; k < 2; ++k)
        if (pending[k]) ops.push_back({kSchedWait, 0, nblocks, 0, 0, 2 + k});
    return ops;
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        check_cuda(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q),
                   "cudaGetDriverEntryPointByVersion(cuTensorMapEncodeTiled)");
        if (q != cudaDriverEntryPointSuccess || !p) fail(SG_ECUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

void make_map_2d(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer,
                 uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle sw =
        box_inner == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    const CUresult r = get_encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base),
                                       dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(SG_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

// 2-D map of 32-bit words [outer][inner] (row stride inner * 4 bytes), no swizzle
void make_map_2d_u32(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer,
                     uint32_t box_inner, uint32_t box_outer) {
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * 4};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = get_encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(base),
                                       dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(SG_ECUDA, "cuTensorMapEncodeTiled (32-bit) failed (" + std::to_string((int)r) + ")");
}

// 2-D map of 16-bit words [outer][inner] (row stride inner * 2 bytes), no swizzle
void make_map_2d_u16(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer,
                     uint32_t box_inner, uint32_t box_outer) {
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * 2};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = get_encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(base),
                                       dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(SG_ECUDA, "cuTensorMapEncodeTiled (16-bit) failed (" + std::to_string((int)r) + ")");
}

class SkModel : public Model {
public:
    // prefer few CTAs per persistent launch (set before attach by a batch)
    void set_compact(bool c) { compact_ = c; }

    SkModel(int n, const int8_t* J, int n_replicas, const double* temps, uint64_t seed, int kernel,
            int block, const std::vector<int64_t>& tw_, const std::vector<int64_t>& tm_) {
        if (kernel != SG_SK_PLAIN && kernel != SG_SK_BLOCKED) fail(SG_EINVAL, "unknown SK kernel");
        if (n < 2 || n > 32768) fail(SG_EINVAL, "SK needs 2 <= n <= 32768");
        if (!J || !temps) fail(SG_EINVAL, "null array");
        if (n_replicas < 1) fail(SG_EINVAL, "n_replicas must be >= 1");
        kernel_ = kernel;
        n_ = n;
        R = n_replicas;
        L = 1;
        n_inst = 1;
        tw = tw_;
        tm = tm_;
        seed_ = seed;
        if (kernel == SG_SK_BLOCKED) {
            if (!(block == 0 || block == 64 || block == 128 || block == 256 || block == 512))
                fail(SG_EINVAL, "block must be 0 (autotune), 64, 128, 256 or 512");
            if (R % 16) fail(SG_EINVAL, "blocked SK needs a multiple of 16 replicas");
            if (R > 128 && R % 128) fail(SG_EINVAL, "more than 128 replicas must be a multiple of 128");
            autotune_ = block == 0;
            B_ = autotune_ ? 128 : block;
            kw_ = B_ >= 128 ? 128 : 64;
            NT_ = R <= 128 ? R : 128;
            // autotuning picks among 64, 128, 256 and (for n >= 2048, where the padding to a
            // multiple of 512 costs at most a quarter more) 512
            const int unit = autotune_ ? (n >= 2048 ? 512 : 256) : std::max(128, B_);
            Np_ = (n + unit - 1) / unit * unit;
        } else {
            Np_ = (n + 127) / 128 * 128;
            if (sk_plain_smem_bytes(Np_) > 200 * 1024) fail(SG_EINVAL, "n too large for the plain SK kernel");
        }
        // couplings
        const int words = Np_ / 32;
        h_J8_.assign((size_t)Np_ * Np_, 0);
        h_JbT_.assign((size_t)words * Np_, 0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const int8_t v = J[(size_t)i * n + j];
                if (i == j) {
                    if (v != 0) fail(SG_EINVAL, "J_ii must be 0");
                    continue;
                }
                if (v != 1 && v != -1) fail(SG_EINVAL, "off-diagonal J must be +-1");
                if (v != J[(size_t)j * n + i]) fail(SG_EINVAL, "J must be symmetric");
                h_J8_[(size_t)i * Np_ + j] = v > 0 ? 0x38 : 0xB8;
                if (v < 0) h_JbT_[(size_t)(j / 32) * Np_ + i] |= 1u << (j & 31);
            }
        // threshold tables, one per distinct temperature
        std::map<double, int> idx;
        for (int r = 0; r < R; ++r) {
            const double T = temps[r];
            if (!(T >= 0.0)) fail(SG_EINVAL, "temperature must be >= 0 (or +inf)");
            auto it = idx.find(T);
            if (it == idx.end()) {
                const int k0 = (int)idx.size();
                idx[T] = k0;
                const double beta = 1.0 / T;
                const size_t off = h_thr_.size();
                h_thr_.resize(off + n);
                h_thr_[off] = 0xFFFFFFFFu;
                for (int k = 1; k < n; ++k)
                    h_thr_[off + k] = metropolis_threshold(-(2.0 * beta * k) / sqrt((double)n));
                for (int k = 1; k < n; ++k)
                    if (h_thr_[off + k] > h_thr_[off + k - 1]) fail(SG_EINVAL, "threshold table not monotone");
                it = idx.find(T);
            }
            h_tidx_.push_back(it->second);
            h_coef_.push_back((float)(sqrt((double)n) * T / 2.0));
        }
        Carver c;
        carve(c);
        ws_bytes_ = c.off;
    }

    // computed once at construction: carving with a null base would reset the device views
    size_t workspace_bytes() const override { return ws_bytes_; }

    void attach(char* ws, cudaStream_t st) override {
        Carver c;
        c.base = ws;
        carve(c);
        auto up = [&](void* dst, const void* src, size_t bytes) {
            if (bytes) check_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st), "H2D copy");
            h2d_bytes += (int64_t)bytes;
        };
        up((void*)d_.JbT, h_JbT_.data(), h_JbT_.size() * 4);
        up((void*)d_.J8, h_J8_.data(), h_J8_.size());
        up((void*)d_.thr, h_thr_.data(), h_thr_.size() * 4);
        up((void*)d_.temp_index, h_tidx_.data(), h_tidx_.size() * 4);
        up((void*)d_.coef, h_coef_.data(), h_coef_.size() * 4);
        if (kernel_ == SG_SK_BLOCKED) {
            if (!side_) {
                check_cuda(cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking), "cudaStreamCreate");
                for (int k = 0; k < 2; ++k) {
                    check_cuda(cudaEventCreateWithFlags(&side_done_[k], cudaEventDisableTiming), "cudaEventCreate");
                    check_cuda(cudaEventCreateWithFlags(&inblock_done_[k], cudaEventDisableTiming), "cudaEventCreate");
                }
            }
            if (sk_inblock_prepare() != 0) fail(SG_ECUDA, "cannot raise the in-block kernel's shared memory limit");
            if (autotune_) tune_block(st);
            set_block(B_);
        } else {
            if (sk_plain_prepare(Np_) != 0) fail(SG_ECUDA, "cannot raise the plain kernel's shared memory limit");
        }
        init_state(st);
        check_cuda(cudaGetLastError(), "init launch");
        check_cuda(cudaStreamSynchronize(st), "attach");
        if (device_status(st)) fail(SG_ETIMEOUT, "device wait expired during initialisation");
    }

    ~SkModel() override {
        for (int k = 0; k < 2; ++k) {
            if (side_done_[k]) cudaEventDestroy(side_done_[k]);
            if (inblock_done_[k]) cudaEventDestroy(inblock_done_[k]);
        }
        if (side_) cudaStreamDestroy(side_);
    }

    void sweep(uint32_t t_off, cudaStream_t st) override {
        if (kernel_ == SG_SK_PLAIN) {
            launches += sk_plain_sweep(d_, clock_dev, t_off, st);
            return;
        }
        if (persist_) {
            sweep_many(t_off, 1, st);
            return;
        }
        // the schedule of one blocked sweep (sk_blocked_schedule), issued in order
        if (sched_B_ != B_) {
            sched_ = sk_blocked_schedule(n_, B_, Np_);
            sched_B_ = B_;
        }
        for (const SkSchedOp& o : sched_) {
            cudaStream_t os = o.stream ? side_ : st;
            const int b0 = o.block * B_;
            switch (o.op) {
                case kSchedKstar:
                    launches += sk_kstar_sweep(d_, clock_dev, t_off, os);
                    break;
                case kSchedInblock:
                {
                    // B >= 128: the in-block kernel also folds the previous block's flips
                    const bool fold = B_ >= 128 && o.block > 0;
                    if (sk_inblock(d_, b0, fold ? b0 - B_ : -1, B_, fold, os) < 0)
                        fail(SG_ECUDA, "in-block launch failed");
                }
                    ++launches;
                    break;
                case kSchedFieldAll:
                    launches += sk_field_update(d_, mapJ_, mapD_, b0, B_, kw_, NT_, 2, os);
                    break;
                case kSchedFieldRows:
                    launches += sk_field_update_rows(d_, mapJ_, mapD_, b0, B_, kw_, NT_, 2, o.skip0,
                                                     o.skip1, 0, os);
                    break;
                case kSchedRecord:
                    check_cuda(cudaEventRecord(o.event < 2 ? inblock_done_[o.event] : side_done_[o.event - 2], os),
                               "cudaEventRecord");
                    break;
                default:
                    check_cuda(cudaStreamWaitEvent(os, o.event < 2 ? inblock_done_[o.event] : side_done_[o.event - 2], 0),
                               "cudaStreamWaitEvent");
            }
        }
    }

    // persistent sweeps: one cooperative launch for all n (fields resident in tensor memory,
    // chains on their own CTAs, K* of each next sweep computed inside the launch)
    void sweep_many(uint32_t t_off, int n, cudaStream_t st) override {
        if (!persist_) {
            Model::sweep_many(t_off, n, st);
            return;
        }
        for (int done = 0; done < n;) {
            SkPersistArgs a = pa_;
            a.clock = clock_dev;
            a.t_off = t_off + (uint32_t)done;
            a.n_sweeps = std::min(n - done, kSkPersistMaxSweeps);
            const int k = sk_persist_sweeps(d_, a, mapJ_, mapDr_, pmaps_, st);
            if (k < 0) fail(SG_ECUDA, "persistent sweep launch failed");
            launches += k;
            done += a.n_sweeps;
        }
    }

    void snapshot(int w, cudaStream_t st) override { launches += sk_snapshot(d_, w, st); }

    // add the raw values at time tau into column u of arrays with ncol columns
    void measure_into(int64_t* Cb, int64_t* Qb, int64_t* Eb, int64_t ncol, int64_t u, int64_t tau,
                      cudaStream_t st) {
        const int64_t ntw = (int64_t)tw.size();
        int active = 0;
        while (active < (int)ntw && tw[active] <= tau) ++active;
        launches += sk_measure(d_, active, Cb + u, ntw * ncol, ncol, R >= 2 ? Qb + u : nullptr, ncol,
                               Eb + u, ncol, st);
    }

    void measure_scheduled(int u, int64_t tau, cudaStream_t st) override {
        measure_into(dC_, dQ_, dE_, (int64_t)tm.size(), u, tau, st);
    }

    void set_windows(int64_t nb) override {
        n_bins = nb;
        Carver c;
        carve(c);
        ws_bytes_ = c.off;
    }

    void measure_window(int m, int64_t tau, cudaStream_t st) override {
        measure_into(wC_, wQ_, wE_, n_bins, m, tau, st);
    }

    void read_windows(const int64_t* cnt_c, const int64_t* cnt_q, int64_t* C, int64_t* q,
                      int64_t* E, cudaStream_t st) override {
        std::vector<int64_t> c(nwC()), qq(nwQ()), e(nwE());
        down(c.data(), wC_, c.size() * 8, st);
        down(qq.data(), wQ_, qq.size() * 8, st);
        down(e.data(), wE_, e.size() * 8, st);
        check_cuda(cudaStreamSynchronize(st), "read windows");
        const int64_t ntw = (int64_t)tw.size(), nb = n_bins;
        for (int r = 0; r < R; ++r)
            for (int64_t m = 0; m < nb; ++m) {
                for (int64_t w = 0; w < ntw; ++w) {
                    const int64_t k = ((int64_t)r * ntw + w) * nb + m;
                    C[k] = cnt_c[w * nb + m] * n_ - 2 * c[k];
                }
                E[(int64_t)r * nb + m] = e[(int64_t)r * nb + m];
                if (r < R / 2) q[(int64_t)r * nb + m] = cnt_q[m] * n_ - 2 * qq[(int64_t)r * nb + m];
            }
    }

    void measure_now(int64_t tau, cudaStream_t st) override {
        const int64_t ntw = (int64_t)tw.size();
        int active = 0;
        while (active < (int)ntw && tw[active] <= tau) ++active;
        check_cuda(cudaMemsetAsync(mC_, 0, nmC() * 8, st), "memset");
        if (nmQ()) check_cuda(cudaMemsetAsync(mQ_, 0, nmQ() * 8, st), "memset");
        check_cuda(cudaMemsetAsync(mE_, 0, nmE() * 8, st), "memset");
        launches += sk_measure(d_, active, mC_, ntw, 1, R >= 2 ? mQ_ : nullptr, 1, mE_, 1, st);
    }

    void read_scheduled(int64_t tau, int64_t* C, int64_t* q, int64_t* E, cudaStream_t st) override {
        std::vector<int64_t> c(nC()), qq(nQ()), e(nE());
        down(c.data(), dC_, c.size() * 8, st);
        down(qq.data(), dQ_, qq.size() * 8, st);
        down(e.data(), dE_, e.size() * 8, st);
        check_cuda(cudaStreamSynchronize(st), "read results");
        const int64_t ntw = (int64_t)tw.size(), ntm = (int64_t)tm.size();
        for (int r = 0; r < R; ++r)
            for (int64_t u = 0; u < ntm; ++u) {
                const bool done = tm[u] <= tau;
                for (int64_t w = 0; w < ntw; ++w) {
                    const int64_t k = ((int64_t)r * ntw + w) * ntm + u;
                    C[k] = (done && tw[w] <= tm[u]) ? n_ - 2 * c[k] : 0;
                }
                E[(int64_t)r * ntm + u] = done ? e[(int64_t)r * ntm + u] : 0;
                if (r < R / 2) q[(int64_t)r * ntm + u] = done ? n_ - 2 * qq[(int64_t)r * ntm + u] : 0;
            }
    }

    void read_now(int64_t tau, int64_t* C, int64_t* q, int64_t* E, cudaStream_t st) override {
        std::vector<int64_t> c(nmC()), qq(nmQ()), e(nmE());
        down(c.data(), mC_, c.size() * 8, st);
        down(qq.data(), mQ_, qq.size() * 8, st);
        down(e.data(), mE_, e.size() * 8, st);
        check_cuda(cudaStreamSynchronize(st), "read measurement");
        const int64_t ntw = (int64_t)tw.size();
        for (int r = 0; r < R; ++r) {
            for (int64_t w = 0; w < ntw; ++w)
                C[r * ntw + w] = tw[w] <= tau ? n_ - 2 * c[r * ntw + w] : 0;
            E[r] = e[r];
            if (r < R / 2) q[r] = n_ - 2 * qq[r];
        }
    }

    size_t spins_bytes() const override { return (size_t)R * n_; }

    void get_spins(void* dst, cudaStream_t st) override {
        const int words = Np_ / 32;
        std::vector<uint32_t> S((size_t)R * words);
        down(S.data(), d_.S, S.size() * 4, st);
        check_cuda(cudaStreamSynchronize(st), "read spins");
        int8_t* out = static_cast<int8_t*>(dst);
        for (int r = 0; r < R; ++r)
            for (int i = 0; i < n_; ++i)
                out[(size_t)r * n_ + i] = ((S[(size_t)r * words + i / 32] >> (i & 31)) & 1u) ? -1 : 1;
    }

    std::vector<uint32_t> thresholds() const override {
        std::vector<uint32_t> t((size_t)R * n_);
        for (int r = 0; r < R; ++r)
            std::copy(h_thr_.begin() + (size_t)h_tidx_[r] * n_, h_thr_.begin() + (size_t)(h_tidx_[r] + 1) * n_,
                      t.begin() + (size_t)r * n_);
        return t;
    }

    std::vector<std::pair<void*, size_t>> state_regions() override {
        const size_t sw = (size_t)R * (Np_ / 32) * 4;
        return {{d_.S, sw}, {d_.H, (size_t)R * Np_ * 4}, {d_.snap, tw.size() * sw},
                {dC_, nC() * 8}, {dQ_, nQ() * 8}, {dE_, nE() * 8},
                {wC_, nwC() * 8}, {wQ_, nwQ() * 8}, {wE_, nwE() * 8}};
    }

    int device_status(cudaStream_t st) override {
        int v = 0;
        if (d_.err) {
            check_cuda(cudaMemcpyAsync(&v, d_.err, 4, cudaMemcpyDeviceToHost, st), "status copy");
            check_cuda(cudaStreamSynchronize(st), "status");
        }
        return v;
    }

private:
    size_t nC() const { return (size_t)R * tw.size() * tm.size(); }
    size_t nQ() const { return (size_t)(R / 2) * tm.size(); }
    size_t nE() const { return (size_t)R * tm.size(); }
    size_t nmC() const { return (size_t)R * tw.size(); }
    size_t nmQ() const { return (size_t)(R / 2); }
    size_t nmE() const { return (size_t)R; }
    size_t nwC() const { return (size_t)R * tw.size() * n_bins; }
    size_t nwQ() const { return (size_t)(R / 2) * n_bins; }
    size_t nwE() const { return (size_t)R * n_bins; }

    void down(void* dst, const void* src, size_t bytes, cudaStream_t st) {
        d2h_bytes += (int64_t)bytes;
        if (bytes) check_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st), "D2H copy");
    }

    void fields_direct(cudaStream_t st);

    // Persistent sweep (B = 128): field CTAs with TPC row tiles each in tensor memory, chain CTAs
    // of W replica warps; the smallest TPC and then W for which every CTA is resident.
    // SG_SK_PERSISTENT=0 keeps the launch-per-block sequence (results are the same);
    // SG_SK_LOOKAHEAD=<L> (4, 6 or 8; default 6, lowered below the number of blocks) sets the
    // blocks of flips folded on chip (L - 1 of them by the fold warps).
    bool plan_persist() {
        const char* e = getenv("SG_SK_PERSISTENT");
        if (e && e[0] == '0' && !e[1]) return false;
        if (R < 32 || R > 256 || R % 32 || Np_ % 128) return false;
        int dev = 0, sms = 0;
        check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
        check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
        int L = 6;
        if (const char* l = getenv("SG_SK_LOOKAHEAD")) L = atoi(l);
        if (!sk_persist_lookahead_supported(L)) return false;
        SkPersistArgs a = pa_;
        a.nb = Np_ / 128;
        // a fold window never holds a block twice: the largest compiled L below nb
        while (L >= a.nb && L > 0) L -= 2;
        if (L < 4) return false;  // the smallest compiled window (the staging needs L >= 2)
        a.L = L;
        a.n_sweeps = 1;
        a.Q = kPersistSlots;
        // alone: the smallest TPC and W whose CTAs all fit (the field work spread widest); in a
        // batch (compact_): the largest, so that more samples' launches run side by side
        const int Ws[2] = {compact_ ? 8 : 4, compact_ ? 4 : 8};
        const int TPCs[3] = {compact_ ? 4 : 1, 2, compact_ ? 1 : 4};
        for (int W : Ws) {
            if (R % W) continue;
            for (int TPC : TPCs) {
                if (TPC * R > 512) continue;
                a.W = W;
                a.nC = R / W;
                a.TPC = TPC;
                a.nG = (a.nb + TPC - 1) / TPC;
                for (int nst : {3, 2}) {
                    a.nst = nst;
                    if (sk_persist_fits(d_, a, sms)) {
                        pa_ = a;
                        make_map_2d(&mapDr_, pa_.Dring, 128, (uint64_t)kPersistSlots * R, 128, 128, R);
                        make_map_2d_u32(&pmaps_.jb, d_.JbT, Np_, Np_ / 32, 128, 4);
                        make_map_2d_u16(&pmaps_.kst, pa_.kst16, Np_, (uint64_t)kSkPersistMaxSweeps * R, 128, W);
                        make_map_2d_u32(&pmaps_.h, d_.H, Np_, R, 128, W);
                        make_map_2d_u32(&pmaps_.hpub, pa_.Hpub, Np_, R, 128, W);
                        return true;
                    }
                }
            }
        }
        return false;
    }

    void set_block(int B) {
        B_ = B;
        persist_ = false;
        kw_ = B >= 128 ? 128 : 64;
        // replica tile of the field GEMM: 64 columns for the short (K <= 128) updates, which
        // doubles the CTAs sharing each row tile's epilogue; 128 for the longer ones
        NT_ = R <= 64 ? R : (B <= 128 && R % 64 == 0 ? 64 : std::min(R, 128));
        if (sk_field_prepare(B_, kw_, NT_) != 0)
            fail(SG_ECUDA, "cannot raise the field kernel's shared memory limit");
        make_map_2d(&mapJ_, d_.J8, Np_, Np_, Np_, kw_, 128);
        make_map_2d(&mapD_, d_.D, Np_, R, Np_, kw_, NT_);
        if (B == 128) persist_ = plan_persist();
    }

    // tau = 0 state: initial spins, exact fields, zero counters (waits keep their full bound
    // here even in a test of the timeout path, which concerns the sweeps)
    void init_state(cudaStream_t st) {
        const int nowait = d_.test_nowait;
        d_.test_nowait = 0;
        check_cuda(cudaMemsetAsync(d_.H, 0, (size_t)R * Np_ * 4, st), "memset");
        check_cuda(cudaMemsetAsync(d_.err, 0, 4, st), "memset");
        check_cuda(cudaMemsetAsync(dC_, 0, nC() * 8, st), "memset");
        check_cuda(cudaMemsetAsync(dQ_, 0, nQ() * 8, st), "memset");
        check_cuda(cudaMemsetAsync(dE_, 0, nE() * 8, st), "memset");
        if (n_bins) {
            check_cuda(cudaMemsetAsync(wC_, 0, nwC() * 8, st), "memset");
            check_cuda(cudaMemsetAsync(wQ_, 0, nwQ() * 8, st), "memset");
            check_cuda(cudaMemsetAsync(wE_, 0, nwE() * 8, st), "memset");
        }
        launches += sk_init(d_, st);
        if (kernel_ == SG_SK_BLOCKED) {
            // initial fields h = J s, one block of columns at a time (D holds s)
            for (int b0 = 0; b0 < Np_; b0 += B_)
                launches += sk_field_update(d_, mapJ_, mapD_, b0, B_, kw_, NT_, 1, st);
        } else {
            fields_direct(st);  // h = J s on CUDA cores
        }
        d_.test_nowait = nowait;
    }

    // Autotuner: time two sweeps with each block size that divides Np and keep the fastest.
    // The trial sweeps run from a fresh state which init_state() then rebuilds, so the choice
    // never changes the trajectory (every block size gives the same integers).
    void tune_block(cudaStream_t st) {
        cudaEvent_t e0, e1;
        check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
        check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
        float best_ms = 0.f;
        int best = 128;
        for (int B : {64, 128, 256, 512}) {
            if (Np_ % B) continue;
            set_block(B);
            init_state(st);
            check_cuda(cudaMemsetAsync(clock_dev, 0, 4, st), "memset");
            sweep(0, st);  // warm-up
            check_cuda(cudaEventRecord(e0, st), "cudaEventRecord");
            sweep_many(1, 2, st);  // as the replayed graphs run them
            check_cuda(cudaEventRecord(e1, st), "cudaEventRecord");
            check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
            float ms = 0.f;
            check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
            if (best_ms == 0.f || ms < best_ms) {
                best_ms = ms;
                best = B;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        B_ = best;
    }

    void carve(Carver& c) {
        const int words = Np_ / 32;
        clock_dev = c.take<uint32_t>(1);
        d_.JbT = c.take<uint32_t>(h_JbT_.size());
        d_.J8 = c.take<uint8_t>(h_J8_.size());
        d_.thr = c.take<uint32_t>(h_thr_.size());
        d_.temp_index = c.take<int32_t>(h_tidx_.size());
        d_.coef = c.take<float>(h_coef_.size());
        d_.S = c.take<uint32_t>((size_t)R * words);
        d_.D = c.take<uint8_t>((size_t)R * Np_);
        d_.H = c.take<int32_t>((size_t)R * Np_);
        d_.kst = c.take<int32_t>(kernel_ == SG_SK_BLOCKED ? (size_t)R * Np_ : 0);
        d_.flips = c.take<uint32_t>(kernel_ == SG_SK_BLOCKED ? (size_t)R * words : 0);
        d_.snap = c.take<uint32_t>((size_t)R * words * tw.size());
        d_.err = c.take<int>(1);
        // persistent sweep: spin-change ring, published fields, counters
        const bool blk = kernel_ == SG_SK_BLOCKED;
        pa_.Dring = c.take<uint8_t>(blk ? (size_t)kPersistSlots * R * 128 : 0);
        pa_.Hpub = c.take<int32_t>(blk ? (size_t)R * Np_ : 0);
        pa_.sync = c.take<uint32_t>(blk ? (size_t)(2 * kPersistSlots + Np_ / 128) : 0);
        pa_.kst16 = c.take<int16_t>(blk ? (size_t)kSkPersistMaxSweeps * R * Np_ : 0);
        d_.seed = seed_;
        d_.N = n_;
        d_.Np = Np_;
        d_.R = R;
        // replica warps per in-block CTA: 4 spreads the replicas over twice the SMs of 8 and
        // measured faster (the per-replica decision chain has fewer warps beside it on each
        // scheduler); SG_SK_INBLOCK_WARPS = 2, 4 or 8 pins a split (results never change)
        {
            const char* e = getenv("SG_SK_INBLOCK_WARPS");
            const int v = e ? atoi(e) : 4;
            d_.inblock_warps = (v == 2 || v == 4 || v == 8) ? v : 4;
        }
        // SG_TEST_STAGE_WAIT_NS=0 (tests of the timeout path only) turns every bounded device
        // wait of a sweep into a single test, so that a wait gives up without a GPU fault
        {
            const char* w = getenv("SG_TEST_STAGE_WAIT_NS");
            d_.test_nowait = (w && strtoull(w, nullptr, 10) == 0) ? 1 : 0;
        }
        dC_ = c.take<int64_t>(nC());
        dQ_ = c.take<int64_t>(nQ());
        dE_ = c.take<int64_t>(nE());
        mC_ = c.take<int64_t>(nmC());
        mQ_ = c.take<int64_t>(nmQ());
        mE_ = c.take<int64_t>(nmE());
        wC_ = c.take<int64_t>(nwC());
        wQ_ = c.take<int64_t>(nwQ());
        wE_ = c.take<int64_t>(nwE());
    }

    static constexpr int kPersistSlots = kSkPersistSlots;  // spin-change ring slots
    int kernel_ = SG_SK_BLOCKED;
    bool autotune_ = false;
    bool compact_ = false;
    bool persist_ = false;   // B = 128 sweeps run as one persistent launch
    SkPersistArgs pa_{};
    CUtensorMap mapDr_{};
    SkPersistMaps pmaps_{};
    size_t ws_bytes_ = 0;
    cudaStream_t side_ = nullptr;                      // branch for the off-critical-path update
    std::vector<SkSchedOp> sched_;                     // the blocked sweep's schedule for sched_B_
    int sched_B_ = 0;
    cudaEvent_t side_done_[2] = {}, inblock_done_[2] = {};
    int n_ = 0, Np_ = 0, B_ = 128, kw_ = 128, NT_ = 128;
    uint64_t seed_ = 0;
    pinned_vector<uint8_t> h_J8_;   // the large images copied at attach: page-locked
    pinned_vector<uint32_t> h_JbT_;
    std::vector<uint32_t> h_thr_;
    std::vector<int32_t> h_tidx_;
    std::vector<float> h_coef_;
    SkDev d_{};
    CUtensorMap mapJ_{}, mapD_{};
    int64_t *dC_ = nullptr, *dQ_ = nullptr, *dE_ = nullptr;
    int64_t *mC_ = nullptr, *mQ_ = nullptr, *mE_ = nullptr;
    int64_t *wC_ = nullptr, *wQ_ = nullptr, *wE_ = nullptr;  // window sums
};

// h_i = sum_j J_ij s_j on CUDA cores (initial fields of the plain path)
__global__ void k_sk_fields_direct(SkDev d) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.Np) return;
    const int words = d.Np / 32;
    const uint32_t* S = d.S + (int64_t)r * words;
    const uint8_t* row = d.J8 + (int64_t)i * d.Np;
    int acc = 0;
    for (int j = 0; j < d.N; ++j) {
        const uint8_t b = row[j];
        const int J = b == 0x38 ? 1 : (b == 0xB8 ? -1 : 0);
        const int s = ((S[j >> 5] >> (j & 31)) & 1u) ? -1 : 1;
        acc += J * s;
    }
    d.H[(int64_t)r * d.Np + i] = acc;
}

void SkModel::fields_direct(cudaStream_t st) {
    dim3 grid((unsigned)((Np_ + 127) / 128), (unsigned)R);
    k_sk_fields_direct<<<grid, 128, 0, st>>>(d_);
    ++launches;
}

// A batch of independent SK samples (uneven N) advancing in lock-step.  Each sweep forks one
// branch per sample onto its own stream and joins them, so that under stream capture a sweep
// becomes one CUDA graph whose branches run concurrently.
class SkBatchModel : public Model {
public:
    SkBatchModel(const sg_sk_sample* samples, int n_samples, int n_replicas, int kernel, int block,
                 const std::vector<int64_t>& tw_, const std::vector<int64_t>& tm_) {
        if (!samples || n_samples < 1) fail(SG_EINVAL, "need at least one sample");
        n_inst = n_samples;
        R = n_replicas;
        L = 1;
        tw = tw_;
        tm = tm_;
        for (int b = 0; b < n_samples; ++b) {
            const sg_sk_sample& x = samples[b];
            try {
                subs_.emplace_back(new SkModel(x.n, x.J, n_replicas, x.temps, x.seed, kernel, block, tw, tm));
                // the samples' persistent launches share the GPU: few CTAs each
                // (SG_SK_BATCH_COMPACT=0: each as if alone; the results are the same)
                const char* c = getenv("SG_SK_BATCH_COMPACT");
                subs_.back()->set_compact(!(c && c[0] == '0' && !c[1]));
            } catch (const Error& e) {
                fail(e.code, "sample " + std::to_string(b) + ": " + e.msg);
            }
        }
    }

    ~SkBatchModel() override {
        for (auto& e : events_) cudaEventDestroy(e);
        if (fork_) cudaEventDestroy(fork_);
        for (auto& st : streams_) cudaStreamDestroy(st);
    }

    size_t workspace_bytes() const override {
        size_t off = 256;  // batch clock
        for (auto& m : subs_) off = ((off + 255) & ~size_t(255)) + m->workspace_bytes();
        return off;
    }

    void attach(char* ws, cudaStream_t st) override {
        clock_dev = reinterpret_cast<uint32_t*>(ws);
        size_t off = 256;
        for (auto& m : subs_) {
            off = (off + 255) & ~size_t(255);
            m->attach(ws + off, st);
            off += m->workspace_bytes();
            launches += m->launches;
            m->launches = 0;
            m->clock_dev = clock_dev;  // every sample reads the batch clock
        }
        check_cuda(cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming), "cudaEventCreate");
        for (size_t b = 0; b < subs_.size(); ++b) {
            cudaStream_t s2;
            cudaEvent_t e;
            check_cuda(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking), "cudaStreamCreate");
            streams_.push_back(s2);
            check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
            events_.push_back(e);
        }
    }

    void sweep(uint32_t t_off, cudaStream_t st) override { sweep_many(t_off, 1, st); }

    // every sample's n sweeps on its own branch, joined once
    void sweep_many(uint32_t t_off, int n, cudaStream_t st) override {
        check_cuda(cudaEventRecord(fork_, st), "cudaEventRecord");
        for (size_t b = 0; b < subs_.size(); ++b) {
            check_cuda(cudaStreamWaitEvent(streams_[b], fork_, 0), "cudaStreamWaitEvent");
            subs_[b]->sweep_many(t_off, n, streams_[b]);
            check_cuda(cudaEventRecord(events_[b], streams_[b]), "cudaEventRecord");
        }
        for (size_t b = 0; b < subs_.size(); ++b)
            check_cuda(cudaStreamWaitEvent(st, events_[b], 0), "cudaStreamWaitEvent");
        collect();
    }

    void snapshot(int w, cudaStream_t st) override {
        for (auto& m : subs_) m->snapshot(w, st);
        collect();
    }

    void measure_scheduled(int u, int64_t tau, cudaStream_t st) override {
        for (auto& m : subs_) m->measure_scheduled(u, tau, st);
        collect();
    }

    void measure_now(int64_t tau, cudaStream_t st) override {
        for (auto& m : subs_) m->measure_now(tau, st);
        collect();
    }

    void set_windows(int64_t nb) override {
        n_bins = nb;
        for (auto& m : subs_) m->set_windows(nb);
    }

    void set_schedule(const std::vector<int64_t>& tw_, const std::vector<int64_t>& tm_,
                      bool attached) override {
        tw = tw_;
        tm = tm_;
        for (auto& m : subs_) m->set_schedule(tw_, tm_, attached);
    }

    void measure_window(int mw, int64_t tau, cudaStream_t st) override {
        for (auto& m : subs_) m->measure_window(mw, tau, st);
        collect();
    }

    void read_windows(const int64_t* cnt_c, const int64_t* cnt_q, int64_t* C, int64_t* q,
                      int64_t* E, cudaStream_t st) override {
        const size_t nc = (size_t)R * tw.size() * n_bins, nq = (size_t)(R / 2) * n_bins,
                     ne = (size_t)R * n_bins;
        for (size_t b = 0; b < subs_.size(); ++b)
            subs_[b]->read_windows(cnt_c, cnt_q, C + b * nc, q + b * nq, E + b * ne, st);
    }

    void read_scheduled(int64_t tau, int64_t* C, int64_t* q, int64_t* E, cudaStream_t st) override {
        const size_t nc = (size_t)R * tw.size() * tm.size(), nq = (size_t)(R / 2) * tm.size(),
                     ne = (size_t)R * tm.size();
        for (size_t b = 0; b < subs_.size(); ++b)
            subs_[b]->read_scheduled(tau, C + b * nc, q + b * nq, E + b * ne, st);
    }

    void read_now(int64_t tau, int64_t* C, int64_t* q, int64_t* E, cudaStream_t st) override {
        const size_t nc = (size_t)R * tw.size(), nq = (size_t)(R / 2), ne = (size_t)R;
        for (size_t b = 0; b < subs_.size(); ++b)
            subs_[b]->read_now(tau, C + b * nc, q + b * nq, E + b * ne, st);
    }

    size_t spins_bytes() const override {
        size_t t = 0;
        for (auto& m : subs_) t += m->spins_bytes();
        return t;
    }

    void get_spins(void* dst, cudaStream_t st) override {
        char* p = static_cast<char*>(dst);
        for (auto& m : subs_) {
            m->get_spins(p, st);
            p += m->spins_bytes();
        }
    }

    std::vector<uint32_t> thresholds() const override {
        std::vector<uint32_t> t;
        for (auto& m : subs_) {
            auto x = m->thresholds();
            t.insert(t.end(), x.begin(), x.end());
        }
        return t;
    }

    std::vector<std::pair<void*, size_t>> state_regions() override {
        std::vector<std::pair<void*, size_t>> v;
        for (auto& m : subs_) {
            auto x = m->state_regions();
            v.insert(v.end(), x.begin(), x.end());
        }
        return v;
    }

    int device_status(cudaStream_t st) override {
        int v = 0;
        for (auto& m : subs_) v |= m->device_status(st);
        return v;
    }

private:
    void collect() {
        for (auto& m : subs_) {
            launches += m->launches;
            m->launches = 0;
        }
    }

    void transfer_bytes(int64_t& h2d, int64_t& d2h) const override {
        h2d = h2d_bytes;
        d2h = d2h_bytes;
        for (auto& m : subs_) {
            h2d += m->h2d_bytes;
            d2h += m->d2h_bytes;
        }
    }

    std::vector<std::unique_ptr<SkModel>> subs_;
    std::vector<cudaStream_t> streams_;
    std::vector<cudaEvent_t> events_;
    cudaEvent_t fork_ = nullptr;
};

}  // namespace

Model* make_sk_batch_model(const void* samples, int n_samples, int n_replicas, int kernel,
                           int block, const std::vector<int64_t>& tw,
                           const std::vector<int64_t>& tm) {
    return new SkBatchModel(static_cast<const sg_sk_sample*>(samples), n_samples, n_replicas,
                            kernel, block, tw, tm);
}

Model* make_sk_model(int n, const int8_t* J, int n_replicas, const double* temps, uint64_t seed,
                     int kernel, int block, const std::vector<int64_t>& tw,
                     const std::vector<int64_t>& tm) {
    return new SkModel(n, J, n_replicas, temps, seed, kernel, block, tw, tm);
}

}  // namespace sg

// the blocked sweep's schedule, for host-side checks (no device needed)
extern "C" int sg_sk_blocked_schedule(int32_t n, int32_t block, int32_t* ops, int32_t cap,
                                      int32_t* n_ops) {
    if (!n_ops || (cap > 0 && !ops)) {
        sg::record_error("null argument");
        return SG_EINVAL;
    }
    if (n < 2 || n > 32768 || !(block == 64 || block == 128 || block == 256 || block == 512)) {
        sg::record_error("need 2 <= n <= 32768 and block 64, 128, 256 or 512");
        return SG_EINVAL;
    }
    const int unit = std::max(128, (int)block);
    const int Np = (n + unit - 1) / unit * unit;
    const std::vector<sg::SkSchedOp> sched = sg::sk_blocked_schedule(n, block, Np);
    *n_ops = (int32_t)sched.size();
    if ((int64_t)sched.size() > (int64_t)cap) {
        sg::record_error("ops capacity " + std::to_string(cap) + " < " + std::to_string(sched.size()));
        return SG_EINVAL;
    }
    for (size_t i = 0; i < sched.size(); ++i) {
        const sg::SkSchedOp& o = sched[i];
        const int32_t v[6] = {o.op, o.stream, o.block, o.skip0, o.skip1, o.event};
        for (int k = 0; k < 6; ++k) ops[6 * i + k] = v[k];
    }
    return SG_OK;
}
