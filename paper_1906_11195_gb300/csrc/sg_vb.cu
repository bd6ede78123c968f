// sg_vb.cu -- Viana-Bray model, host side: validation, greedy colouring, device layouts
// (plain colour-major CSR and packed sliced-ELL), measurement bookkeeping.
//
// Update order: the vertices of a graph are coloured greedily in vertex order (each vertex gets
// the smallest colour not used by an already-coloured neighbour), then greedily once more in the
// order of decreasing colour (increasing label inside a colour); a sweep updates colour class
// 0, then 1, ...  Each class is an independent set, so its vertices can be updated in parallel;
// this generalises the bipartite half-updates of SI section 3 to the Poissonian graphs of the
// Viana-Bray ensemble (Eq. 3).  The random number of a vertex is keyed by its original label,
// so relabelling and slicing never change the trajectory.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/sg.h"
#include "sg_internal.cuh"
#include "sg_model.h"

namespace sg {
namespace {

struct Graph {
    int32_t n = 0;
    int64_t edges = 0;  // undirected
    std::vector<int32_t> row_ptr, col;
    std::vector<uint64_t> jb;
    std::vector<int32_t> colour;
    int n_colours = 0;
    uint64_t seed = 0;
    std::vector<double> temps;
};

void load_graph(const sg_vb_graph& in, int R, int idx, Graph& g) {
    const std::string tag = "graph " + std::to_string(idx) + ": ";
    if (in.n < 2 || in.n > SG_VB_MAX_N) fail(SG_EINVAL, tag + "n out of range");
    if (!in.row_ptr || !in.col || !in.jbits || !in.temps) fail(SG_EINVAL, tag + "null array");
    const int32_t n = in.n;
    if (in.row_ptr[0] != 0) fail(SG_EINVAL, tag + "row_ptr[0] != 0");
    for (int32_t i = 0; i < n; ++i) {
        const int32_t d = in.row_ptr[i + 1] - in.row_ptr[i];
        if (d < 0) fail(SG_EINVAL, tag + "row_ptr not monotone");
        if (d > SG_VB_MAX_DEGREE) fail(SG_EINVAL, tag + "degree above " + std::to_string(SG_VB_MAX_DEGREE));
    }
    const int64_t nnz = in.row_ptr[n];
    if (nnz % 2) fail(SG_EINVAL, tag + "odd number of directed entries (not symmetric)");
    g.n = n;
    g.edges = nnz / 2;
    g.row_ptr.assign(in.row_ptr, in.row_ptr + n + 1);
    g.col.assign(in.col, in.col + nnz);
    g.jb.assign(in.jbits, in.jbits + nnz);
    // sorted copy of every row for the structural checks
    std::vector<std::pair<int32_t, uint64_t>> srt(nnz);
    for (int64_t e = 0; e < nnz; ++e) {
        if (g.col[e] < 0 || g.col[e] >= n) fail(SG_EINVAL, tag + "neighbour index out of range");
        srt[e] = {g.col[e], g.jb[e]};
    }
    for (int32_t i = 0; i < n; ++i) {
        auto b = srt.begin() + g.row_ptr[i], e = srt.begin() + g.row_ptr[i + 1];
        std::sort(b, e);
        for (auto it = b; it != e; ++it) {
            if (it->first == i) fail(SG_EINVAL, tag + "self-loop at vertex " + std::to_string(i));
            if (it + 1 != e && (it + 1)->first == it->first)
                fail(SG_EINVAL, tag + "duplicate edge at vertex " + std::to_string(i));
        }
    }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e) {
            const int32_t j = srt[e].first;
            auto b = srt.begin() + g.row_ptr[j], en = srt.begin() + g.row_ptr[j + 1];
            auto it = std::lower_bound(b, en, std::make_pair(i, (uint64_t)0),
                                       [](const std::pair<int32_t, uint64_t>& a,
                                          const std::pair<int32_t, uint64_t>& c) {
                                           return a.first < c.first;
                                       });
            if (it == en || it->first != i)
                fail(SG_EINVAL, tag + "edge (" + std::to_string(i) + "," + std::to_string(j) +
                                    ") has no reverse entry");
            if (it->second != srt[e].second)
                fail(SG_EINVAL, tag + "couplings of edge (" + std::to_string(i) + "," +
                                    std::to_string(j) + ") differ between directions");
        }
    g.temps.assign(in.temps, in.temps + R);
    for (double T : g.temps)
        if (!(T >= 0.0)) fail(SG_EINVAL, tag + "temperature must be >= 0 (or +inf)");
    g.seed = in.seed;
    // greedy colouring in vertex order
    g.colour.assign(n, -1);
    std::vector<char> used(SG_VB_MAX_DEGREE + 2, 0);
    int nc = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e) {
            const int c = g.colour[g.col[e]];
            if (c >= 0) used[c] = 1;
        }
        int c = 0;
        while (used[c]) ++c;
        g.colour[i] = c;
        nc = std::max(nc, c + 1);
        for (int32_t e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e) {
            const int cj = g.colour[g.col[e]];
            if (cj >= 0) used[cj] = 0;
        }
    }
    // one recolouring pass: greedy again, visiting the classes from the last to the first
    // (vertex order inside a class).  Each old class is an independent set, so no colour is
    // added, and the thin last classes of the first pass are folded into the others.
    std::vector<int32_t> start(nc + 1, 0), order(n);
    for (int32_t i = 0; i < n; ++i) ++start[nc - g.colour[i]];
    for (int c = 0; c < nc; ++c) start[c + 1] += start[c];
    for (int32_t i = 0; i < n; ++i) order[start[nc - 1 - g.colour[i]]++] = i;
    std::vector<int32_t> fresh(n, -1);
    int nc2 = 0;
    for (int32_t i : order) {
        for (int32_t e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e) {
            const int c = fresh[g.col[e]];
            if (c >= 0) used[c] = 1;
        }
        int c = 0;
        while (used[c]) ++c;
        fresh[i] = c;
        nc2 = std::max(nc2, c + 1);
        for (int32_t e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e) {
            const int cj = fresh[g.col[e]];
            if (cj >= 0) used[cj] = 0;
        }
    }
    g.colour.swap(fresh);
    g.n_colours = nc2;
}

// Validate and colour every graph of a batch, one graph per task on the host's cores (the
// graphs are independent; a batch of hundreds of uneven graphs is mostly this work).  The first
// failing graph's error, in graph order, is raised after all tasks have ended.
void load_graphs(const sg_vb_graph* in, int n_graphs, int R, std::vector<Graph>& out) {
    out.resize(n_graphs);
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nt = (int)std::min<unsigned>(hw, (unsigned)n_graphs);
    std::vector<std::unique_ptr<Error>> errs(n_graphs);
    std::atomic<int> next{0};
    auto work = [&] {
        for (;;) {
            const int b = next.fetch_add(1);
            if (b >= n_graphs) return;
            try {
                load_graph(in[b], R, b, out[b]);
            } catch (const Error& e) {
                errs[b].reset(new Error(e));
            } catch (const std::bad_alloc&) {
                errs[b].reset(new Error{SG_ENOMEM, "host allocation failed"});
            }
        }
    };
    if (nt <= 1) {
        work();
    } else {
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t) pool.emplace_back(work);
        for (auto& th : pool) th.join();
    }
    for (auto& e : errs)
        if (e) throw *e;
}

// Run f(lo, hi) over [0, n) cut into contiguous ranges, one per host thread (f must only write
// what its own range owns).
template <class F>
void parallel_ranges(int64_t n, F&& f) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t nt = std::min<int64_t>((int64_t)hw, std::max<int64_t>(1, n / 4096));
    if (nt <= 1) {
        f((int64_t)0, n);
        return;
    }
    std::vector<std::thread> pool;
    for (int64_t t = 0; t < nt; ++t) pool.emplace_back([&, t] { f(n * t / nt, n * (t + 1) / nt); });
    for (auto& th : pool) th.join();
}

std::vector<uint32_t> vb_table(double T) {
    std::vector<uint32_t> t(kVbThrStride);
    const double beta = 1.0 / T;
    t[0] = 0xFFFFFFFFu;
    for (int m = 1; m < kVbThrStride; ++m) t[m] = metropolis_threshold(-2.0 * beta * m);
    return t;
}

class VbModel : public Model {
public:
    VbModel(const sg_vb_graph* graphs, int n_graphs, int n_lanes, int n_replicas, int kernel,
            const std::vector<int64_t>& tw_, const std::vector<int64_t>& tm_) {
        if (kernel != SG_VB_PLAIN && kernel != SG_VB_PACKED) fail(SG_EINVAL, "unknown VB kernel");
        if (n_lanes < 1 || n_lanes > 64) fail(SG_EINVAL, "n_lanes must be 1..64");
        if (n_replicas < 1) fail(SG_EINVAL, "n_replicas must be >= 1");
        if (kernel == SG_VB_PACKED && !(n_replicas == 1 || n_replicas == 2 || n_replicas == 4))
            fail(SG_EINVAL, "packed kernel supports 1, 2 or 4 replicas");
        if (kernel == SG_VB_PLAIN && n_graphs != 1) fail(SG_EINVAL, "plain kernel takes one graph");
        kernel_ = kernel;
        n_inst = n_graphs;
        R = n_replicas;
        L = n_lanes;
        Lc_ = kernel == SG_VB_PACKED ? 64 : L;
        tw = tw_;
        tm = tm_;
        load_graphs(graphs, n_graphs, R, graphs_);
        for (const Graph& g : graphs_)
            for (int r = 0; r < R; ++r) {
                auto t = vb_table(g.temps[r]);
                for (int m = 1; m < kVbThrStride; ++m)
                    if (t[m] > t[m - 1]) fail(SG_EINVAL, "threshold table not monotone");
                thr_.insert(thr_.end(), t.begin(), t.end());
            }
        if (kernel == SG_VB_PACKED) build_packed();
        else build_plain();
        // the energy of a measured state taken by the next sweep (one instance, packed);
        // SG_VB_FUSED_MEAS=0 keeps the standalone energy kernel (the results are the same)
        const char* fm = getenv("SG_VB_FUSED_MEAS");
        fuse_e_ = kernel == SG_VB_PACKED && n_graphs == 1 && !(fm && fm[0] == '0' && !fm[1]);
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
        up((void*)d_thr_, thr_.data(), thr_.size() * 4);
        if (kernel_ == SG_VB_PACKED) {
            up((void*)pk_.vinfo, h_vinfo_.data(), h_vinfo_.size() * 4);
            up((void*)pk_.slice_base, h_slice_base_.data(), h_slice_base_.size() * 4);
            up((void*)pk_.slice_graph, h_slice_graph_.data(), h_slice_graph_.size() * 4);
            up((void*)pk_.col, h_col_.data(), h_col_.size() * 4);
            up((void*)pk_.groups, h_groups_.data(), h_groups_.size() * sizeof(uint4));
            up((void*)pk_.slice_meta, h_slice_meta_.data(), h_slice_meta_.size() * sizeof(uint4));
            up((void*)pk_.group_graph, h_group_graph_.data(), h_group_graph_.size() * 4);
            up((void*)pk_.gtab, h_gtab_.data(), h_gtab_.size());
            check_cuda(cudaMemsetAsync(pk_.err, 0, 4, st), "memset");
            up((void*)pk_.colour_groups, colour_group_.data(), colour_group_.size() * 4);
            check_cuda(cudaMemsetAsync(pk_.gbar, 0, 8, st), "memset");
            up((void*)pk_.jb, h_jb_.data(), h_jb_.size() * 8);
            std::vector<uint64_t> seeds(n_inst);
            for (int b = 0; b < n_inst; ++b) seeds[b] = graphs_[b].seed;
            up((void*)pk_.seeds, seeds.data(), seeds.size() * 8);
            up((void*)pk_.up_slice_base, h_up_base_.data(), h_up_base_.size() * 4);
            launches += vb_packed_build_upper(pk_, st);  // from col and jb, on the device
            launches += vb_packed_init(pk_, st);
            // SG_VB_COLOUR_VARIANT=<k> and SG_VB_FUSED=<0|1> pin the pipeline shape and the
            // launch form (reproducible timings of one choice); otherwise the autotuner picks
            const char* pin = getenv("SG_VB_COLOUR_VARIANT");
            const char* pin_f = getenv("SG_VB_FUSED");
            const bool pinned = pin && *pin >= '0' && *pin < '0' + kVbColourVariants && !pin[1];
            const bool pinned_f = pin_f && (*pin_f == '0' || *pin_f == '1') && !pin_f[1];
            if (pinned && pinned_f) {
                variant_ = *pin - '0';
                fused_ = *pin_f == '1';
            } else if (!pinned && !pinned_f && tuned_before()) {
                // an instance of the same layout was tuned in this process: its choice holds
            } else {
                tune_variant(st, pinned ? *pin - '0' : -1, pinned_f ? *pin_f - '0' : -1);
                if (!pinned && !pinned_f) remember_tuning();
            }
            if (fuse_e_) {
                // one measuring sweep (into the scratch energy counts of sg_measure, cleared
                // before each use) sets its kernel up before the first measurement; the initial
                // spins are drawn again afterwards
                check_cuda(cudaMemsetAsync(clock_dev, 0, 4, st), "memset");
                const VbSweepMeas m{mE_, (int64_t)Lc_, 1};
                const int n = vb_packed_sweep_meas(pk_, colour_group_.data(), clock_dev, 0, variant_,
                                                   fused_, m, st);
                if (n < 0) fail(SG_ECUDA, "measuring colour kernel launch failed");
                launches += n + vb_packed_init(pk_, st);
            }
        } else {
            up((void*)pl_.row_ptr, h_row_ptr_.data(), h_row_ptr_.size() * 4);
            up((void*)pl_.col, h_col_i_.data(), h_col_i_.size() * 4);
            up((void*)pl_.jb, h_jb_.data(), h_jb_.size() * 8);
            up((void*)pl_.orig, h_orig_.data(), h_orig_.size() * 4);
            launches += vb_plain_init(pl_, st);
        }
        check_cuda(cudaMemsetAsync(dC_, 0, nC() * 8, st), "memset");
        check_cuda(cudaMemsetAsync(dQ_, 0, nQ() * 8, st), "memset");
        check_cuda(cudaMemsetAsync(dE_, 0, nE() * 8, st), "memset");
        if (n_bins) {
            check_cuda(cudaMemsetAsync(wC_, 0, nwC() * 8, st), "memset");
            check_cuda(cudaMemsetAsync(wQ_, 0, nwQ() * 8, st), "memset");
            check_cuda(cudaMemsetAsync(wE_, 0, nwE() * 8, st), "memset");
        }
        check_cuda(cudaGetLastError(), "init launch");
        check_cuda(cudaStreamSynchronize(st), "attach");
    }

    // The autotuner's choice per layout shape (slots, entries, colour classes, groups, replicas,
    // device), kept for the process: the timings depend on nothing else.
    using TuneKey = std::vector<int64_t>;
    static std::mutex& tune_mutex() {
        static std::mutex m;
        return m;
    }
    static std::map<TuneKey, std::pair<int, bool>>& tune_cache() {
        static std::map<TuneKey, std::pair<int, bool>> c;
        return c;
    }
    TuneKey tune_key() const {
        int dev = 0;
        cudaGetDevice(&dev);
        TuneKey k{dev, n_slots_, (int64_t)h_col_.size(), (int64_t)colour_group_.size(),
                  (int64_t)h_groups_.size(), R, n_inst};
        k.insert(k.end(), colour_group_.begin(), colour_group_.end());
        return k;
    }
    bool tuned_before() {
        std::lock_guard<std::mutex> g(tune_mutex());
        auto it = tune_cache().find(tune_key());
        if (it == tune_cache().end()) return false;
        variant_ = it->second.first;
        fused_ = it->second.second;
        return true;
    }
    void remember_tuning() {
        std::lock_guard<std::mutex> g(tune_mutex());
        tune_cache()[tune_key()] = {variant_, fused_};
    }

    // Autotuner: time two sweeps with each pipeline shape of the colour kernel, launched per
    // colour class and (R = 2, 4) fused into one cooperative launch per sweep, and keep the
    // fastest; then redraw the initial spins (the trial sweeps leave no trace: the initial
    // configuration is a pure function of the seed, and no measurement was taken).  A choice
    // whose launch is refused (e.g. a cooperative grid that cannot be resident) is skipped.
    // only_v / only_f >= 0 restrict the search to one shape / launch form.
    void tune_variant(cudaStream_t st, int only_v, int only_f) {
        cudaEvent_t e0, e1;
        check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
        check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
        float best = 0.f;
        int best_v = -1;
        bool best_f = false;
        const bool can_fuse = R != 1 && colour_group_.size() > 2;
        if (!can_fuse) only_f = -1;  // a fused request runs per class (as the sweep does)
        for (int f = 0; f < (can_fuse ? 2 : 1); ++f) {
            if (only_f >= 0 && f != only_f) continue;
            for (int v = 0; v < kVbColourVariants; ++v) {
                if (only_v >= 0 && v != only_v) continue;
                variant_ = v;
                fused_ = f == 1;
                float ms = 0.f;
                try {
                    check_cuda(cudaMemsetAsync(clock_dev, 0, 4, st), "memset");
                    sweep(0, st);  // warm-up
                    check_cuda(cudaEventRecord(e0, st), "cudaEventRecord");
                    sweep(1, st);
                    sweep(2, st);
                    check_cuda(cudaEventRecord(e1, st), "cudaEventRecord");
                    check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
                    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
                } catch (const Error&) {
                    cudaGetLastError();
                    check_cuda(cudaStreamSynchronize(st), "autotuner");
                    continue;
                }
                if (best_v < 0 || ms < best) {
                    best = ms;
                    best_v = v;
                    best_f = fused_;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (best_v < 0) fail(SG_ECUDA, "no colour-kernel configuration could be launched");
        if (device_status(st)) fail(SG_ETIMEOUT, "device wait expired while tuning the colour kernel");
        variant_ = best_v;
        fused_ = best_f;
        launches += vb_packed_init(pk_, st);
    }

    void sweep(uint32_t t_off, cudaStream_t st) override {
        if (kernel_ == SG_VB_PACKED) {
            const int n = vb_packed_sweep(pk_, colour_group_.data(), clock_dev, t_off, variant_,
                                          fused_, st);
            if (n < 0) fail(SG_ECUDA, "colour kernel launch failed");
            launches += n;
        } else {
            for (size_t c = 0; c + 1 < colour_begin_.size(); ++c)
                launches += vb_plain_colour(pl_, colour_begin_[c], colour_begin_[c + 1], clock_dev,
                                            t_off, st);
        }
    }

    bool has_pending() const override { return pend_; }

    void sweep_pending(uint32_t t_off, cudaStream_t st) override {
        if (!pend_) return sweep(t_off, st);
        pend_ = false;
        const VbSweepMeas m{pend_job_.dst, pend_job_.stride_r, pend_job_.stride_k};
        const int n = vb_packed_sweep_meas(pk_, colour_group_.data(), clock_dev, t_off, variant_,
                                           fused_, m, st);
        if (n < 0) fail(SG_ECUDA, "measuring colour kernel launch failed");
        launches += n;
    }

    void flush_pending(cudaStream_t st) override {
        if (!pend_) return;
        pend_ = false;
        run_job(pend_job_, st);
    }

    void snapshot(int w, cudaStream_t st) override {
        if (kernel_ == SG_VB_PACKED) launches += vb_packed_snapshot(pk_, w, st);
        else if (vb_plain_snapshot(pl_, w, st) < 0) fail(SG_ECUDA, "snapshot copy failed");
    }

    // add the raw counts at time tau into column u of count arrays with ncol columns
    void measure_into(int64_t* Cb, int64_t* Qb, int64_t* Eb, int64_t ncol, int64_t u, int64_t tau,
                      cudaStream_t st) {
        const int64_t ntw = (int64_t)tw.size();
        int64_t active = 0;
        while (active < ntw && tw[active] <= tau) ++active;
        const VbCountJob qj{1, 0, Qb + u, (int64_t)(R / 2) * Lc_ * ncol, (int64_t)Lc_ * ncol, ncol, 0, 0};
        if (kernel_ == SG_VB_PACKED && active > 0) {
            // every active snapshot and the replica overlaps in one pass over the current spins
            VbCountJob j{3, (int)active, Cb + u, (int64_t)R * Lc_ * ntw * ncol,
                         (int64_t)Lc_ * ntw * ncol, ntw * ncol, ncol, 0};
            launches += vb_packed_count(pk_, j, st, R >= 2 ? &qj : nullptr);
        } else {
            for (int64_t w = 0; w < active; ++w) {
                VbCountJob j{0, (int)w, Cb + w * ncol + u, (int64_t)R * Lc_ * ntw * ncol,
                             (int64_t)Lc_ * ntw * ncol, ntw * ncol, 0, 0};
                run_job(j, st);
            }
            if (R >= 2) run_job(qj, st);
        }
        const VbCountJob ej{2, 0, Eb + u, (int64_t)R * Lc_ * ncol, (int64_t)Lc_ * ncol, ncol, 0, 0};
        if (fuse_e_) {
            flush_pending(st);  // two measurements of one state (a schedule and a window)
            pend_ = true;
            pend_job_ = ej;
        } else {
            run_job(ej, st);
        }
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
        for (int b = 0; b < n_inst; ++b) {
            const int64_t N = graphs_[b].n, M = graphs_[b].edges;
            for (int r = 0; r < R; ++r)
                for (int k = 0; k < L; ++k)
                    for (int64_t m = 0; m < nb; ++m) {
                        for (int64_t w = 0; w < ntw; ++w) {
                            const int64_t src = ((((int64_t)b * R + r) * Lc_ + k) * ntw + w) * nb + m;
                            const int64_t dst = ((((int64_t)b * R + r) * L + k) * ntw + w) * nb + m;
                            C[dst] = cnt_c[w * nb + m] * N - 2 * c[src];
                        }
                        const int64_t se = (((int64_t)b * R + r) * Lc_ + k) * nb + m;
                        const int64_t de = (((int64_t)b * R + r) * L + k) * nb + m;
                        E[de] = cnt_q[m] * M - e[se];
                        if (r < R / 2) {
                            const int64_t sq = (((int64_t)b * (R / 2) + r) * Lc_ + k) * nb + m;
                            const int64_t dq = (((int64_t)b * (R / 2) + r) * L + k) * nb + m;
                            q[dq] = cnt_q[m] * N - 2 * qq[sq];
                        }
                    }
        }
    }

    void measure_now(int64_t tau, cudaStream_t st) override {
        flush_pending(st);
        const int64_t ntw = (int64_t)tw.size();
        check_cuda(cudaMemsetAsync(mC_, 0, nmC() * 8, st), "memset");
        check_cuda(cudaMemsetAsync(mQ_, 0, nmQ() * 8, st), "memset");
        check_cuda(cudaMemsetAsync(mE_, 0, nmE() * 8, st), "memset");
        for (int64_t w = 0; w < ntw; ++w) {
            if (tw[w] > tau) break;
            VbCountJob j{0, (int)w, mC_ + w, (int64_t)R * Lc_ * ntw, (int64_t)Lc_ * ntw, ntw, 0};
            run_job(j, st);
        }
        if (R >= 2) {
            VbCountJob j{1, 0, mQ_, (int64_t)(R / 2) * Lc_, (int64_t)Lc_, 1, 0};
            run_job(j, st);
        }
        VbCountJob j{2, 0, mE_, (int64_t)R * Lc_, (int64_t)Lc_, 1, 0};
        run_job(j, st);
    }

    void read_scheduled(int64_t tau, int64_t* C, int64_t* q, int64_t* E, cudaStream_t st) override {
        std::vector<int64_t> c(nC()), qq(nQ()), e(nE());
        down(c.data(), dC_, c.size() * 8, st);
        down(qq.data(), dQ_, qq.size() * 8, st);
        down(e.data(), dE_, e.size() * 8, st);
        check_cuda(cudaStreamSynchronize(st), "read results");
        const int64_t ntw = (int64_t)tw.size(), ntm = (int64_t)tm.size();
        for (int b = 0; b < n_inst; ++b) {
            const int64_t N = graphs_[b].n, M = graphs_[b].edges;
            for (int r = 0; r < R; ++r)
                for (int k = 0; k < L; ++k)
                    for (int64_t u = 0; u < ntm; ++u) {
                        const bool done = tm[u] <= tau;
                        for (int64_t w = 0; w < ntw; ++w) {
                            const bool ok = done && tw[w] <= tm[u];
                            const int64_t src = ((((int64_t)b * R + r) * Lc_ + k) * ntw + w) * ntm + u;
                            const int64_t dst = ((((int64_t)b * R + r) * L + k) * ntw + w) * ntm + u;
                            C[dst] = ok ? N - 2 * c[src] : 0;
                        }
                        const int64_t se = (((int64_t)b * R + r) * Lc_ + k) * ntm + u;
                        const int64_t de = (((int64_t)b * R + r) * L + k) * ntm + u;
                        E[de] = done ? M - e[se] : 0;
                        if (r < R / 2) {
                            const int64_t sq = (((int64_t)b * (R / 2) + r) * Lc_ + k) * ntm + u;
                            const int64_t dq = (((int64_t)b * (R / 2) + r) * L + k) * ntm + u;
                            q[dq] = done ? N - 2 * qq[sq] : 0;
                        }
                    }
        }
    }

    void read_now(int64_t tau, int64_t* C, int64_t* q, int64_t* E, cudaStream_t st) override {
        std::vector<int64_t> c(nmC()), qq(nmQ()), e(nmE());
        down(c.data(), mC_, c.size() * 8, st);
        down(qq.data(), mQ_, qq.size() * 8, st);
        down(e.data(), mE_, e.size() * 8, st);
        check_cuda(cudaStreamSynchronize(st), "read measurement");
        const int64_t ntw = (int64_t)tw.size();
        for (int b = 0; b < n_inst; ++b) {
            const int64_t N = graphs_[b].n, M = graphs_[b].edges;
            for (int r = 0; r < R; ++r)
                for (int k = 0; k < L; ++k) {
                    for (int64_t w = 0; w < ntw; ++w) {
                        const int64_t src = (((int64_t)b * R + r) * Lc_ + k) * ntw + w;
                        const int64_t dst = (((int64_t)b * R + r) * L + k) * ntw + w;
                        C[dst] = tw[w] <= tau ? N - 2 * c[src] : 0;
                    }
                    E[((int64_t)b * R + r) * L + k] = M - e[((int64_t)b * R + r) * Lc_ + k];
                    if (r < R / 2)
                        q[((int64_t)b * (R / 2) + r) * L + k] =
                            N - 2 * qq[((int64_t)b * (R / 2) + r) * Lc_ + k];
                }
        }
    }

    size_t spins_bytes() const override {
        int64_t tot = 0;
        for (const Graph& g : graphs_) tot += (int64_t)R * g.n;
        return (size_t)tot * 8;
    }

    void get_spins(void* dst, cudaStream_t st) override {
        uint64_t* out = static_cast<uint64_t*>(dst);
        if (kernel_ == SG_VB_PACKED) {
            std::vector<uint64_t> S((size_t)pk_.n_slots * R);
            down(S.data(), pk_.S, S.size() * 8, st);
            check_cuda(cudaStreamSynchronize(st), "read spins");
            int64_t off = 0;
            for (int b = 0; b < n_inst; ++b) {
                const Graph& g = graphs_[b];
                for (int r = 0; r < R; ++r)
                    for (int32_t v = 0; v < g.n; ++v)
                        out[off + (int64_t)r * g.n + v] = S[(size_t)slot_of_[b][v] * R + r];
                off += (int64_t)R * g.n;
            }
        } else {
            const int32_t N = pl_.N;
            std::vector<int8_t> s((size_t)R * L * N);
            down(s.data(), pl_.s, s.size(), st);
            check_cuda(cudaStreamSynchronize(st), "read spins");
            for (int r = 0; r < R; ++r)
                for (int32_t v = 0; v < N; ++v) {
                    const int32_t nv = new_of_[v];
                    uint64_t w = 0;
                    for (int k = 0; k < L; ++k)
                        if (s[((size_t)r * L + k) * N + nv] < 0) w |= 1ull << k;
                    out[(int64_t)r * N + v] = w;
                }
        }
    }

    std::vector<uint32_t> thresholds() const override { return thr_; }

    std::vector<int32_t> colouring(int b, int* n_colours) const override {
        if (b < 0 || b >= n_inst) fail(SG_EINVAL, "graph index out of range");
        *n_colours = graphs_[b].n_colours;
        return graphs_[b].colour;
    }

    int device_status(cudaStream_t st) override {
        int v = 0;
        if (kernel_ == SG_VB_PACKED && pk_.err) {
            check_cuda(cudaMemcpyAsync(&v, pk_.err, 4, cudaMemcpyDeviceToHost, st), "status copy");
            check_cuda(cudaStreamSynchronize(st), "status");
        }
        return v;
    }

    std::vector<std::pair<void*, size_t>> state_regions() override {
        std::vector<std::pair<void*, size_t>> v;
        if (kernel_ == SG_VB_PACKED) {
            v.push_back({pk_.S, (size_t)pk_.n_slots * R * 8});
            v.push_back({pk_.snap, (size_t)tw.size() * pk_.n_slots * R * 8});
        } else {
            const size_t n = (size_t)R * L * pl_.N;
            v.push_back({pl_.s, n});
            v.push_back({pl_.snap, tw.size() * n});
        }
        v.push_back({dC_, nC() * 8});
        v.push_back({dQ_, nQ() * 8});
        v.push_back({dE_, nE() * 8});
        if (n_bins) {
            v.push_back({wC_, nwC() * 8});
            v.push_back({wQ_, nwQ() * 8});
            v.push_back({wE_, nwE() * 8});
        }
        return v;
    }

private:
    size_t nC() const { return (size_t)n_inst * R * Lc_ * tw.size() * tm.size(); }
    size_t nQ() const { return (size_t)n_inst * (R / 2) * Lc_ * tm.size(); }
    size_t nE() const { return (size_t)n_inst * R * Lc_ * tm.size(); }
    size_t nmC() const { return (size_t)n_inst * R * Lc_ * tw.size(); }
    size_t nwC() const { return (size_t)n_inst * R * Lc_ * tw.size() * n_bins; }
    size_t nwQ() const { return (size_t)n_inst * (R / 2) * Lc_ * n_bins; }
    size_t nwE() const { return (size_t)n_inst * R * Lc_ * n_bins; }
    size_t nmQ() const { return (size_t)n_inst * (R / 2) * Lc_; }
    size_t nmE() const { return (size_t)n_inst * R * Lc_; }

    void down(void* dst, const void* src, size_t bytes, cudaStream_t st) {
        d2h_bytes += (int64_t)bytes;
        if (bytes) check_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st), "D2H copy");
    }

    void run_job(const VbCountJob& j, cudaStream_t st) {
        if (kernel_ == SG_VB_PACKED) launches += vb_packed_count(pk_, j, st);
        else launches += vb_plain_count(pl_, j, st);
    }

    void carve(Carver& c) {
        clock_dev = c.take<uint32_t>(1);
        d_thr_ = c.take<uint32_t>(thr_.size());
        if (kernel_ == SG_VB_PACKED) {
            pk_.vinfo = c.take<uint32_t>(h_vinfo_.size());
            pk_.slice_base = c.take<uint32_t>(h_slice_base_.size());
            pk_.slice_graph = c.take<uint32_t>(h_slice_graph_.size());
            pk_.col = c.take<uint32_t>(h_col_.size());
            pk_.groups = c.take<uint4>(h_groups_.size());
            pk_.slice_meta = c.take<uint4>(h_slice_meta_.size());
            pk_.group_graph = c.take<uint32_t>(h_group_graph_.size());
            pk_.gtab = c.take<uint8_t>(h_gtab_.size());
            pk_.err = c.take<int>(1);
            pk_.colour_groups = c.take<uint32_t>(colour_group_.size());
            pk_.gbar = c.take<uint32_t>(2);
            pk_.jb = c.take<uint64_t>(h_jb_.size());
            pk_.seeds = c.take<uint64_t>(n_inst);
            pk_.up_slice_base = c.take<uint32_t>(h_up_base_.size());
            pk_.up_col = c.take<uint32_t>(up_entries_);
            pk_.up_jb = c.take<uint64_t>(up_entries_);
            pk_.S = c.take<uint64_t>((size_t)n_slots_ * R);
            pk_.snap = c.take<uint64_t>((size_t)n_slots_ * R * tw.size());
            pk_.thr = d_thr_;
            pk_.n_slots = n_slots_;
            pk_.n_slices = (int32_t)(n_slots_ / 32);
            pk_.R = R;
            pk_.n_colours = (int32_t)colour_group_.size() - 1;
            // SG_TEST_STAGE_WAIT_NS shortens the colour kernel's pipeline waits: a test of the
            // timeout path (the kernel gives up, flags SG_ETIMEOUT and exits cleanly)
            pk_.stage_wait_ns = 2000000000ull;
            if (const char* w = getenv("SG_TEST_STAGE_WAIT_NS")) pk_.stage_wait_ns = strtoull(w, nullptr, 10);
            if (pk_.n_colours > kVbMaxColours) fail(SG_EINVAL, "more colour classes than supported");
        } else {
            const Graph& g = graphs_[0];
            pl_.row_ptr = c.take<int32_t>(h_row_ptr_.size());
            pl_.col = c.take<int32_t>(h_col_i_.size());
            pl_.jb = c.take<uint64_t>(h_jb_.size());
            pl_.orig = c.take<uint32_t>(h_orig_.size());
            pl_.s = c.take<int8_t>((size_t)R * L * g.n);
            pl_.snap = c.take<int8_t>((size_t)R * L * g.n * tw.size());
            pl_.thr = d_thr_;
            pl_.seed = g.seed;
            pl_.N = g.n;
            pl_.R = R;
            pl_.L = L;
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

    // colour-major CSR of the single graph (plain kernel)
    void build_plain() {
        const Graph& g = graphs_[0];
        const int32_t n = g.n;
        colour_begin_.assign(g.n_colours + 1, 0);
        for (int32_t i = 0; i < n; ++i) colour_begin_[g.colour[i] + 1]++;
        for (int c = 0; c < g.n_colours; ++c) colour_begin_[c + 1] += colour_begin_[c];
        std::vector<int32_t> cursor(colour_begin_.begin(), colour_begin_.end() - 1);
        new_of_.assign(n, 0);
        h_orig_.assign(n, 0);
        for (int32_t i = 0; i < n; ++i) {
            const int32_t nv = cursor[g.colour[i]]++;
            new_of_[i] = nv;
            h_orig_[nv] = (uint32_t)i;
        }
        h_row_ptr_.assign(n + 1, 0);
        for (int32_t nv = 0; nv < n; ++nv) {
            const int32_t i = (int32_t)h_orig_[nv];
            h_row_ptr_[nv + 1] = h_row_ptr_[nv] + (g.row_ptr[i + 1] - g.row_ptr[i]);
        }
        h_col_i_.resize(g.col.size());
        h_jb_.resize(g.col.size());
        for (int32_t nv = 0; nv < n; ++nv) {
            const int32_t i = (int32_t)h_orig_[nv];
            int32_t o = h_row_ptr_[nv];
            for (int32_t e = g.row_ptr[i]; e < g.row_ptr[i + 1]; ++e, ++o) {
                h_col_i_[o] = new_of_[g.col[e]];
                h_jb_[o] = g.jb[e];
            }
        }
    }

    // sliced-ELL over slots ordered by (colour, graph, degree descending, original label)
    void build_packed() {
        int cmax = 0;
        for (const Graph& g : graphs_) cmax = std::max(cmax, g.n_colours);
        slot_of_.resize(n_inst);
        for (int b = 0; b < n_inst; ++b) slot_of_[b].assign(graphs_[b].n, -1);
        // bucket vertices by (colour, degree) per graph, in original-label order
        std::vector<std::vector<std::vector<int32_t>>> bucket(n_inst);
        for (int b = 0; b < n_inst; ++b) {
            const Graph& g = graphs_[b];
            bucket[b].assign((size_t)g.n_colours * (SG_VB_MAX_DEGREE + 1), {});
            for (int32_t i = 0; i < g.n; ++i) {
                const int d = g.row_ptr[i + 1] - g.row_ptr[i];
                bucket[b][(size_t)g.colour[i] * (SG_VB_MAX_DEGREE + 1) + d].push_back(i);
            }
        }
        int64_t cursor = 0;
        colour_slice_.assign(cmax + 1, 0);
        std::vector<int32_t> slot_graph_vertex;  // original label per slot, -1 for padding
        std::vector<int32_t> slot_graph;
        for (int c = 0; c < cmax; ++c) {
            colour_slice_[c] = (uint32_t)(cursor / 32);
            for (int b = 0; b < n_inst; ++b) {
                const Graph& g = graphs_[b];
                if (c >= g.n_colours) continue;
                const int64_t start = cursor;
                // highest degree first: the longest slices start early instead of forming the tail
                for (int d = SG_VB_MAX_DEGREE; d >= 0; --d)
                    for (int32_t i : bucket[b][(size_t)c * (SG_VB_MAX_DEGREE + 1) + d]) {
                        slot_of_[b][i] = cursor++;
                        slot_graph_vertex.push_back(i);
                        slot_graph.push_back(b);
                    }
                if (cursor == start) continue;
                while (cursor % 32) {
                    ++cursor;
                    slot_graph_vertex.push_back(-1);
                    slot_graph.push_back(b);
                }
            }
        }
        colour_slice_[cmax] = (uint32_t)(cursor / 32);
        n_slots_ = cursor;
        const int64_t n_slices = n_slots_ / 32;
        h_vinfo_.assign(n_slots_, kInactive);
        h_slice_graph_.assign(n_slices, 0);
        h_slice_base_.assign(n_slices + 1, 0);
        std::vector<int32_t> width_of(n_slices, 0);
        parallel_ranges(n_slices, [&](int64_t s0, int64_t s1) {
            for (int64_t s = s0; s < s1; ++s) {
                const int b = slot_graph[s * 32];
                h_slice_graph_[s] = (uint32_t)b;
                const Graph& g = graphs_[b];
                int width = 0;
                for (int l = 0; l < 32; ++l) {
                    const int32_t i = slot_graph_vertex[s * 32 + l];
                    if (i < 0) continue;
                    const int d = g.row_ptr[i + 1] - g.row_ptr[i];
                    width = std::max(width, d);
                    h_vinfo_[s * 32 + l] = (uint32_t)i | ((uint32_t)d << kDegShift);
                }
                width_of[s] = width;
            }
        });
        int64_t entries = 0;
        for (int64_t s = 0; s < n_slices; ++s) {
            h_slice_base_[s] = (uint32_t)entries;
            entries += 32 * (int64_t)width_of[s];
            if (entries >= (int64_t(1) << 32)) fail(SG_EINVAL, "too many graph entries for one batch");
        }
        h_slice_base_[n_slices] = (uint32_t)entries;
        h_col_.assign(entries, 0);
        h_jb_.assign(entries, 0);
        // every slice writes only its own entries
        parallel_ranges(n_slices, [&](int64_t s0, int64_t s1) {
            for (int64_t s = s0; s < s1; ++s) {
                const int b = (int)h_slice_graph_[s];
                const Graph& g = graphs_[b];
                const int64_t base = h_slice_base_[s];
                const int width = (int)((h_slice_base_[s + 1] - base) / 32);
                for (int l = 0; l < 32; ++l) {
                    const int64_t slot = s * 32 + l;
                    const int32_t i = slot_graph_vertex[slot];
                    int e = 0;
                    if (i >= 0)
                        for (int32_t k = g.row_ptr[i]; k < g.row_ptr[i + 1]; ++k, ++e) {
                            h_col_[base + (int64_t)e * 32 + l] = (uint32_t)slot_of_[b][g.col[k]];
                            h_jb_[base + (int64_t)e * 32 + l] = g.jb[k];
                        }
                    for (; e < width; ++e) {
                        h_col_[base + (int64_t)e * 32 + l] = (uint32_t)slot;
                        h_jb_[base + (int64_t)e * 32 + l] = 0;
                    }
                }
            }
        });
        // upper entries (energy measurement): neighbours in later colour classes only
        h_up_base_.assign(n_slices + 1, 0);
        std::vector<int32_t> up_width(n_slices, 0);
        std::vector<uint32_t> up_kind(n_slices, kUpNone);
        parallel_ranges(n_slices, [&](int64_t s0, int64_t s1) {
            for (int64_t s = s0; s < s1; ++s) {
                const int b = (int)h_slice_graph_[s];
                const Graph& g = graphs_[b];
                int w = 0;
                bool all = true;
                for (int l = 0; l < 32; ++l) {
                    const int64_t slot = s * 32 + l;
                    const int32_t i = slot_graph_vertex[slot];
                    if (i < 0) continue;
                    int n_up = 0;
                    for (int32_t k = g.row_ptr[i]; k < g.row_ptr[i + 1]; ++k)
                        n_up += slot_of_[b][g.col[k]] > slot;
                    w = std::max(w, n_up);
                    all = all && n_up == g.row_ptr[i + 1] - g.row_ptr[i];
                }
                up_width[s] = w;
                up_kind[s] = w == 0 ? kUpNone : all ? kUpAll : kUpMixed;
            }
        });
        int64_t up_entries = 0;
        for (int64_t s = 0; s < n_slices; ++s) {
            h_up_base_[s] = (uint32_t)up_entries;
            up_entries += 32 * (int64_t)up_width[s];
        }
        h_up_base_[n_slices] = (uint32_t)up_entries;
        up_entries_ = up_entries;  // filled on the device at attach (vb_packed_build_upper)
        h_slice_meta_.resize(n_slices);
        for (int64_t s = 0; s < n_slices; ++s) {
            uint4 m;
            m.x = h_slice_base_[s];
            m.y = (h_slice_base_[s + 1] - h_slice_base_[s]) / 32;
            m.z = h_slice_graph_[s];
            m.w = (uint32_t)up_width[s] | up_kind[s] << 16;
            h_slice_meta_[s] = m;
        }
        // staging groups: consecutive slices of one colour, <= 8 slices and <= 1024 entries;
        // a single slice wider than that (degree > 32) forms a group flagged "wide"
        colour_group_.assign(cmax + 1, 0);
        for (int c = 0; c < cmax; ++c) {
            colour_group_[c] = (uint32_t)h_groups_.size();
            int64_t s = colour_slice_[c];
            while (s < (int64_t)colour_slice_[c + 1]) {
                const int64_t first = s;
                while (s < (int64_t)colour_slice_[c + 1] && s - first < 8 &&
                       h_slice_graph_[s] == h_slice_graph_[first] &&
                       (int64_t)h_slice_base_[s + 1] - (int64_t)h_slice_base_[first] <= 1024)
                    ++s;
                bool wide = false;
                if (s == first) {  // one slice alone exceeds the stage
                    ++s;
                    wide = true;
                }
                uint4 gi;
                gi.x = (uint32_t)first;
                gi.y = (uint32_t)(s - first) | (wide ? 0x80000000u : 0u);
                gi.z = h_slice_base_[first];
                gi.w = h_slice_base_[s] - h_slice_base_[first];
                h_groups_.push_back(gi);
                h_group_graph_.push_back(h_slice_graph_[first]);
            }
        }
        // per-graph table staged with each group: thresholds of the R replicas, then the key
        const size_t gtab_bytes = (size_t)R * kVbThrStride * 4 + 16;
        h_gtab_.assign(gtab_bytes * n_inst, 0);
        for (int b = 0; b < n_inst; ++b) {
            memcpy(&h_gtab_[b * gtab_bytes], &thr_[(size_t)b * R * kVbThrStride],
                   (size_t)R * kVbThrStride * 4);
            memcpy(&h_gtab_[b * gtab_bytes + (size_t)R * kVbThrStride * 4], &graphs_[b].seed, 8);
        }
        colour_group_[cmax] = (uint32_t)h_groups_.size();
    }

    int kernel_ = SG_VB_PACKED;
    bool fuse_e_ = false;  // the energy of a measured state is taken by the next sweep
    bool pend_ = false;    // such a measurement is waiting for that sweep (pend_job_ its target)
    VbCountJob pend_job_{};
    int variant_ = 0;     // colour-kernel pipeline shape chosen by the autotuner at attach
    bool fused_ = false;  // one cooperative launch per sweep (else one launch per colour class)
    int Lc_ = 64;
    size_t ws_bytes_ = 0;
    std::vector<Graph> graphs_;
    std::vector<uint32_t> thr_;
    // packed host layout
    std::vector<uint32_t> colour_slice_, colour_group_;
    std::vector<uint4> h_groups_, h_slice_meta_;
    std::vector<uint32_t> h_group_graph_;
    std::vector<uint8_t> h_gtab_;
    std::vector<std::vector<int64_t>> slot_of_;
    int64_t n_slots_ = 0;
    std::vector<uint32_t> h_slice_base_, h_slice_graph_;
    pinned_vector<uint32_t> h_vinfo_, h_col_;  // the large images copied at attach: page-locked
    pinned_vector<uint64_t> h_jb_;
    std::vector<uint32_t> h_up_base_;  // upper entries (energy measurement): slice bases
    int64_t up_entries_ = 0;
    // plain host layout
    std::vector<int32_t> colour_begin_, new_of_, h_row_ptr_, h_col_i_;
    std::vector<uint32_t> h_orig_;
    // device views
    VbPackedDev pk_{};
    VbPlainDev pl_{};
    uint32_t* d_thr_ = nullptr;
    int64_t *dC_ = nullptr, *dQ_ = nullptr, *dE_ = nullptr;
    int64_t *mC_ = nullptr, *mQ_ = nullptr, *mE_ = nullptr;
    int64_t *wC_ = nullptr, *wQ_ = nullptr, *wE_ = nullptr;  // window sums of raw counts
};

}  // namespace

Model* make_vb_model(const void* graphs, int n_graphs, int n_lanes, int n_replicas, int kernel,
                     const std::vector<int64_t>& tw, const std::vector<int64_t>& tm) {
    return new VbModel(static_cast<const sg_vb_graph*>(graphs), n_graphs, n_lanes, n_replicas,
                       kernel, tw, tm);
}

}  // namespace sg
