// sg_api.cu -- the extern "C" boundary of libsg (declared in include/sg.h): argument checking,
// the measurement schedule and the sweep clock, error codes and messages.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/sg.h"
#include "sg_model.h"

namespace sg {

[[noreturn]] void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) fail(SG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

uint32_t metropolis_threshold(double x) {
    const double v = ldexp(exp(x), 32);
    if (!(v < 4294967295.0)) return 0xFFFFFFFFu;
    return (uint32_t)floor(v);
}

// the device-side sweep clock read by the sweep kernels (t = *clock + offset)
__global__ void k_clock_set(uint32_t* c, uint32_t v) { *c = v; }
__global__ void k_clock_add(uint32_t* c, uint32_t v) { *c += v; }

}  // namespace sg

// Sweeps are replayed from CUDA graphs of 2^k sweeps (k <= kMaxGraphLog), all captured on a
// private stream the first time sweeps run and launched on the caller's stream; the graph size
// is also capped in nodes.
static const int kMaxGraphLog = 6;
static const int64_t kMaxGraphNodes = 4096;

struct sg_ctx {
    std::unique_ptr<sg::Model> model;
    std::vector<int64_t> tw, tm;
    std::vector<int64_t> wb;  // window bounds (window m: wb[m] <= tau < wb[m+1]); empty: none
    int64_t tau = 0;
    bool attached = false;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    size_t next_tw = 0, next_tm = 0;  // first schedule entries with time > tau
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graphs[kMaxGraphLog + 1] = {};
    int64_t graph_kernels[kMaxGraphLog + 1] = {};
    int max_graph_log = -1;  // decided at the first capture
    ~sg_ctx() {
        for (auto& g : graphs)
            if (g) cudaGraphExecDestroy(g);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

static thread_local std::string g_last_error;

void sg::record_error(const std::string& msg) { g_last_error = msg; }

static int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

template <class F>
static int guarded(F&& f) {
    try {
        g_last_error.clear();
        f();
        return SG_OK;
    } catch (const sg::Error& e) {
        return set_error(e.code, e.msg);
    } catch (const std::bad_alloc&) {
        return set_error(SG_ENOMEM, "host allocation failed");
    } catch (const std::exception& e) {
        return set_error(SG_EINVAL, e.what());
    } catch (...) {
        return set_error(SG_EINVAL, "unknown error");
    }
}

static std::vector<int64_t> read_schedule(const int64_t* a, int32_t n, const char* name) {
    if (n < 0 || (n > 0 && !a)) sg::fail(SG_EINVAL, std::string(name) + ": bad array");
    std::vector<int64_t> v(a, a + n);
    for (int32_t i = 0; i < n; ++i) {
        if (v[i] < 0) sg::fail(SG_EINVAL, std::string(name) + ": negative time");
        if (v[i] >= (int64_t(1) << 32)) sg::fail(SG_EINVAL, std::string(name) + ": time >= 2^32");
        if (i && v[i] <= v[i - 1]) sg::fail(SG_EINVAL, std::string(name) + ": not strictly increasing");
    }
    return v;
}

// capture (once) a graph running 2^k sweeps at clock offsets 0..2^k-1 and advancing the clock
static cudaGraphExec_t sweep_graph(sg_handle h, int k) {
    if (h->graphs[k]) return h->graphs[k];
    sg::Model& m = *h->model;
    if (!h->cap_stream)
        sg::check_cuda(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking),
                       "cudaStreamCreateWithFlags");
    const int64_t before = m.launches;
    const uint32_t n = 1u << k;
    sg::check_cuda(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal),
                   "cudaStreamBeginCapture");
    cudaGraph_t g = nullptr;
    try {
        m.sweep_many(0, (int)n, h->cap_stream);
        sg::k_clock_add<<<1, 1, 0, h->cap_stream>>>(m.clock_dev, n);
    } catch (...) {
        cudaStreamEndCapture(h->cap_stream, &g);
        if (g) cudaGraphDestroy(g);
        m.launches = before;
        throw;
    }
    sg::check_cuda(cudaStreamEndCapture(h->cap_stream, &g), "cudaStreamEndCapture");
    const cudaError_t e = cudaGraphInstantiate(&h->graphs[k], g, 0);
    cudaGraphDestroy(g);
    sg::check_cuda(e, "cudaGraphInstantiate");
    h->graph_kernels[k] = m.launches - before + 1;
    m.launches = before;
    return h->graphs[k];
}

// queue sweeps t0 .. t0+len-1 on the handle's stream
static void run_sweeps(sg_handle h, int64_t t0, int64_t len) {
    if (len <= 0) return;
    sg::Model& m = *h->model;
    if (m.has_pending()) {
        // the first sweep takes the deferred measurement of the state it starts from: the clock
        // is set past it and the sweep runs at offset -1 (index t0)
        sg::k_clock_set<<<1, 1, 0, h->stream>>>(m.clock_dev, (uint32_t)(t0 + 1));
        m.launches += 1;
        m.sweep_pending(0xFFFFFFFFu, h->stream);
        ++t0;
        if (--len == 0) return;
    } else {
        sg::k_clock_set<<<1, 1, 0, h->stream>>>(m.clock_dev, (uint32_t)t0);
        m.launches += 1;
    }
    if (h->max_graph_log < 0) {
        sweep_graph(h, 0);
        const int64_t per_sweep = std::max<int64_t>(1, h->graph_kernels[0] - 1);
        int k = 0;
        while (k < kMaxGraphLog && ((int64_t)2 << k) * per_sweep <= kMaxGraphNodes) ++k;
        h->max_graph_log = k;
        // every size now, so that a later call (a timed one) only replays
        for (int j = 1; j <= k; ++j) sweep_graph(h, j);
    }
    int64_t done = 0;
    for (int k = h->max_graph_log; k >= 0; --k) {
        const int64_t g = int64_t(1) << k;
        while (len - done >= g) {
            sg::check_cuda(cudaGraphLaunch(sweep_graph(h, k), h->stream), "cudaGraphLaunch");
            m.launches += h->graph_kernels[k];
            done += g;
        }
    }
}

static void require_attached(sg_handle h) {
    if (!h) sg::fail(SG_EINVAL, "null handle");
    if (!h->attached) sg::fail(SG_ESTATE, "handle has no workspace (call sg_attach first)");
}

// take a measurement the model deferred into its next sweep now (the counts are about to be
// read, or the state replaced)
static void settle(sg_handle h) {
    h->model->flush_pending(h->stream);
    sg::check_cuda(cudaGetLastError(), "measure launch");
}

// snapshot/measure at the current tau if the schedule says so
static void events_at_tau(sg_handle h) {
    sg::Model& m = *h->model;
    while (h->next_tw < h->tw.size() && h->tw[h->next_tw] == h->tau) {
        m.snapshot((int)h->next_tw, h->stream);
        ++h->next_tw;
    }
    while (h->next_tm < h->tm.size() && h->tm[h->next_tm] == h->tau) {
        m.measure_scheduled((int)h->next_tm, h->tau, h->stream);
        ++h->next_tm;
    }
    if (!h->wb.empty() && h->tau >= h->wb.front() && h->tau < h->wb.back()) {
        const int w = (int)(std::upper_bound(h->wb.begin(), h->wb.end(), h->tau) - h->wb.begin()) - 1;
        m.measure_window(w, h->tau, h->stream);
    }
    sg::check_cuda(cudaGetLastError(), "kernel launch");
}

// the next time after tau at which a window measurement is due (or -1)
static int64_t next_window_tau(const sg_ctx* h) {
    if (h->wb.empty()) return -1;
    const int64_t t = std::max(h->tau + 1, h->wb.front());
    return t < h->wb.back() ? t : -1;
}

extern "C" {

const char* sg_last_error(void) { return g_last_error.c_str(); }

int sg_create_vb(const sg_vb_graph* graphs, int32_t n_graphs, int32_t n_lanes, int32_t n_replicas,
                 int32_t kernel, const int64_t* tw, int32_t n_tw, const int64_t* tm, int32_t n_tm,
                 sg_handle* out) {
    return guarded([&] {
        if (!out) sg::fail(SG_EINVAL, "out is null");
        *out = nullptr;
        if (!graphs || n_graphs < 1) sg::fail(SG_EINVAL, "need at least one graph");
        std::unique_ptr<sg_ctx> h(new sg_ctx());
        h->tw = read_schedule(tw, n_tw, "tw");
        h->tm = read_schedule(tm, n_tm, "tm");
        h->model.reset(sg::make_vb_model(graphs, n_graphs, n_lanes, n_replicas, kernel, h->tw, h->tm));
        *out = h.release();
    });
}

int sg_create_sk(int32_t n, const int8_t* J, int32_t n_replicas, const double* temps, uint64_t seed,
                 int32_t kernel, int32_t block, const int64_t* tw, int32_t n_tw, const int64_t* tm,
                 int32_t n_tm, sg_handle* out) {
    return guarded([&] {
        if (!out) sg::fail(SG_EINVAL, "out is null");
        *out = nullptr;
        std::unique_ptr<sg_ctx> h(new sg_ctx());
        h->tw = read_schedule(tw, n_tw, "tw");
        h->tm = read_schedule(tm, n_tm, "tm");
        h->model.reset(sg::make_sk_model(n, J, n_replicas, temps, seed, kernel, block, h->tw, h->tm));
        *out = h.release();
    });
}

int sg_create_sk_batch(const sg_sk_sample* samples, int32_t n_samples, int32_t n_replicas,
                       int32_t kernel, int32_t block, const int64_t* tw, int32_t n_tw,
                       const int64_t* tm, int32_t n_tm, sg_handle* out) {
    return guarded([&] {
        if (!out) sg::fail(SG_EINVAL, "out is null");
        *out = nullptr;
        std::unique_ptr<sg_ctx> h(new sg_ctx());
        h->tw = read_schedule(tw, n_tw, "tw");
        h->tm = read_schedule(tm, n_tm, "tm");
        h->model.reset(sg::make_sk_batch_model(samples, n_samples, n_replicas, kernel, block, h->tw,
                                               h->tm));
        *out = h.release();
    });
}

int sg_set_schedule(sg_handle h, const int64_t* tw, int32_t n_tw, const int64_t* tm,
                    int32_t n_tm) {
    return guarded([&] {
        if (!h) sg::fail(SG_EINVAL, "null handle");
        std::vector<int64_t> a = read_schedule(tw, n_tw, "tw");
        std::vector<int64_t> b = read_schedule(tm, n_tm, "tm");
        if (h->attached) {
            if (h->next_tw > 0 || h->next_tm > 0)
                sg::fail(SG_ESTATE, "a scheduled time has already been reached");
            if (a.size() != h->tw.size() || b.size() != h->tm.size())
                sg::fail(SG_ESTATE, "after sg_attach the schedule must keep n_tw and n_tm");
            if ((!a.empty() && a.front() <= h->tau) || (!b.empty() && b.front() <= h->tau))
                sg::fail(SG_ESTATE, "after sg_attach every new time must be later than tau");
        }
        h->model->set_schedule(a, b, h->attached);
        h->tw = std::move(a);
        h->tm = std::move(b);
    });
}

int sg_workspace_bytes(sg_handle h, size_t* bytes) {
    return guarded([&] {
        if (!h || !bytes) sg::fail(SG_EINVAL, "null argument");
        *bytes = h->model->workspace_bytes();
    });
}

int sg_attach(sg_handle h, void* dev_workspace, size_t bytes, void* cuda_stream) {
    return guarded([&] {
        if (!h) sg::fail(SG_EINVAL, "null handle");
        if (h->attached) sg::fail(SG_ESTATE, "already attached");
        const size_t need = h->model->workspace_bytes();
        if (!dev_workspace || bytes < need)
            sg::fail(SG_ENOMEM, "workspace too small: need " + std::to_string(need) + " bytes");
        if (reinterpret_cast<uintptr_t>(dev_workspace) & 255)
            sg::fail(SG_ENOMEM, "workspace must be 256-byte aligned");
        cudaPointerAttributes attr;
        sg::check_cuda(cudaPointerGetAttributes(&attr, dev_workspace), "cudaPointerGetAttributes");
        if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
            sg::fail(SG_EINVAL, "workspace is not device memory");
        h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
        h->ws = static_cast<char*>(dev_workspace);
        h->ws_bytes = bytes;
        h->model->attach(h->ws, h->stream);
        h->attached = true;
        h->tau = 0;
        h->next_tw = h->next_tm = 0;
        events_at_tau(h);
    });
}

int sg_sweep(sg_handle h, int64_t n) {
    return guarded([&] {
        require_attached(h);
        if (n < 0) sg::fail(SG_EINVAL, "negative sweep count");
        if (h->tau + n >= (int64_t(1) << 32)) sg::fail(SG_EINVAL, "time would exceed 2^32 sweeps");
        sg::Model& m = *h->model;
        const int64_t end = h->tau + n;
        while (h->tau < end) {
            int64_t stop = end;
            if (h->next_tw < h->tw.size()) stop = std::min(stop, h->tw[h->next_tw]);
            if (h->next_tm < h->tm.size()) stop = std::min(stop, h->tm[h->next_tm]);
            const int64_t tw_next = next_window_tau(h);
            if (tw_next >= 0) stop = std::min(stop, tw_next);
            run_sweeps(h, h->tau, stop - h->tau);
            sg::check_cuda(cudaGetLastError(), "sweep launch");
            h->tau = stop;
            events_at_tau(h);
        }
    });
}

int sg_set_windows(sg_handle h, const int64_t* bounds, int32_t n_bounds) {
    return guarded([&] {
        if (!h) sg::fail(SG_EINVAL, "null handle");
        if (h->attached) sg::fail(SG_ESTATE, "windows must be set before sg_attach");
        if (!bounds || n_bounds < 2 || n_bounds > (1 << 16))
            sg::fail(SG_EINVAL, "need 2 .. 65536 window bounds");
        std::vector<int64_t> b(bounds, bounds + n_bounds);
        if (b[0] < 0) sg::fail(SG_EINVAL, "window bounds must be >= 0");
        for (int32_t i = 1; i < n_bounds; ++i)
            if (b[i] <= b[i - 1]) sg::fail(SG_EINVAL, "window bounds must increase strictly");
        if (b.back() > (int64_t(1) << 32)) sg::fail(SG_EINVAL, "window bounds beyond 2^32 sweeps");
        h->model->set_windows(n_bounds - 1);
        h->wb = std::move(b);
    });
}

int sg_read_windows(sg_handle h, int64_t* C, int64_t* q, int64_t* E, int64_t* n_meas) {
    return guarded([&] {
        require_attached(h);
        if (h->wb.empty()) sg::fail(SG_ESTATE, "no measurement windows were set");
        if (!C || !q || !E || !n_meas) sg::fail(SG_EINVAL, "null output array");
        settle(h);
        sg::Model& m = *h->model;
        const int64_t nb = (int64_t)h->wb.size() - 1, ntw = (int64_t)h->tw.size();
        // sweeps measured so far in each window: tau' in [wb[m], wb[m+1]) with tau' <= tau
        // (and tau' >= tw[w] for the correlation with snapshot w)
        std::vector<int64_t> cnt((size_t)(ntw + 1) * nb);
        for (int64_t k = 0; k < nb; ++k) {
            const int64_t lo = h->wb[k], hi = std::min(h->wb[k + 1], h->tau + 1);
            for (int64_t w = 0; w < ntw; ++w) cnt[w * nb + k] = std::max<int64_t>(0, hi - std::max(lo, h->tw[w]));
            cnt[ntw * nb + k] = std::max<int64_t>(0, hi - lo);
        }
        m.read_windows(cnt.data(), cnt.data() + ntw * nb, C, q, E, h->stream);
        std::copy(cnt.begin(), cnt.end(), n_meas);
    });
}

int sg_time(sg_handle h, int64_t* tau) {
    return guarded([&] {
        if (!h || !tau) sg::fail(SG_EINVAL, "null argument");
        *tau = h->tau;
    });
}

int sg_synchronize(sg_handle h) {
    return guarded([&] {
        require_attached(h);
        sg::check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        const int st = h->model->device_status(h->stream);
        if (st) sg::fail(SG_ETIMEOUT, "device-side wait expired (status " + std::to_string(st) + ")");
    });
}

int sg_result_shape(sg_handle h, int32_t* shape5) {
    return guarded([&] {
        if (!h || !shape5) sg::fail(SG_EINVAL, "null argument");
        const sg::Model& m = *h->model;
        shape5[0] = m.n_inst;
        shape5[1] = m.R;
        shape5[2] = m.L;
        shape5[3] = (int32_t)h->tw.size();
        shape5[4] = (int32_t)h->tm.size();
    });
}

static void check_len(size_t have, size_t need, const char* name) {
    if (have < need)
        sg::fail(SG_EINVAL, std::string(name) + ": capacity " + std::to_string(have) + " < " +
                                std::to_string(need));
}

int sg_read_results(sg_handle h, int64_t* C, size_t C_len, int64_t* q, size_t q_len, int64_t* E,
                    size_t E_len) {
    return guarded([&] {
        require_attached(h);
        settle(h);
        const sg::Model& m = *h->model;
        const size_t ntw = h->tw.size(), ntm = h->tm.size();
        const size_t nC = (size_t)m.n_inst * m.R * m.L * ntw * ntm;
        const size_t nq = (size_t)m.n_inst * (m.R / 2) * m.L * ntm;
        const size_t nE = (size_t)m.n_inst * m.R * m.L * ntm;
        std::vector<int64_t> c(nC), qq(nq), e(nE);
        h->model->read_scheduled(h->tau, c.data(), qq.data(), e.data(), h->stream);
        if (C) { check_len(C_len, nC, "C"); std::copy(c.begin(), c.end(), C); }
        if (q) { check_len(q_len, nq, "q"); std::copy(qq.begin(), qq.end(), q); }
        if (E) { check_len(E_len, nE, "E"); std::copy(e.begin(), e.end(), E); }
    });
}

int sg_measure(sg_handle h, int64_t* C, size_t C_len, int64_t* q, size_t q_len, int64_t* E,
               size_t E_len) {
    return guarded([&] {
        require_attached(h);
        const sg::Model& m = *h->model;
        const size_t ntw = h->tw.size();
        const size_t nC = (size_t)m.n_inst * m.R * m.L * ntw;
        const size_t nq = (size_t)m.n_inst * (m.R / 2) * m.L;
        const size_t nE = (size_t)m.n_inst * m.R * m.L;
        h->model->measure_now(h->tau, h->stream);
        sg::check_cuda(cudaGetLastError(), "measure launch");
        std::vector<int64_t> c(nC), qq(nq), e(nE);
        h->model->read_now(h->tau, c.data(), qq.data(), e.data(), h->stream);
        if (C) { check_len(C_len, nC, "C"); std::copy(c.begin(), c.end(), C); }
        if (q) { check_len(q_len, nq, "q"); std::copy(qq.begin(), qq.end(), q); }
        if (E) { check_len(E_len, nE, "E"); std::copy(e.begin(), e.end(), E); }
    });
}

int sg_get_spins(sg_handle h, void* host_dst, size_t bytes) {
    return guarded([&] {
        require_attached(h);
        if (!host_dst) sg::fail(SG_EINVAL, "null destination");
        if (bytes != h->model->spins_bytes())
            sg::fail(SG_EINVAL, "spin buffer must be exactly " +
                                    std::to_string(h->model->spins_bytes()) + " bytes");
        h->model->get_spins(host_dst, h->stream);
    });
}

int sg_get_thresholds(sg_handle h, uint32_t* dst, size_t len) {
    return guarded([&] {
        if (!h || !dst) sg::fail(SG_EINVAL, "null argument");
        const std::vector<uint32_t> t = h->model->thresholds();
        check_len(len, t.size(), "thresholds");
        std::copy(t.begin(), t.end(), dst);
    });
}

int sg_vb_colouring(sg_handle h, int32_t graph, int32_t* colour, size_t len, int32_t* n_colours) {
    return guarded([&] {
        if (!h || !colour || !n_colours) sg::fail(SG_EINVAL, "null argument");
        int nc = 0;
        const std::vector<int32_t> c = h->model->colouring(graph, &nc);
        if (c.empty()) sg::fail(SG_EINVAL, "the handle has no colouring (not a VB handle)");
        check_len(len, c.size(), "colour");
        std::copy(c.begin(), c.end(), colour);
        *n_colours = nc;
    });
}

// checkpoint blob: magic, version, tau, next_tw, next_tm, region sizes, region bytes
static const uint64_t kStateMagic = 0x5347535441544531ull;  // "SGSTATE1"

int sg_state_bytes(sg_handle h, size_t* bytes) {
    return guarded([&] {
        require_attached(h);
        if (!bytes) sg::fail(SG_EINVAL, "null argument");
        auto regs = h->model->state_regions();
        size_t total = 8 * 5 + 8 * regs.size();
        for (auto& r : regs) total += r.second;
        *bytes = total;
    });
}

int sg_save_state(sg_handle h, void* host_dst, size_t bytes) {
    return guarded([&] {
        require_attached(h);
        auto regs = h->model->state_regions();
        size_t total = 8 * 5 + 8 * regs.size();
        for (auto& r : regs) total += r.second;
        if (!host_dst || bytes != total) sg::fail(SG_EINVAL, "state buffer has the wrong size");
        settle(h);
        sg::check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        uint64_t* hdr = static_cast<uint64_t*>(host_dst);
        hdr[0] = kStateMagic;
        hdr[1] = regs.size();
        hdr[2] = (uint64_t)h->tau;
        hdr[3] = h->next_tw;
        hdr[4] = h->next_tm;
        for (size_t i = 0; i < regs.size(); ++i) hdr[5 + i] = regs[i].second;
        char* p = static_cast<char*>(host_dst) + 8 * (5 + regs.size());
        for (auto& r : regs) {
            sg::check_cuda(cudaMemcpyAsync(p, r.first, r.second, cudaMemcpyDeviceToHost, h->stream),
                           "state copy");
            h->model->d2h_bytes += (int64_t)r.second;
            p += r.second;
        }
        sg::check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    });
}

int sg_load_state(sg_handle h, const void* host_src, size_t bytes) {
    return guarded([&] {
        require_attached(h);
        auto regs = h->model->state_regions();
        size_t total = 8 * 5 + 8 * regs.size();
        for (auto& r : regs) total += r.second;
        if (!host_src || bytes != total) sg::fail(SG_EINVAL, "state blob has the wrong size");
        settle(h);
        const uint64_t* hdr = static_cast<const uint64_t*>(host_src);
        if (hdr[0] != kStateMagic || hdr[1] != regs.size())
            sg::fail(SG_EINVAL, "state blob does not match this handle");
        for (size_t i = 0; i < regs.size(); ++i)
            if (hdr[5 + i] != regs[i].second) sg::fail(SG_EINVAL, "state blob region size mismatch");
        const char* p = static_cast<const char*>(host_src) + 8 * (5 + regs.size());
        for (auto& r : regs) {
            sg::check_cuda(cudaMemcpyAsync(r.first, p, r.second, cudaMemcpyHostToDevice, h->stream),
                           "state copy");
            h->model->h2d_bytes += (int64_t)r.second;
            p += r.second;
        }
        sg::check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        h->tau = (int64_t)hdr[2];
        h->next_tw = hdr[3];
        h->next_tm = hdr[4];
    });
}

int sg_destroy(sg_handle h) {
    return guarded([&] {
        if (!h) return;
        if (h->attached) cudaStreamSynchronize(h->stream);
        delete h;
    });
}

int sg_transfer_bytes(sg_handle h, int64_t* h2d, int64_t* d2h) {
    return guarded([&] {
        if (!h || !h2d || !d2h) sg::fail(SG_EINVAL, "null argument");
        h->model->transfer_bytes(*h2d, *d2h);
    });
}

int sg_launch_count(sg_handle h, int64_t* count) {
    return guarded([&] {
        if (!h || !count) sg::fail(SG_EINVAL, "null argument");
        *count = h->model->launches;
    });
}

}  // extern "C"
