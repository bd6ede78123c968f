// sg_model.h -- host-side model interface behind the C ABI.  sg_api.cu owns the handle, the
// schedule and the clock; a Model owns its device layout and launches its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdlib.h>

#include <new>
#include <string>
#include <utility>
#include <vector>

namespace sg {

// Error raised inside the host library; converted to a status code at the ABI boundary.
struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg);
// set the message returned by sg_last_error() on this thread
void record_error(const std::string& msg);
void check_cuda(cudaError_t e, const char* what);

// Page-locked host memory for the large host-side images that sg_attach copies to the device
// (so the copies run at DMA speed); plain heap memory where no CUDA device is present.  A
// 64-byte header before each block records which of the two it came from.
template <class T>
struct PinnedAllocator {
    using value_type = T;
    PinnedAllocator() = default;
    template <class U>
    PinnedAllocator(const PinnedAllocator<U>&) {}
    T* allocate(size_t n) {
        const size_t bytes = n * sizeof(T) + 64;
        void* p = nullptr;
        int pinned = 1;
        if (cudaMallocHost(&p, bytes) != cudaSuccess || !p) {
            cudaGetLastError();
            pinned = 0;
            p = malloc(bytes);
            if (!p) throw std::bad_alloc();
        }
        *static_cast<int*>(p) = pinned;
        return reinterpret_cast<T*>(static_cast<char*>(p) + 64);
    }
    void deallocate(T* q, size_t) {
        char* p = reinterpret_cast<char*>(q) - 64;
        if (*reinterpret_cast<int*>(p)) cudaFreeHost(p);
        else free(p);
    }
    template <class U>
    bool operator==(const PinnedAllocator<U>&) const { return true; }
    template <class U>
    bool operator!=(const PinnedAllocator<U>&) const { return false; }
};
template <class T>
using pinned_vector = std::vector<T, PinnedAllocator<T>>;

// 256-byte aligned carving of one caller-provided workspace (a null base only measures).
struct Carver {
    char* base = nullptr;
    size_t off = 0;
    template <class T>
    T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

class Model {
public:
    virtual ~Model() = default;
    // bytes of device workspace
    virtual size_t workspace_bytes() const = 0;
    // copy the instance into ws, draw the initial spins, zero the counters (synchronous)
    virtual void attach(char* ws, cudaStream_t st) = 0;
    // one sweep with sweep index *clock_dev + t_off (queued; also used under stream capture)
    virtual void sweep(uint32_t t_off, cudaStream_t st) = 0;
    // n consecutive sweeps with indices *clock_dev + t_off + 0 .. n - 1 (a model may run them in
    // fewer launches than n)
    virtual void sweep_many(uint32_t t_off, int n, cudaStream_t st) {
        for (int s = 0; s < n; ++s) sweep(t_off + (uint32_t)s, st);
    }
    // A measurement a model defers into the next sweep (which takes it from the state it starts
    // from): has_pending says one is waiting; sweep_pending runs that next sweep (index
    // *clock_dev + t_off) with it; flush_pending takes it with the standalone kernels instead,
    // before anything reads the counts or changes the state.
    virtual bool has_pending() const { return false; }
    virtual void sweep_pending(uint32_t t_off, cudaStream_t st) { sweep(t_off, st); }
    virtual void flush_pending(cudaStream_t st) { (void)st; }
    // snapshot w <- current spins
    virtual void snapshot(int w, cudaStream_t st) = 0;
    // scheduled measurement column u at time tau (snapshots with tw <= tau exist)
    virtual void measure_scheduled(int u, int64_t tau, cudaStream_t st) = 0;
    // immediate measurement at time tau into the model's own scratch counts
    virtual void measure_now(int64_t tau, cudaStream_t st) = 0;
    // copy counts to the host and finalise them into C, q, E (see sg.h for layouts)
    virtual void read_scheduled(int64_t tau, int64_t* C, int64_t* q, int64_t* E,
                                cudaStream_t st) = 0;
    virtual void read_now(int64_t tau, int64_t* C, int64_t* q, int64_t* E, cudaStream_t st) = 0;
    virtual size_t spins_bytes() const = 0;
    virtual void get_spins(void* dst, cudaStream_t st) = 0;
    virtual std::vector<uint32_t> thresholds() const = 0;
    // VB: the colour class of every vertex of graph b (original labels) and the number of
    // classes; empty for a model without a colouring
    virtual std::vector<int32_t> colouring(int b, int* n_colours) const {
        (void)b;
        *n_colours = 0;
        return {};
    }
    // device regions that hold the dynamic state (checkpoint/restore)
    virtual std::vector<std::pair<void*, size_t>> state_regions() = 0;
    // device-side error word (0 = fine), read after synchronisation
    virtual int device_status(cudaStream_t st) { (void)st; return 0; }
    // bytes copied host -> device and device -> host by the model so far
    virtual void transfer_bytes(int64_t& h2d, int64_t& d2h) const {
        h2d = h2d_bytes;
        d2h = d2h_bytes;
    }

    // Window-averaged measurement (set before attach): n_bins windows of sweeps; every sweep
    // inside window m adds its point values into window m's sums.
    virtual void set_windows(int64_t n_bins) = 0;
    // add the point values at time tau into window m
    virtual void measure_window(int m, int64_t tau, cudaStream_t st) = 0;
    // copy the window sums to the host and finalise them into sums of C, q, E; cnt_c[w][m] and
    // cnt_q[m] are the numbers of sweeps measured in window m (with tw[w] <= tau for C)
    virtual void read_windows(const int64_t* cnt_c, const int64_t* cnt_q, int64_t* C, int64_t* q,
                              int64_t* E, cudaStream_t st) = 0;
    int64_t n_bins = 0;

    // Replace the schedule.  Before attach the workspace is re-measured for the new sizes;
    // after attach the sizes are unchanged (checked by the caller) and only the times change.
    virtual void set_schedule(const std::vector<int64_t>& tw_, const std::vector<int64_t>& tm_,
                              bool attached) {
        tw = tw_;
        tm = tm_;
        if (!attached) set_windows(n_bins);
    }

    int n_inst = 1, R = 1, L = 1;
    uint32_t* clock_dev = nullptr;  // device word holding the index of the next sweep
    std::vector<int64_t> tw, tm;
    int64_t launches = 0;
    int64_t h2d_bytes = 0, d2h_bytes = 0;  // bytes copied between host and device so far
};

Model* make_vb_model(const void* graphs, int n_graphs, int n_lanes, int n_replicas, int kernel,
                     const std::vector<int64_t>& tw, const std::vector<int64_t>& tm);
Model* make_sk_batch_model(const void* samples, int n_samples, int n_replicas, int kernel,
                           int block, const std::vector<int64_t>& tw,
                           const std::vector<int64_t>& tm);
Model* make_sk_model(int n, const int8_t* J, int n_replicas, const double* temps, uint64_t seed,
                     int kernel, int block, const std::vector<int64_t>& tw,
                     const std::vector<int64_t>& tm);

// threshold f(x) = min(2^32-1, floor(2^32 exp(x))) in double precision
uint32_t metropolis_threshold(double x);

}  // namespace sg
