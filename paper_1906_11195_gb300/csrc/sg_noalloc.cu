// sg_noalloc.cu -- SK local fields h = J s without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need this computation: a
// host application that hands the library a fixed memory budget and forbids further
// allocations, or a plugin whose process owns every device allocation.  sg_sk_fields_noalloc
// serves them: the caller passes its own input and output buffers, and the intermediate
// tensor-core operand images live in one fixed-size array in the library's static device
// memory, which every GPU that loads the library holds until the process exits.  The call
// waits for its own work (it synchronises the caller's stream before returning).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

#include "../../include/sg.h"
#include "sg_internal.cuh"
#include "sg_model.h"
#include "sk_internal.cuh"

namespace sg {
namespace {

constexpr int kNoallocMaxN = 2048;      // spins (padded to a multiple of 128)
constexpr int kNoallocMaxR = 128;       // replicas
constexpr size_t kJ8Bytes = (size_t)kNoallocMaxN * kNoallocMaxN;        // e4m3 couplings
constexpr size_t kDBytes = (size_t)kNoallocMaxR * kNoallocMaxN;         // e4m3 spins
constexpr size_t kHBytes = (size_t)kNoallocMaxR * kNoallocMaxN * 4;     // int32 fields
constexpr size_t kScratchBytes = kJ8Bytes + kDBytes + kHBytes + 256;    // + status word

// The scratch array.  Host code must not use this name as an address: in host code it is a
// stand-in, and the device address comes from cudaGetSymbolAddress (per device, below).
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_dev[64] = {};  // device address of the scratch, per device ordinal

void* scratch_address() {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) fail(SG_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
        g_scratch_dev[dev] = p;
    }
    return g_scratch_dev[dev];
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        check_cuda(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q),
                   "cudaGetDriverEntryPointByVersion");
        if (q != cudaDriverEntryPointSuccess || !p) fail(SG_ECUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

void tile_map(CUtensorMap* map, void* base, uint64_t inner, uint64_t outer, uint32_t box_outer) {
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner};
    const cuuint32_t box[2] = {128, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box,
                                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(SG_ECUDA, "cuTensorMapEncodeTiled failed");
}

__device__ __forceinline__ uint8_t e4m3_pm1(int v) {
    return v > 0 ? (uint8_t)0x38 : (v < 0 ? (uint8_t)0xB8 : (uint8_t)0x00);
}

// J (int8, n x n) -> e4m3 image (Np x Np, zero padding); spins -> e4m3 (R x Np); fields zeroed
__global__ void k_noalloc_stage(const int8_t* __restrict__ J, const int8_t* __restrict__ s, int n,
                                int Np, int R, uint8_t* J8, uint8_t* D, int32_t* H, int* err) {
    const int64_t tot_j = (int64_t)Np * Np, tot_s = (int64_t)R * Np;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < tot_j;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(k / Np), j = (int)(k % Np);
        J8[k] = (i < n && j < n) ? e4m3_pm1(J[(int64_t)i * n + j]) : (uint8_t)0;
        if (k < tot_s) {
            const int r = (int)(k / Np), c = (int)(k % Np);
            D[k] = c < n ? e4m3_pm1(s[(int64_t)r * n + c]) : (uint8_t)0;
            H[k] = 0;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *err = 0;
}

__global__ void k_noalloc_unpad(const int32_t* __restrict__ H, int n, int Np, int R,
                                int32_t* __restrict__ h) {
    const int64_t tot = (int64_t)R * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < tot;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(k / n), i = (int)(k % n);
        h[k] = H[(int64_t)r * Np + i];
    }
}

// The device that owns p: its ordinal for device memory, -2 for managed memory (usable from
// any device), -1 for anything else (host memory, or no CUDA device at all).  A buffer on
// another GPU would be dereferenced as a peer address, which faults when peer access is not
// enabled, so the caller compares the ordinal with the current device.
int pointer_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (a.type == cudaMemoryTypeManaged) return -2;
    return a.type == cudaMemoryTypeDevice ? a.device : -1;
}

}  // namespace
}  // namespace sg

extern "C" int sg_sk_fields_noalloc(const int8_t* J, const int8_t* s, int32_t n, int32_t n_replicas,
                                    int32_t* h, void* cuda_stream) {
    using namespace sg;
    try {
        if (!J || !s || !h) fail(SG_EINVAL, "null pointer");
        if (n < 2 || n > kNoallocMaxN)
            fail(SG_EINVAL, "n must be in [2, " + std::to_string(kNoallocMaxN) + "]");
        if (n_replicas < 16 || n_replicas > kNoallocMaxR || n_replicas % 16)
            fail(SG_EINVAL, "n_replicas must be a multiple of 16 in [16, " +
                                std::to_string(kNoallocMaxR) + "]");
        const int owner[3] = {pointer_device(J), pointer_device(s), pointer_device(h)};
        for (int o : owner)
            if (o == -1) fail(SG_EINVAL, "J, s and h must be device memory");
        int dev = 0;
        check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
        for (int o : owner)
            if (o >= 0 && o != dev) fail(SG_EINVAL, "J, s and h must be memory of the current device");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
        uint8_t* base = static_cast<uint8_t*>(scratch_address());
        const int Np = (n + 127) / 128 * 128;
        const int R = n_replicas;
        uint8_t* J8 = base;
        uint8_t* D = base + kJ8Bytes;
        int32_t* H = reinterpret_cast<int32_t*>(base + kJ8Bytes + kDBytes);
        int* err = reinterpret_cast<int*>(base + kJ8Bytes + kDBytes + kHBytes);
        k_noalloc_stage<<<304, 256, 0, st>>>(J, s, n, Np, R, J8, D, H, err);
        check_cuda(cudaGetLastError(), "stage launch");
        SkDev d{};
        d.J8 = J8;
        d.D = D;
        d.H = H;
        d.err = err;
        d.N = n;
        d.Np = Np;
        d.R = R;
        CUtensorMap mapJ, mapD;
        tile_map(&mapJ, J8, Np, Np, 128);
        tile_map(&mapD, D, Np, R, R);
        if (sk_field_prepare(128, 128, R) != 0) fail(SG_ECUDA, "cannot configure the field kernel");
        for (int b0 = 0; b0 < Np; b0 += 128) sk_field_update(d, mapJ, mapD, b0, 128, 128, R, 1, st);
        check_cuda(cudaGetLastError(), "field launch");
        k_noalloc_unpad<<<152, 256, 0, st>>>(H, n, Np, R, h);
        check_cuda(cudaGetLastError(), "unpad launch");
        int status = 0;
        check_cuda(cudaMemcpyAsync(&status, err, 4, cudaMemcpyDeviceToHost, st), "status copy");
        check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
        if (status) fail(SG_ETIMEOUT, "a device-side wait expired in the field kernel");
        record_error("");
        return SG_OK;
    } catch (const sg::Error& e) {
        record_error(e.msg);
        return e.code;
    } catch (...) {
        record_error("unknown error");
        return SG_EINVAL;
    }
}
