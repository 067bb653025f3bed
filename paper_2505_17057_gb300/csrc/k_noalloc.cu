// k_noalloc.cu -- mmfd_reduce_static: the deterministic FP64 field reduction of mmfd_reduce,
// for callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc/cudaFree at the point of use -- cudaFree
// synchronises the whole device and both can block on the driver, which a caller in the middle
// of an asynchronous pipeline, a custom allocator's own bookkeeping path, or a component held
// to a fixed pre-reserved memory budget cannot afford.  This variant takes its per-block
// partial sums from a fixed file-scope device array instead of a buffer the caller or the
// library allocates.
//
// Scratch: kStaticParts = 1024 doubles (8 KB) in __device__ memory, present on every GPU that
// loads the library until the process exits.  One block reduces up to kElemsPerBlock elements,
// so a call handles at most kStaticParts * kElemsPerBlock = 2^27 elements; larger requests are
// rejected with MMFD_ERR_ARG.  Every call shares the array and overwrites the slots it uses
// (nothing needs to start at zero); two calls that overlap on the GPU (different streams, or
// different threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/mmfd.h"
#include "solver.h"

namespace mmfd {

namespace {

constexpr int kStaticParts = 1024;
constexpr int kStaticThreads = 256;
constexpr long long kElemsPerBlock = 1ll << 17;  // 131072 elements per block

__device__ __align__(256) double g_static_parts[kStaticParts];

__device__ __forceinline__ double combine1(int op, double x, double y) {
    return op == MMFD_RED_MAXABS ? fmax(x, y) : x + y;
}

// Block b reduces elements [b * kElemsPerBlock, min(count, (b + 1) * kElemsPerBlock)) in a
// fixed order and writes its partial into parts[b].
__global__ void __launch_bounds__(kStaticThreads) k_static_parts(const void* __restrict__ field, int dtype,
                                                                  long long count, int op, double* __restrict__ parts) {
    __shared__ double sh[kStaticThreads];
    const long long lo = blockIdx.x * kElemsPerBlock;
    const long long hi = lo + kElemsPerBlock < count ? lo + kElemsPerBlock : count;
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += kStaticThreads) {
        const double v = dtype == MMFD_DT_F64 ? static_cast<const double*>(field)[i]
                                              : (double)static_cast<const float*>(field)[i];
        const double e = op == MMFD_RED_SUM ? v : op == MMFD_RED_MAXABS ? fabs(v) : (isfinite(v) ? 0.0 : 1.0);
        acc = combine1(op, acc, e);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kStaticThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = combine1(op, sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kStaticThreads) k_static_final(const double* __restrict__ parts, int nparts, int op,
                                                                  double* __restrict__ out) {
    __shared__ double sh[kStaticThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kStaticThreads) acc = combine1(op, acc, parts[i]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kStaticThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = combine1(op, sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// Device address of g_static_parts for the current device.  In host code the symbol's name is
// only a host-side stand-in, not a device address, so the address is looked up with the device
// current.  Outside stream capture it is looked up on every call (cheap once the module is
// loaded; after cudaDeviceReset the module is loaded again and the array may move); during
// capture the address cached by the last uncaptured call on that device is used, so the first
// call on a device must come before any capture (MMFD_ERR_STATE otherwise).
constexpr int kMaxDevices = 64;
double* g_parts_addr[kMaxDevices] = {};
std::mutex g_parts_mu;

int static_parts_for_current_device(int dev, cudaStream_t stream, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return set_error(MMFD_ERR_ARG, "device ordinal out of range");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lock(g_parts_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_parts);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        g_parts_addr[dev] = static_cast<double*>(p);
    } else if (!g_parts_addr[dev]) {
        return set_error(MMFD_ERR_STATE, "the first mmfd_reduce_static call on a device must precede stream capture");
    }
    *out = g_parts_addr[dev];
    return MMFD_OK;
}

// field and out must be device memory of the current device (or managed memory): a host
// pointer or another GPU's pointer handed to the kernels would fault the GPU.
int check_device_pointer(const void* p, int dev, const char* name) {
    cudaPointerAttributes pa{};
    cudaError_t e = cudaPointerGetAttributes(&pa, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(MMFD_ERR_ARG, std::string(name) + " is not a device pointer");
    }
    if (pa.type == cudaMemoryTypeManaged) return MMFD_OK;
    if (pa.type != cudaMemoryTypeDevice) return set_error(MMFD_ERR_ARG, std::string(name) + " is not device memory");
    if (pa.device != dev) return set_error(MMFD_ERR_ARG, std::string(name) + " belongs to another device");
    return MMFD_OK;
}

}  // namespace

}  // namespace mmfd

extern "C" int mmfd_reduce_static(const void* field, int dtype, long long count, int what, double* out,
                                  void* stream) {
    using namespace mmfd;
    if (!field || !out) return set_error(MMFD_ERR_ARG, "null argument");
    if (dtype != MMFD_DT_F64 && dtype != MMFD_DT_F32) return set_error(MMFD_ERR_ARG, "dtype must be F64 or F32");
    if (what < MMFD_RED_SUM || what > MMFD_RED_NONFINITE) return set_error(MMFD_ERR_ARG, "unknown reduction");
    if (count < 1) return set_error(MMFD_ERR_ARG, "count must be positive");
    if (count > (long long)kStaticParts * kElemsPerBlock)
        return set_error(MMFD_ERR_ARG, "count exceeds the static scratch capacity of 2^27 elements");
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) return cuda_fail(e0, "cudaGetDevice");
    int rc = check_device_pointer(field, dev, "field");
    if (rc == MMFD_OK) rc = check_device_pointer(out, dev, "out");
    if (rc != MMFD_OK) return rc;
    double* parts = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = static_parts_for_current_device(dev, s, &parts);
    if (rc != MMFD_OK) return rc;
    const int nblocks = (int)((count + kElemsPerBlock - 1) / kElemsPerBlock);
    k_static_parts<<<nblocks, kStaticThreads, 0, s>>>(field, dtype, count, what, parts);
    k_static_final<<<1, kStaticThreads, 0, s>>>(parts, nblocks, what, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "static reduction kernels");
    return MMFD_OK;
}
