// lbm_noalloc.cu -- lbm_conservation_noalloc: the global mass and momentum sums
// over a caller's stored distributions, for callers that cannot allocate device
// memory at all.
//
// Who needs this: code that runs where a cudaMalloc is not allowed or not safe --
// a plugin inside a host application whose framework owns every byte of device
// memory through its own pool, a process whose memory is already fully reserved
// by another allocator, or a latency-critical loop in which an allocation (which
// may synchronise the device) is forbidden.  lbm_conservation needs a solver and
// its caller-allocated workspace; this entry point needs neither.
//
// Its scratch (one FP64 partial sum per z-plane and value, plus the final four
// sums) lives in the file-scope device array below, of a fixed size.  Every GPU
// on which the library's kernels are loaded holds this array (about 128 KiB)
// until the process exits.  Under CUDA's lazy module loading (the default since
// CUDA 12.2) that memory is committed at the first call on each device, not when
// the library is loaded, so a caller whose device memory another allocator will
// reserve should make one call early.  Host code must not pass the array's name
// to a kernel: on the host the name is only a stand-in, not a device address.
// The device address comes from cudaGetSymbolAddress with the device current.
// The first call on a device does this set-up; make it before any stream
// capture.  Later calls look the address up again (a cheap host query), so that
// a device reset between calls, after which the module and its array may be
// loaded at a new address, is harmless; a call on a capturing stream reuses the
// address found by the last call on that device.
//
// All calls share the one array, and it keeps the contents of the last call.
// Each call first writes every slot it later reads (nothing accumulates across
// calls), so no clearing is needed; calls whose work overlaps on the GPU (on
// different streams, or from several host threads) race on the array and must
// be serialised by the caller.
#include <cuda_runtime.h>

#include <math.h>

#include <mutex>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {
namespace {

constexpr int kNoallocMaxPlanes = 4096;  // largest nz this entry point accepts
constexpr int kNoallocThreads = kReduceThreads;
constexpr int kMaxDevices = 64;
// block_reduce_store sizes its shared array for kReduceThreads threads per block
static_assert(kNoallocThreads == kReduceThreads, "plane_sums_kernel runs the shared block reduction");

static __device__ __align__(256) double g_noalloc_scratch[kNoallocMaxPlanes * 4 + 4];

std::mutex g_addr_mutex;
double *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  Outside stream capture it is
// looked up on every call (a device reset may move the array); on a capturing stream the
// address found by the last call on this device is reused.
cudaError_t scratch_address(cudaStream_t stream, double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (cap == cudaStreamCaptureStatusNone || !g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// One block per z-plane: sums of rho and rho u over that plane, written to the
// plane's own four slots (no accumulation into earlier contents).
template <class LT, class ST>
__global__ void __launch_bounds__(kNoallocThreads) plane_sums_kernel(const typename ST::S *__restrict__ src,
                                                                     long long plane_cells, long long P, double rho0,
                                                                     double *__restrict__ partials) {
    double acc[LT::Q];
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) acc[i] = 0.0;
    const long long base = (long long)blockIdx.x * plane_cells;
    long long n = 0;
    for (long long k = threadIdx.x; k < plane_cells; k += blockDim.x) {
#pragma unroll
        for (int i = 0; i < LT::Q; ++i) acc[i] += double(decode<ST>(src[(long long)i * P + base + k], QScale{}, i));
        ++n;
    }
    double v[4] = {double(n) * rho0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < LT::Q; ++i) {
        const double gsum = weight<LT>(i) * acc[i];  // stored values are scaled by 1/w_i
        v[0] += gsum;
#pragma unroll
        for (int a = 0; a < 3; ++a) v[1 + a] += double(vel<LT>(i, a)) * gsum;
    }
    block_reduce_store<4>(v, partials);
}

template <class LT, class ST>
cudaError_t launch_plane_sums(const void *src, int nx, int ny, int nz, double rho0, double *scratch, double *out,
                              cudaStream_t stream) {
    const long long plane = (long long)nx * ny;
    plane_sums_kernel<LT, ST><<<nz, kNoallocThreads, 0, stream>>>(static_cast<const typename ST::S *>(src), plane,
                                                                   plane * nz, rho0, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    final_reduce_kernel<4><<<1, 4 * 32, 0, stream>>>(scratch, nz, out);
    return cudaGetLastError();
}

template <class LT>
cudaError_t dispatch_storage(lbm_storage st, const void *src, int nx, int ny, int nz, double rho0, double *scratch,
                             double *out, cudaStream_t stream) {
    switch (st) {
    case LBM_STORE_F32: return launch_plane_sums<LT, StoreF32>(src, nx, ny, nz, rho0, scratch, out, stream);
    case LBM_STORE_F16: return launch_plane_sums<LT, StoreF16>(src, nx, ny, nz, rho0, scratch, out, stream);
    case LBM_STORE_BF16: return launch_plane_sums<LT, StoreBF16>(src, nx, ny, nz, rho0, scratch, out, stream);
    case LBM_STORE_F64: return launch_plane_sums<LT, StoreF64>(src, nx, ny, nz, rho0, scratch, out, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_conservation_noalloc(lbm_lattice lattice, lbm_storage storage, const int64_t dims[3],
                                               double rho0, const void *distributions, double out[4], lbm_mem out_mem,
                                               void *cuda_stream) {
    if (!dims || !distributions || !out) return set_error(LBM_ERR_INVALID_ARG, "dims, distributions and out are required");
    if (out_mem != LBM_MEM_HOST && out_mem != LBM_MEM_DEVICE) return set_error(LBM_ERR_INVALID_ARG, "bad lbm_mem");
    if (storage == LBM_STORE_Q16)
        return set_error(LBM_ERR_UNSUPPORTED, "the fixed-point storage needs its range: use lbm_conservation");
    if (has_reference_planes(storage))
        return set_error(LBM_ERR_UNSUPPORTED, "the reference-velocity storage forms: use lbm_conservation");
    if (storage != LBM_STORE_F32 && storage != LBM_STORE_F16 && storage != LBM_STORE_BF16 && storage != LBM_STORE_F64)
        return set_error(LBM_ERR_UNSUPPORTED, "unknown storage");
    // the same per-dimension limits as lbm_create (each side >= max|c|, nx and ny <= 2^24,
    // nz == 1 for D2Q9, fewer than 2^31 cells), checked before any product is formed
    const std::string dp = dims_check(lattice, dims);
    if (!dp.empty()) return set_error(LBM_ERR_INVALID_ARG, ("lbm_conservation_noalloc: dims: " + dp).c_str());
    if (dims[2] > kNoallocMaxPlanes)
        return set_error(LBM_ERR_INVALID_ARG,
                         "lbm_conservation_noalloc: nz exceeds the static scratch limit of 4096 z-planes");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    double *scratch = nullptr;
    cudaError_t e = scratch_address(stream, &scratch);
    if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
    double *result = out_mem == LBM_MEM_DEVICE ? out : scratch + kNoallocMaxPlanes * 4;
    const int nx = int(dims[0]), ny = int(dims[1]), nz = int(dims[2]);
    switch (lattice) {
    case LBM_D2Q9: e = dispatch_storage<D2Q9>(storage, distributions, nx, ny, nz, rho0, scratch, result, stream); break;
    case LBM_D3Q15: e = dispatch_storage<D3Q15>(storage, distributions, nx, ny, nz, rho0, scratch, result, stream); break;
    case LBM_D3Q19: e = dispatch_storage<D3Q19>(storage, distributions, nx, ny, nz, rho0, scratch, result, stream); break;
    case LBM_D3Q27: e = dispatch_storage<D3Q27>(storage, distributions, nx, ny, nz, rho0, scratch, result, stream); break;
    case LBM_D3Q39: e = dispatch_storage<D3Q39>(storage, distributions, nx, ny, nz, rho0, scratch, result, stream); break;
    default: return set_error(LBM_ERR_INVALID_ARG, "unknown lattice");
    }
    if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
    if (out_mem == LBM_MEM_HOST) {
        e = cudaMemcpyAsync(out, result, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return set_error(LBM_ERR_CUDA, cudaGetErrorString(e));
        for (int q = 0; q < 4; ++q)
            if (!isfinite(out[q]))
                return set_error(LBM_ERR_NONFINITE, "conservation sum is not finite");
    }
    return LBM_OK;
}
