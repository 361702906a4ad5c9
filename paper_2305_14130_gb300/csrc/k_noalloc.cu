// Allocation-free variant of the consistency-term gradient (the computation of
// efwi_regularization_grad), for callers that cannot let a library allocate
// device memory: applications that hand out all device memory through their
// own pool or fixed budget, or that must not pay for creating a plan (plan
// creation allocates the whole time-stepping workspace) just to evaluate the
// regularization.
//
// The only scratch the computation needs -- one FP64 partial sum of phi_reg
// per thread block -- lives in a file-scope __device__ array of fixed size.
// Every GPU that loads this library holds that array (32 KB) until the
// process exits.  Host code cannot use the array's name as a device address,
// so every call made outside a stream capture looks the address up with
// cudaGetSymbolAddress (with the caller's device current) and remembers it for
// that device; a call made while its stream is being captured cannot look it up
// and uses the remembered address, so the first call on each device must come
// before any stream capture.  A device reset (cudaDeviceReset) or the
// destruction of the primary context unloads the module and may move the
// array: the next uncaptured call looks it up again, but a graph captured
// before the reset holds the old address and must not be replayed.  All calls
// share the array: calls that overlap on the GPU (different streams, or host
// threads racing on one device) race on it.  Every call writes all the
// partials it later reads, so nothing has to be cleared between calls.
#include <cmath>
#include <mutex>
#include <string>

#include "plan.hpp"
#include "reg_pixel.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaBlocks = 4096;                                   // partials held by the scratch array
constexpr long long kNaMaxPixels = (long long)kNaBlocks * kNaThreads;   // one pixel per thread

static __device__ __align__(256) double g_na_partials[kNaBlocks];

__device__ double na_block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

// One pixel per thread; the per-pixel arithmetic of eqs. 8, 11, 12 is
// reg_pixel, the same as the plan's kernel.
__global__ void k_reg_noalloc(const float *m, const float *b, const float *bp, const uint8_t *sink, int ns,
                              long long npix, double eta2, float *g, double *partial) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (p < npix) acc = efwi::reg_pixel(m, b, bp, sink, ns, npix, p, eta2, g);
    acc = na_block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void k_sum_noalloc(const double *partial, int n, double scale, double *out) {
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += partial[k];
    v = na_block_sum(v);
    if (threadIdx.x == 0) *out = scale * v;
}

// Device address of the scratch array on the current device: looked up on every
// call outside a stream capture (so a reloaded module is found again), the last
// address looked up on this device inside a capture.
int scratch_address(cudaStream_t st, double **out, std::string &err) {
    static std::mutex mu;
    static double *addr[128] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        err = std::string("cudaGetDevice failed: ") + cudaGetErrorString(e);
        return EFWI_ERR_CUDA;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;     // cannot tell: do not touch the module
    }
    std::lock_guard<std::mutex> lock(mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_partials);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e);
            return EFWI_ERR_CUDA;
        }
        addr[dev] = static_cast<double *>(p);
    } else if (!addr[dev]) {
        err = "efwi_regularization_grad_noalloc was first called on this device inside a stream capture; "
              "call it once outside any capture first (the scratch address is looked up there)";
        return EFWI_ERR_CUDA;
    }
    *out = addr[dev];
    return EFWI_OK;
}

}  // namespace

extern "C" int efwi_regularization_grad_noalloc(int ns, int nx, int nz, const float *m, const float *b,
                                                const float *bp, const uint8_t *sink, double eta, double *phi_reg,
                                                float *g, efwi_stream_t stream) {
    std::string err;
    if (ns < 1 || nx < 1 || nz < 1) {
        efwi::set_thread_error("ns, nx and nz must be >= 1");
        return EFWI_ERR_ARG;
    }
    if (!m || !b || !bp || !sink || !phi_reg || !g) {
        efwi::set_thread_error("NULL device pointer");
        return EFWI_ERR_ARG;
    }
    if (!std::isfinite(eta)) {
        efwi::set_thread_error("eta must be finite");
        return EFWI_ERR_ARG;
    }
    const long long npix = (long long)nx * nz;
    if (npix > kNaMaxPixels) {
        efwi::set_thread_error("nx * nz = " + std::to_string(npix) +
                               " exceeds the 1048576-pixel limit of the allocation-free entry point "
                               "(its static scratch holds 4096 block partials of 256 pixels); "
                               "use efwi_regularization_grad");
        return EFWI_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double *partial = nullptr;
    int rc = scratch_address(st, &partial, err);
    if (rc != EFWI_OK) {
        efwi::set_thread_error(err);
        return rc;
    }
    const int blocks = (int)((npix + kNaThreads - 1) / kNaThreads);
    k_reg_noalloc<<<blocks, kNaThreads, 0, st>>>(m, b, bp, sink, ns, npix, eta * eta, g, partial);
    k_sum_noalloc<<<1, 1024, 0, st>>>(partial, blocks, 0.5 * eta * eta, phi_reg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        efwi::set_thread_error(std::string("launch failed: ") + cudaGetErrorString(e));
        return EFWI_ERR_CUDA;
    }
    return EFWI_OK;
}
