// forward_noalloc.cu -- gpair_forward_noalloc: the forward operator for callers that must not
// allocate device memory while they run.
//
// gpair_forward grows a per-stream scratch pool with cudaMalloc the first time it sees a
// problem size.  Some callers cannot accept that: a reconstruction embedded in a host framework
// that owns all device memory through its own arena, or a real-time acquisition loop that has
// reserved its memory up front and must not stall (or fail) on a driver allocation mid-run.  This
// entry point takes its scratch from one file-scope device array of fixed size instead, so it
// never calls cudaMalloc, cudaFree or any allocating library routine.
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "gpair_internal.cuh"

namespace gp {
gpair_status forward_into_scratch(const gpair_gaussians* gi, const gpair_array* ai, float* y, cudaStream_t st,
                                  void* scratch, size_t cap, int* status);
}

namespace {

// 64 MiB per device: enough for the 256 x 256 x 128 Gaussian, 1024-sensor, 4096-sample problem
// (the plan coarsens its slabs to fit).  Every device that loads the library holds this array
// until the process exits.  The first 256 bytes hold the device status word.
constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr size_t kStatusBytes = 256;
static __device__ __align__(256) unsigned char g_forward_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.  The
// symbol's host-side name is only a stand-in; kernels must be given this address.
gpair_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return GPAIR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_forward_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GPAIR_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return GPAIR_OK;
}

// A device-side failure (a bounded wait that ran out) leaves some slab partials stale; make
// that visible in the output rather than returning a plausible-looking signal.
__global__ void poison_on_failure(const int* __restrict__ status, float* __restrict__ y, int64_t n) {
    if (*status == 0) return;
    const float nan = __int_as_float(0x7fc00000);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = nan;
}

}  // namespace

extern "C" gpair_status gpair_forward_noalloc(const gpair_gaussians* g, const gpair_array* arr, float* y,
                                              void* stream) {
    if (!arr || arr->n_sensors <= 0 || arr->n_samples <= 0) return GPAIR_ERR_INVALID_ARG;
    void* base = nullptr;
    gpair_status s = scratch_address(&base);
    if (s != GPAIR_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* status = static_cast<int*>(base);
    // The status word must start at zero; everything else the forward writes before it reads.
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return GPAIR_ERR_CUDA;
    s = gp::forward_into_scratch(g, arr, y, st, static_cast<unsigned char*>(base) + kStatusBytes,
                                 kScratchBytes - kStatusBytes, status);
    if (s != GPAIR_OK) return s;
    const int64_t n = (int64_t)arr->n_sensors * arr->n_samples;
    poison_on_failure<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(status, y, n);
    return cudaGetLastError() == cudaSuccess ? GPAIR_OK : GPAIR_ERR_CUDA;
}
