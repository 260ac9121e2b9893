// step.cu -- elementwise and reduction kernels of one reconstruction iteration (Algorithm 2):
// the nonnegative parameterisation x = (z + eps)^2 and its chain rule (Methods, NPC), the data
// loss |y - b|^2 / N and residual norm reduced in FP64, the Adam update, and the exact line
// search step of the steepest-descent variant.  All HBM-bound; FP64 is used only inside the
// reductions.
#include "gpair_internal.cuh"

namespace gp {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 152 * 4;     // block partials; a second pass sums them in order

__global__ void npc_kernel(const float* __restrict__ z, float* __restrict__ x, int64_t M, int npc, float eps) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        float zi = z[i];
        x[i] = npc ? (zi + eps) * (zi + eps) : zi;
    }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

// r = y - b; delta = scale * r (may alias nothing); partial[blk][0] = sum r^2 (FP64).
__global__ void __launch_bounds__(RED_THREADS)
resid_kernel(const float* __restrict__ y, const float* __restrict__ b, float* __restrict__ delta, float scale,
             int64_t n, double* __restrict__ partial) {
    __shared__ double red[RED_THREADS / 32];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float r = y[i] - b[i];
        acc += (double)r * (double)r;
        delta[i] = scale * r;
    }
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Generic FP64 reductions: partial[blk] = (sum (a - b)^2, sum a * c).  b, c may be NULL.
__global__ void __launch_bounds__(RED_THREADS)
reduce2_kernel(const float* __restrict__ a, const float* __restrict__ b, const float* __restrict__ c, int64_t n,
               double* __restrict__ partial) {
    __shared__ double red[RED_THREADS / 32];
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double ai = a[i];
        double d = b ? ai - (double)b[i] : ai;
        s0 += d * d;
        if (c) s1 += ai * (double)c[i];
    }
    double t0 = block_sum(s0, red);
    double t1 = block_sum(s1, red);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = t0;
        partial[2 * blockIdx.x + 1] = t1;
    }
}

// out[q] = sum_blk partial[blk * stride + q] for q < nq, in block order (deterministic).
__global__ void finish_kernel(const double* __restrict__ partial, int nblk, int stride, int nq,
                              double* __restrict__ out) {
    __shared__ double red[RED_THREADS / 32];
    for (int q = 0; q < nq; ++q) {
        double acc = 0.0;
        for (int k = threadIdx.x; k < nblk; k += blockDim.x) acc += partial[(size_t)k * stride + q];
        double s = block_sum(acc, red);
        if (threadIdx.x == 0) out[q] = s;
        __syncthreads();
    }
}

// Adam on z with gradient g_x (and the NPC chain rule g_z = g_x * 2 (z + eps)).
__global__ void adam_kernel(float* __restrict__ z, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ gx, int64_t M, int npc, float eps, float eta, float b1,
                            float b2, float inv_c1, float inv_sqrt_c2, float adam_eps) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        float zi = z[i];
        float g = gx[i];
        if (npc) g *= 2.f * (zi + eps);
        float mi = b1 * m[i] + (1.f - b1) * g;
        float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        z[i] = zi - eta * (mi * inv_c1) / (sqrtf(vi) * inv_sqrt_c2 + adam_eps);
    }
}

// x <- x - alpha g with alpha = num / den read from device memory (exact line search).
__global__ void ls_update_kernel(float* __restrict__ x, const float* __restrict__ g, int64_t M,
                                 const double* __restrict__ nd) {
    const double den = nd[1];
    const float alpha = den > 0.0 ? (float)(nd[0] / den) : 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        x[i] -= alpha * g[i];
}

// dot(r, Fg) and |Fg|^2 into partials (for the line search).
__global__ void __launch_bounds__(RED_THREADS)
ls_dots_kernel(const float* __restrict__ r, const float* __restrict__ Fg, int64_t n, double* __restrict__ partial) {
    __shared__ double red[RED_THREADS / 32];
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double f = Fg[i];
        s0 += (double)r[i] * f;
        s1 += f * f;
    }
    double t0 = block_sum(s0, red);
    double t1 = block_sum(s1, red);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = t0;
        partial[2 * blockIdx.x + 1] = t1;
    }
}

static int ew_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_npc(const float* z, float* x, int64_t M, int npc, float eps, cudaStream_t st) {
    npc_kernel<<<ew_blocks(M), 256, 0, st>>>(z, x, M, npc, eps);
    return cudaGetLastError();
}

// partial must hold RED_BLOCKS doubles; out[0] = sum r^2.
cudaError_t launch_resid(const float* y, const float* b, float* delta, float scale, int64_t n, double* partial,
                         double* out, cudaStream_t st) {
    resid_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(y, b, delta, scale, n, partial);
    finish_kernel<<<1, RED_THREADS, 0, st>>>(partial, RED_BLOCKS, 1, 1, out);
    return cudaGetLastError();
}

// partial must hold 2 * RED_BLOCKS doubles; out[0..1].
cudaError_t launch_reduce2(const float* a, const float* b, const float* c, int64_t n, double* partial, double* out,
                           cudaStream_t st) {
    reduce2_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(a, b, c, n, partial);
    finish_kernel<<<1, RED_THREADS, 0, st>>>(partial, RED_BLOCKS, 2, 2, out);
    return cudaGetLastError();
}

cudaError_t launch_ls(const float* r, const float* Fg, int64_t n, float* x, const float* g, int64_t M,
                      double* partial, double* nd, cudaStream_t st) {
    ls_dots_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(r, Fg, n, partial);
    finish_kernel<<<1, RED_THREADS, 0, st>>>(partial, RED_BLOCKS, 2, 2, nd);
    ls_update_kernel<<<ew_blocks(M), 256, 0, st>>>(x, g, M, nd);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* z, float* m, float* v, const float* gx, int64_t M, int npc, float eps, float eta,
                        float b1, float b2, float inv_c1, float inv_sqrt_c2, float adam_eps, cudaStream_t st) {
    adam_kernel<<<ew_blocks(M), 256, 0, st>>>(z, m, v, gx, M, npc, eps, eta, b1, b2, inv_c1, inv_sqrt_c2, adam_eps);
    return cudaGetLastError();
}

int red_blocks() { return RED_BLOCKS; }

// Failure-detection self-test: one warp waits on a shared-memory barrier that nothing completes,
// with a bound of `polls` polls; the wait gives up, the timeout goes into the status word and the
// kernel returns normally (no trap, nothing in flight).
__global__ void wait_selftest_kernel(uint32_t polls, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const bool ok = mbar_wait_n(&bar, 0u, polls);
    __syncwarp();
    if (threadIdx.x == 0) {
        if (!ok) set_status(status, DEV_TIMEOUT);
        mbar_inval(&bar);
    }
}

cudaError_t launch_wait_selftest(uint32_t polls, int* status, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(polls, status);
    return cudaGetLastError();
}

}  // namespace gp
