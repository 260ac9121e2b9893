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

// ---- vessel continuity regulariser (Methods: R_VCR = R_H + beta R_TV) on a lattice image --------
// Readings of the unspecified parts: central first differences (x[i+1] - x[i-1]) / 2; second
// differences x[i+1] - 2 x[i] + x[i-1] and the four-point mixed stencil / 4 (counted twice in the
// Frobenius sum, D_pq = D_qp); Neumann boundaries (neighbour indices clamped per axis); unit voxel
// spacing; eps inside each square root.  Image x fastest.

__device__ __forceinline__ int64_t vox(int ix, int iy, int iz, int nx, int ny) {
    return ((int64_t)iz * ny + iy) * nx + ix;
}

// Pass 1: per voxel the derivative terms and the weighted fields
//   F_k = m_k (D_k x) / sqrt(sH + eps)  (k = xx, yy, zz, xy, xz, yz; m = 1, 1, 1, 2, 2, 2),
//   F_{6+d} = beta (D_d x) / sqrt(sT + eps),
// sH = sum_{p,q} (D_pq x)^2, sT = sum_d (D_d x)^2; partial[blk] = sum sqrt(sH + eps) + beta sqrt(sT + eps).
__global__ void __launch_bounds__(RED_THREADS)
vcr_fields_kernel(const float* __restrict__ x, int nx, int ny, int nz, float beta, float eps, float* __restrict__ F,
                  double* __restrict__ partial) {
    __shared__ double red[RED_THREADS / 32];
    const int64_t M = (int64_t)nx * ny * nz;
    double acc = 0.0;
    // blocks stride over (y, z) rows, threads over x: no per-voxel index division
    for (int row = blockIdx.x; row < ny * nz; row += gridDim.x)
    for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
        const int iy = row % ny, iz = row / ny;
        const int64_t i = (int64_t)row * nx + ix;
        const int xm = max(ix - 1, 0), xp = min(ix + 1, nx - 1);
        const int ym = max(iy - 1, 0), yp = min(iy + 1, ny - 1);
        const int zm = max(iz - 1, 0), zp = min(iz + 1, nz - 1);
        auto at = [&](int a, int b, int c) { return __ldg(x + vox(a, b, c, nx, ny)); };
        const float c0 = x[i];
        const float vxp = at(xp, iy, iz), vxm = at(xm, iy, iz);
        const float vyp = at(ix, yp, iz), vym = at(ix, ym, iz);
        const float vzp = at(ix, iy, zp), vzm = at(ix, iy, zm);
        const float d1x = 0.5f * (vxp - vxm), d1y = 0.5f * (vyp - vym), d1z = 0.5f * (vzp - vzm);
        const float hxx = (vxp - c0) + (vxm - c0), hyy = (vyp - c0) + (vym - c0), hzz = (vzp - c0) + (vzm - c0);
        const float hxy = 0.25f * ((at(xp, yp, iz) - at(xp, ym, iz)) - (at(xm, yp, iz) - at(xm, ym, iz)));
        const float hxz = 0.25f * ((at(xp, iy, zp) - at(xp, iy, zm)) - (at(xm, iy, zp) - at(xm, iy, zm)));
        const float hyz = 0.25f * ((at(ix, yp, zp) - at(ix, yp, zm)) - (at(ix, ym, zp) - at(ix, ym, zm)));
        const float sH = hxx * hxx + hyy * hyy + hzz * hzz + 2.f * (hxy * hxy + hxz * hxz + hyz * hyz);
        const float sT = d1x * d1x + d1y * d1y + d1z * d1z;
        const float rH = sqrtf(sH + eps), rT = sqrtf(sT + eps);
        const float wH = 1.f / rH, wT = beta / rT;
        F[i] = wH * hxx;
        F[M + i] = wH * hyy;
        F[2 * M + i] = wH * hzz;
        F[3 * M + i] = 2.f * wH * hxy;
        F[4 * M + i] = 2.f * wH * hxz;
        F[5 * M + i] = 2.f * wH * hyz;
        F[6 * M + i] = wT * d1x;
        F[7 * M + i] = wT * d1y;
        F[8 * M + i] = wT * d1z;
        acc += (double)rH + (double)beta * (double)rT;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Stencil entries of the nine operators: field k, neighbour offset, coefficient.
struct VcrEntry {
    signed char k, ox, oy, oz;
    float c;
};
__constant__ VcrEntry c_vcr[27] = {
    {0, 1, 0, 0, 1.f}, {0, 0, 0, 0, -2.f}, {0, -1, 0, 0, 1.f},
    {1, 0, 1, 0, 1.f}, {1, 0, 0, 0, -2.f}, {1, 0, -1, 0, 1.f},
    {2, 0, 0, 1, 1.f}, {2, 0, 0, 0, -2.f}, {2, 0, 0, -1, 1.f},
    {3, 1, 1, 0, .25f}, {3, 1, -1, 0, -.25f}, {3, -1, 1, 0, -.25f}, {3, -1, -1, 0, .25f},
    {4, 1, 0, 1, .25f}, {4, 1, 0, -1, -.25f}, {4, -1, 0, 1, -.25f}, {4, -1, 0, -1, .25f},
    {5, 0, 1, 1, .25f}, {5, 0, 1, -1, -.25f}, {5, 0, -1, 1, -.25f}, {5, 0, -1, -1, .25f},
    {6, 1, 0, 0, .5f}, {6, -1, 0, 0, -.5f},
    {7, 0, 1, 0, .5f}, {7, 0, -1, 0, -.5f},
    {8, 0, 0, 1, .5f}, {8, 0, 0, -1, -.5f},
};

// Coordinates i in [0, n) with clamp(i + o) == j (o in {-1, 0, 1}): at most two.
__device__ __forceinline__ int vcr_preimage(int j, int o, int n, int* out) {
    int c = 0;
    for (int i = j - o - 1; i <= j - o + 1; ++i)
        if (i >= 0 && i < n && min(max(i + o, 0), n - 1) == j) out[c++] = i;
    return c;
}

// Pass 2: g[j] += lam (sum_k D_k^T F_k)[j].  (D^T F)[j] = sum over the stencil entries (o, c) of
// c F[i] over every i whose clamped neighbour i + o is j; inside the volume that is i = j - o.
__global__ void __launch_bounds__(RED_THREADS, 4)
vcr_grad_kernel(const float* __restrict__ F, int nx, int ny, int nz, float lam, float* __restrict__ g) {
    const int64_t M = (int64_t)nx * ny * nz;
    for (int row = blockIdx.x; row < ny * nz; row += gridDim.x)
    for (int jx = threadIdx.x; jx < nx; jx += blockDim.x) {
        const int jy = row % ny, jz = row / ny;
        const int64_t j = (int64_t)row * nx + jx;
        float acc = 0.f;
        if (jx > 0 && jx < nx - 1 && jy > 0 && jy < ny - 1 && jz > 0 && jz < nz - 1) {
#pragma unroll
            for (int e = 0; e < 27; ++e) {
                const VcrEntry E = c_vcr[e];
                acc = fmaf(E.c, __ldg(F + E.k * M + (j - (E.ox + (int64_t)E.oy * nx + (int64_t)E.oz * nx * ny))), acc);
            }
        } else {
            for (int e = 0; e < 27; ++e) {
                const VcrEntry E = c_vcr[e];
                int px[2], py[2], pz[2];
                const int cx = vcr_preimage(jx, E.ox, nx, px), cy = vcr_preimage(jy, E.oy, ny, py),
                          cz = vcr_preimage(jz, E.oz, nz, pz);
                float s = 0.f;
                for (int a = 0; a < cx; ++a)
                    for (int b = 0; b < cy; ++b)
                        for (int c = 0; c < cz; ++c) s += __ldg(F + E.k * M + vox(px[a], py[b], pz[c], nx, ny));
                acc = fmaf(E.c, s, acc);
            }
        }
        g[j] = fmaf(lam, acc, g[j]);
    }
}

// value_out (device, may be NULL): R_VCR(x) in FP64.  g (may be NULL): g += lam grad R_VCR(x).
// F: 9 M floats of scratch; partial: RED_BLOCKS doubles.
cudaError_t launch_vcr(const float* x, int nx, int ny, int nz, float beta, float eps, float lam, float* F,
                       double* partial, double* value_out, float* g, cudaStream_t st) {
    vcr_fields_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(x, nx, ny, nz, beta, eps, F, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (value_out) {
        finish_kernel<<<1, RED_THREADS, 0, st>>>(partial, RED_BLOCKS, 1, 1, value_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (g) {
        vcr_grad_kernel<<<RED_BLOCKS * 8, RED_THREADS, 0, st>>>(F, nx, ny, nz, lam, g);
        e = cudaGetLastError();
    }
    return e;
}

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
