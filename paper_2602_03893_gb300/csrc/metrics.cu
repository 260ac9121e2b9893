// metrics.cu -- the image metrics the paper tabulates for reconstructions (Results, Table 1): the
// maximum amplitude projection along z, and MSE / PSNR / SSIM of an image against a reference.
// The paper gives no formulas; the common definitions are used: SSIM (Wang et al., 2004) with a
// uniform window of `win` samples per axis, sample (N / (N - 1)) variances and covariance,
// C1 = (0.01 R)^2, C2 = (0.03 R)^2 for the data range R, averaged over the positions whose window
// lies inside the image.  The local sums are separable box filters (x, then y, then z) of five
// fields (x, y, x^2, y^2, x y): fused in shared memory for windows up to 15 (ssim_march_kernel,
// which also sums the squared differences), else one coalesced pass per axis through device memory.
#include "gpair_internal.cuh"

namespace gp {

constexpr int MET_THREADS = 256;
// CTAs of the persistent passes: 4 per SM of the current device.
#define MET_BLOCKS (4 * device_sms())

__global__ void zmap_kernel(const float* __restrict__ vol, int nx, int ny, int nz, float* __restrict__ out) {
    const int64_t nxy = (int64_t)nx * ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nxy; i += (int64_t)gridDim.x * blockDim.x) {
        float m = vol[i];
        for (int z = 1; z < nz; ++z) m = fmaxf(m, vol[(int64_t)z * nxy + i]);
        out[i] = m;
    }
}

// Box sums along x of the five fields of (x, y), valid where p <= ix < nx - p.
__global__ void box_x_kernel(const float* __restrict__ a, const float* __restrict__ b, int nx, int ny, int nz, int p,
                             float* __restrict__ S) {
    const int64_t M = (int64_t)nx * ny * nz;
    for (int row = blockIdx.x; row < ny * nz; row += gridDim.x)
        for (int ix = p + threadIdx.x; ix < nx - p; ix += blockDim.x) {
            const int64_t i = (int64_t)row * nx + ix;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
            for (int d = -p; d <= p; ++d) {
                const float u = a[i + d], v = b[i + d];
                s0 += u; s1 += v; s2 = fmaf(u, u, s2); s3 = fmaf(v, v, s3); s4 = fmaf(u, v, s4);
            }
            S[i] = s0; S[M + i] = s1; S[2 * M + i] = s2; S[3 * M + i] = s3; S[4 * M + i] = s4;
        }
}

// Box sums of the five fields along y (axis 1) or z (axis 2), valid where the window fits on that
// axis (and on the axes summed before).
__global__ void box_yz_kernel(const float* __restrict__ S, int nx, int ny, int nz, int p, int axis,
                              float* __restrict__ T) {
    const int64_t M = (int64_t)nx * ny * nz;
    const int64_t stride = axis == 1 ? nx : (int64_t)nx * ny;
    for (int row = blockIdx.x; row < ny * nz; row += gridDim.x) {
        const int iy = row % ny, iz = row / ny;
        const int c = axis == 1 ? iy : iz, n = axis == 1 ? ny : nz;
        if (c < p || c >= n - p) continue;
        if (axis == 2 && (iy < p || iy >= ny - p)) continue;
        for (int ix = p + threadIdx.x; ix < nx - p; ix += blockDim.x) {
            const int64_t i = (int64_t)row * nx + ix;
            for (int f = 0; f < 5; ++f) {
                float s = 0.f;
                for (int d = -p; d <= p; ++d) s += S[f * M + i + d * stride];
                T[f * M + i] = s;
            }
        }
    }
}

// SSIM at every interior position from the five box sums; FP64 block partials of the sum.
__global__ void __launch_bounds__(MET_THREADS)
ssim_kernel(const float* __restrict__ S, int nx, int ny, int nz, int p, int pz, float invN, float cov, float C1,
            float C2, double* __restrict__ partial) {
    __shared__ double red[MET_THREADS / 32];
    const int64_t M = (int64_t)nx * ny * nz;
    double acc = 0.0;
    for (int row = blockIdx.x; row < ny * nz; row += gridDim.x) {
        const int iy = row % ny, iz = row / ny;
        if (iy < p || iy >= ny - p || iz < pz || iz >= nz - pz) continue;
        for (int ix = p + threadIdx.x; ix < nx - p; ix += blockDim.x) {
            const int64_t i = (int64_t)row * nx + ix;
            const float mx = S[i] * invN, my = S[M + i] * invN;
            const float sxx = cov * (S[2 * M + i] * invN - mx * mx);
            const float syy = cov * (S[3 * M + i] * invN - my * my);
            const float sxy = cov * (S[4 * M + i] * invN - mx * my);
            acc += (double)(((2.f * mx * my + C1) * (2.f * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2)));
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < MET_THREADS / 32; ++k) s += red[k];
        partial[blockIdx.x] = s;
    }
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += partial[k];    // fixed order
        *out = s;
    }
}

// Fused MSE + SSIM, marching along z.  A CTA owns a column of SS_TX x SS_TY output positions and
// a chunk of SS_ZC planes.  Per input plane it stages x and y with a p-voxel halo in x and y,
// box-sums the five fields along x (shared memory), then along y for its own positions, and keeps
// the last 2 pz + 1 such planes in a per-thread ring; an output plane's z box sum adds the ring
// in plane order.  The summation order per position is that of the separable passes above (x, y,
// then z), so every position's SSIM is the same FP32 value; only x and y cross HBM.  Per-thread
// sums of (x - y)^2 over the CTA's own voxels and of SSIM over its interior positions are
// compensated FP32, then FP64 per CTA: partial[2 b] and partial[2 b + 1].
constexpr int SS_TX = 32, SS_TY = 8, SS_ZC = 16, SS_PMAX = 7;
// staged entries per thread: (SS_TY + 2 p)(SS_TX + 2 p) <= 22 * 46 = 1012 <= 4 * 256
constexpr int SS_STAGE = ((SS_TY + 2 * SS_PMAX) * (SS_TX + 2 * SS_PMAX) + 255) / 256;
static_assert(SS_TX * SS_TY == MET_THREADS, "one thread per output column position");

__host__ __device__ __forceinline__ size_t ssim_march_floats(int p, int pz) {
    return (size_t)2 * (SS_TY + 2 * p) * (SS_TX + 2 * p) + (size_t)5 * (SS_TY + 2 * p) * SS_TX +
           (size_t)(2 * pz + 1) * 5 * SS_TY * SS_TX;
}

__global__ void __launch_bounds__(MET_THREADS)
ssim_march_kernel(const float* __restrict__ x, const float* __restrict__ y, int nx, int ny, int nz, int p, int pz,
                  float invN, float cov, float C1, float C2, double* __restrict__ partial) {
    extern __shared__ float ssm[];
    __shared__ double red[2][MET_THREADS / 32];
    const int SW = SS_TX + 2 * p, SH = SS_TY + 2 * p, R = 2 * pz + 1;
    float* sa = ssm;                              // [SH][SW]
    float* sb = sa + SH * SW;                     // [SH][SW]
    float* xb = sb + SH * SW;                     // [5][SH][SS_TX]
    float* ring = xb + 5 * SH * SS_TX;            // [R][5][SS_TY][SS_TX]
    const int tx = threadIdx.x % SS_TX, ty = threadIdx.x / SS_TX;
    const int ncx = (nx + SS_TX - 1) / SS_TX, ncy = (ny + SS_TY - 1) / SS_TY, ncz = (nz + SS_ZC - 1) / SS_ZC;
    const int nitems = ncx * ncy * ncz;
    KahanF ksq, kss;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int cx = item % ncx, cy = (item / ncx) % ncy, cz = item / (ncx * ncy);
        const int X0 = cx * SS_TX, Y0 = cy * SS_TY, Z0 = cz * SS_ZC, Z1 = min(Z0 + SS_ZC, nz);
        const int gx = X0 + tx, gy = Y0 + ty;
        const bool own_xy = gx < nx && gy < ny;
        const bool in_xy = gx >= p && gx < nx - p && gy >= p && gy < ny - p;
        const int zlo = max(Z0 - pz, 0), zhi = min(Z1 - 1 + pz, nz - 1);
        // this thread's staging entries q = threadIdx.x + k MET_THREADS (k < SS_STAGE), loaded one
        // plane ahead into registers so that the loads overlap the previous plane's sums
        float pa[SS_STAGE], pb[SS_STAGE];
        auto load_plane = [&](int zi) {
            const float* xp = x + (int64_t)zi * ny * nx;
            const float* yp = y + (int64_t)zi * ny * nx;
#pragma unroll
            for (int k = 0; k < SS_STAGE; ++k) {
                const int q = threadIdx.x + k * MET_THREADS;
                const int r = q / SW, c = q - r * SW;
                const int ix = X0 - p + c, iy = Y0 - p + r;
                const bool ok = q < SH * SW && ix >= 0 && ix < nx && iy >= 0 && iy < ny;
                const int64_t o = (int64_t)iy * nx + ix;
                pa[k] = ok ? __ldg(xp + o) : 0.f;
                pb[k] = ok ? __ldg(yp + o) : 0.f;
            }
        };
        load_plane(zlo);
        for (int zi = zlo; zi <= zhi; ++zi) {
            __syncthreads();   // the previous plane's readers of sa, sb and xb are done
#pragma unroll
            for (int k = 0; k < SS_STAGE; ++k) {
                const int q = threadIdx.x + k * MET_THREADS;
                if (q < SH * SW) {
                    sa[q] = pa[k];
                    sb[q] = pb[k];
                }
            }
            if (zi < zhi) load_plane(zi + 1);
            __syncthreads();
            if (own_xy && zi >= Z0 && zi < Z1) {
                const float d = sa[(ty + p) * SW + tx + p] - sb[(ty + p) * SW + tx + p];
                ksq.add(d * d);
            }
            for (int q = threadIdx.x; q < SH * SS_TX; q += MET_THREADS) {   // box along x
                const int r = q / SS_TX, c = q - r * SS_TX;
                const float* ra = sa + r * SW + c;
                const float* rb = sb + r * SW + c;
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
                for (int d = 0; d <= 2 * p; ++d) {
                    const float u = ra[d], v = rb[d];
                    s0 += u; s1 += v; s2 = fmaf(u, u, s2); s3 = fmaf(v, v, s3); s4 = fmaf(u, v, s4);
                }
                xb[q] = s0; xb[SH * SS_TX + q] = s1; xb[2 * SH * SS_TX + q] = s2; xb[3 * SH * SS_TX + q] = s3;
                xb[4 * SH * SS_TX + q] = s4;
            }
            __syncthreads();
            float* rslot = ring + (size_t)(zi % R) * 5 * SS_TY * SS_TX + ty * SS_TX + tx;
            for (int f = 0; f < 5; ++f) {                                      // box along y (own position)
                const float* col = xb + (size_t)f * SH * SS_TX + ty * SS_TX + tx;
                float s = 0.f;
                for (int d = 0; d <= 2 * p; ++d) s += col[d * SS_TX];
                rslot[f * SS_TY * SS_TX] = s;
            }
            // output plane zi - pz, once its 2 pz + 1 planes are in the ring (this thread's own entries)
            const int zo = zi - pz;
            if (in_xy && zo >= Z0 && zo < Z1 && zo >= pz && zo < nz - pz) {
                float S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                for (int zz = zo - pz; zz <= zo + pz; ++zz) {
                    const float* slot = ring + (size_t)(zz % R) * 5 * SS_TY * SS_TX + ty * SS_TX + tx;
#pragma unroll
                    for (int f = 0; f < 5; ++f) S[f] += slot[f * SS_TY * SS_TX];
                }
                const float mx = S[0] * invN, my = S[1] * invN;
                const float sxx = cov * (S[2] * invN - mx * mx);
                const float syy = cov * (S[3] * invN - my * my);
                const float sxy = cov * (S[4] * invN - mx * my);
                kss.add(((2.f * mx * my + C1) * (2.f * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2)));
            }
        }
    }
    double a = (double)ksq.s - (double)ksq.c, b = (double)kss.s - (double)kss.c;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][w] = a;
        red[1][w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa2 = 0.0, sb2 = 0.0;
        for (int k = 0; k < MET_THREADS / 32; ++k) {
            sa2 += red[0][k];
            sb2 += red[1][k];
        }
        partial[2 * blockIdx.x] = sa2;
        partial[2 * blockIdx.x + 1] = sb2;
    }
}

// res[0] = sum (x - ref)^2 over all voxels, res[2] = sum of SSIM over the interior positions: each
// thread sums a fixed stride of the CTA partials, then a fixed tree (deterministic).
__global__ void __launch_bounds__(MET_THREADS)
ssim_march_finish_kernel(const double* __restrict__ partial, int n, double* __restrict__ res) {
    __shared__ double sa[MET_THREADS], sb[MET_THREADS];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < n; k += MET_THREADS) {
        a += partial[2 * k];
        b += partial[2 * k + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = MET_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        res[0] = sa[0];
        res[2] = sb[0];
    }
}

size_t ssim_march_partial_doubles() { return 2 * (size_t)MET_BLOCKS; }
int metrics_march_pmax() { return SS_PMAX; }

// cudaErrorNotSupported when the window is wider than the fused kernel handles (caller falls back).
cudaError_t launch_metrics_march(const float* x, const float* y, int nx, int ny, int nz, int win, float range,
                                 double* partial, double* res, cudaStream_t st) {
    const int p = (win - 1) / 2, pz = nz > 1 ? p : 0;
    if (p > SS_PMAX) return cudaErrorNotSupported;
    const double N = nz > 1 ? (double)win * win * win : (double)win * win;
    const size_t sm = ssim_march_floats(p, pz) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(ssim_march_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const float C1 = (0.01f * range) * (0.01f * range), C2 = (0.03f * range) * (0.03f * range);
    ssim_march_kernel<<<MET_BLOCKS, MET_THREADS, sm, st>>>(x, y, nx, ny, nz, p, pz, (float)(1.0 / N),
                                                           (float)(N / (N - 1.0)), C1, C2, partial);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ssim_march_finish_kernel<<<1, MET_THREADS, 0, st>>>(partial, MET_BLOCKS, res);
    return cudaGetLastError();
}

cudaError_t launch_zmap(const float* vol, int nx, int ny, int nz, float* out, cudaStream_t st) {
    zmap_kernel<<<MET_BLOCKS, MET_THREADS, 0, st>>>(vol, nx, ny, nz, out);
    return cudaGetLastError();
}

size_t ssim_scratch_bytes(int64_t M) { return (size_t)M * 10 * sizeof(float) + sizeof(double) * (MET_BLOCKS + 1); }

// out (device): the sum of SSIM over the interior positions.
cudaError_t launch_ssim_sum(const float* x, const float* y, int nx, int ny, int nz, int win, float range, void* scratch,
                            double* out, cudaStream_t st) {
    const int64_t M = (int64_t)nx * ny * nz;
    float* A = static_cast<float*>(scratch);
    float* B = A + 5 * M;
    double* partial = reinterpret_cast<double*>(B + 5 * M);
    const int p = (win - 1) / 2, pz = nz > 1 ? p : 0;
    const int dimsN = nz > 1 ? 3 : 2;
    const double N = dimsN == 3 ? (double)win * win * win : (double)win * win;
    box_x_kernel<<<MET_BLOCKS, MET_THREADS, 0, st>>>(x, y, nx, ny, nz, p, A);
    box_yz_kernel<<<MET_BLOCKS, MET_THREADS, 0, st>>>(A, nx, ny, nz, p, 1, B);
    const float* S = B;
    if (nz > 1) {
        box_yz_kernel<<<MET_BLOCKS, MET_THREADS, 0, st>>>(B, nx, ny, nz, p, 2, A);
        S = A;
    }
    const float C1 = (0.01f * range) * (0.01f * range), C2 = (0.03f * range) * (0.03f * range);
    ssim_kernel<<<MET_BLOCKS, MET_THREADS, 0, st>>>(S, nx, ny, nz, p, pz, (float)(1.0 / N), (float)(N / (N - 1.0)), C1,
                                                    C2, partial);
    sum_partials_kernel<<<1, 32, 0, st>>>(partial, MET_BLOCKS, out);
    return cudaGetLastError();
}

}  // namespace gp
