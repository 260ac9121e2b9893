// metrics.cu -- the image metrics the paper tabulates for reconstructions (Results, Table 1): the
// maximum amplitude projection along z, and MSE / PSNR / SSIM of an image against a reference.
// The paper gives no formulas; the common definitions are used: SSIM (Wang et al., 2004) with a
// uniform window of `win` samples per axis, sample (N / (N - 1)) variances and covariance,
// C1 = (0.01 R)^2, C2 = (0.03 R)^2 for the data range R, averaged over the positions whose window
// lies inside the image.  The local sums are separable box filters (x, then y, then z), each pass
// one coalesced read and write of five fields (x, y, x^2, y^2, x y); HBM-bound.
#include "gpair_internal.cuh"

namespace gp {

constexpr int MET_THREADS = 256;
constexpr int MET_BLOCKS = 152 * 4;

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
