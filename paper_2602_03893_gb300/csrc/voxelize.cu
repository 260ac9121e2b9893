// voxelize.cu -- Eq. (2) (the Gaussian source field p0) sampled at voxel centres, each
// Gaussian truncated to the box |r_a - c_a| <= k sigma on every axis.
//
// Lattice case (Gaussians on the output lattice, shared sigma): the field is A convolved with
// the 1-D taps exp(-(m h)^2 / 2 sigma^2), |m h| <= k sigma, along x, y and z in turn -- three
// separable gather passes, each one coalesced read and write of the volume (HBM-bound).
// Any other Gaussian set: each Gaussian scatters its separable box of factors into the volume.
#include "gpair_internal.cuh"

namespace gp {

constexpr int VOX_MAXTAP = 64;

struct Taps {
    int mm;                      // taps m = -mm..mm
    float t[2 * VOX_MAXTAP + 1];
};

// out = in convolved with taps along one axis.  Threads run along x, blocks over (y, z) rows,
// so no voxel index is divided and every tap's loads are coalesced across the warp.
constexpr int VOX_THREADS = 256;
template <int AXIS>
__global__ void __launch_bounds__(VOX_THREADS)
vox_pass_kernel(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz, Taps taps) {
    const int ix = blockIdx.x * VOX_THREADS + threadIdx.x;
    if (ix >= nx) return;
    const int64_t stride = AXIS == 0 ? 1 : (AXIS == 1 ? (int64_t)nx : (int64_t)nx * ny);
    for (int iz = blockIdx.z; iz < nz; iz += gridDim.z)
        for (int iy = blockIdx.y; iy < ny; iy += gridDim.y) {
            const int64_t v = ((int64_t)iz * ny + iy) * nx + ix;
            const int c = AXIS == 0 ? ix : (AXIS == 1 ? iy : iz), n = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);
            const int lo = max(-taps.mm, -c), hi = min(taps.mm, n - 1 - c);
            float acc = 0.f;
            for (int m = lo; m <= hi; ++m) acc = fmaf(taps.t[m + taps.mm], __ldg(in + v + m * stride), acc);
            out[v] = acc;
        }
}

// The same pass with the tap count fixed at compile time: the 2 MM + 1 loads of a voxel issue
// together (out-of-volume taps load nothing and add fmaf(t, 0, acc) = acc, so the sum is the
// one above, term for term).
template <int AXIS, int MM>
__global__ void __launch_bounds__(VOX_THREADS)
vox_pass_fixed_kernel(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz, Taps taps) {
    const int ix = blockIdx.x * VOX_THREADS + threadIdx.x;
    if (ix >= nx) return;
    const int64_t stride = AXIS == 0 ? 1 : (AXIS == 1 ? (int64_t)nx : (int64_t)nx * ny);
    for (int iz = blockIdx.z; iz < nz; iz += gridDim.z)
        for (int iy = blockIdx.y; iy < ny; iy += gridDim.y) {
            const int64_t v = ((int64_t)iz * ny + iy) * nx + ix;
            const int c = AXIS == 0 ? ix : (AXIS == 1 ? iy : iz), n = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);
            float val[2 * MM + 1];
#pragma unroll
            for (int m = -MM; m <= MM; ++m)
                val[m + MM] = (unsigned)(c + m) < (unsigned)n ? __ldg(in + v + m * stride) : 0.f;
            float acc = 0.f;
#pragma unroll
            for (int m = 0; m <= 2 * MM; ++m) acc = fmaf(taps.t[m], val[m], acc);
            out[v] = acc;
        }
}

// The y or z pass with VOX_RUN consecutive outputs per thread along the pass axis: they share
// their taps' inputs, so a thread loads VOX_RUN + 2 MM values instead of VOX_RUN (2 MM + 1).
// Each output's sum is the one above, term for term.
constexpr int VOX_RUN = 4;
template <int AXIS, int MM>
__global__ void __launch_bounds__(VOX_THREADS)
vox_pass_run_kernel(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz, Taps taps) {
    static_assert(AXIS == 1 || AXIS == 2, "runs along y or z");
    const int ix = blockIdx.x * VOX_THREADS + threadIdx.x;
    if (ix >= nx) return;
    const int n = AXIS == 1 ? ny : nz;
    const int nruns = (n + VOX_RUN - 1) / VOX_RUN;
    const int64_t stride = AXIS == 1 ? (int64_t)nx : (int64_t)nx * ny;
    // blockIdx.y runs over (run, other axis) pairs, blockIdx.z over the rest when they exceed 65535
    for (int64_t u = blockIdx.y + (int64_t)blockIdx.z * gridDim.y; u < (int64_t)nruns * (AXIS == 1 ? nz : ny);
         u += (int64_t)gridDim.y * gridDim.z) {
        const int run = (int)(u % nruns), other = (int)(u / nruns);
        const int c0 = run * VOX_RUN;
        const int iy = AXIS == 1 ? c0 : other, iz = AXIS == 1 ? other : c0;
        const int64_t v0 = ((int64_t)iz * ny + iy) * nx + ix;
        float val[VOX_RUN + 2 * MM];
#pragma unroll
        for (int k = 0; k < VOX_RUN + 2 * MM; ++k) {
            const int c = c0 - MM + k;
            val[k] = (unsigned)c < (unsigned)n ? __ldg(in + v0 + (int64_t)(k - MM) * stride) : 0.f;
        }
#pragma unroll
        for (int r = 0; r < VOX_RUN; ++r) {
            if (c0 + r >= n) break;
            float acc = 0.f;
#pragma unroll
            for (int m = 0; m <= 2 * MM; ++m) acc = fmaf(taps.t[m], val[r + m], acc);
            out[v0 + (int64_t)r * stride] = acc;
        }
    }
}

// All three passes in one kernel, for taps fixed at compile time.  A CTA owns a column block of
// VF_TX x VF_TY outputs and VF_TZ planes, one thread per (x, y) column, and marches z through the
// VF_TZ + 2 MM input planes it needs: each plane's input patch (with an MM halo in x and y, zero
// outside the volume) is staged in shared memory, convolved along x into a second buffer, then
// along y by each thread for its own column; the last 2 MM + 1 such values stay in registers,
// and once a plane's z neighbours are in, the thread writes its output.  The volume is read once
// from DRAM and written once (the halos come from L2), instead of three reads and writes through
// a scratch volume.  Each output is the same three sums as the separate passes', in the same
// order, so the result is the same.
constexpr int VF_TX = 32, VF_TY = 8, VF_TZ = 16;
constexpr int VF_THREADS = VF_TX * VF_TY;

template <int MM>
__global__ void __launch_bounds__(VF_THREADS, 4)
vox_fused_kernel(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz, Taps taps) {
    constexpr int PX = VF_TX + 2 * MM, PY = VF_TY + 2 * MM, NPATCH = PX * PY;
    constexpr int NLOAD = (NPATCH + VF_THREADS - 1) / VF_THREADS;            // patch values per thread
    constexpr int NXP = (PY * VF_TX + VF_THREADS - 1) / VF_THREADS;          // x-pass outputs per thread
    constexpr int NR = 2 * MM + 1;                                          // taps, and planes in the ring
    __shared__ float P[PY][PX];
    __shared__ float Sx[PY][VF_TX];
    const int t = threadIdx.x, tx = t % VF_TX, ty = t / VF_TX;
    const int x0 = blockIdx.x * VF_TX, y0 = blockIdx.y * VF_TY, z0 = blockIdx.z * VF_TZ;
    const int64_t plane = (int64_t)nx * ny;
    // this thread's patch values of input plane zi (zero outside the volume)
    auto load = [&](int zi, float (&v)[NLOAD]) {
#pragma unroll
        for (int u = 0; u < NLOAD; ++u) {
            const int q = t + u * VF_THREADS;
            const int px = q % PX, py = q / PX;
            const int gx = x0 - MM + px, gy = y0 - MM + py;
            const bool ok = q < NPATCH && (unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny &&
                            (unsigned)zi < (unsigned)nz;
            v[u] = ok ? __ldg(in + zi * plane + (int64_t)gy * nx + gx) : 0.f;
        }
    };
    float pre[NLOAD];
    load(z0 - MM, pre);
    float ring[NR];                          // ring[NR - 1] is the newest plane's value
#pragma unroll
    for (int m = 0; m < NR; ++m) ring[m] = 0.f;
    const bool own = x0 + tx < nx && y0 + ty < ny;
#pragma unroll 1
    for (int i = 0; i < VF_TZ + 2 * MM; ++i) {
        __syncthreads();      // the previous plane's x pass is done with P, its y pass with Sx
#pragma unroll
        for (int u = 0; u < NLOAD; ++u) {
            const int q = t + u * VF_THREADS;
            if (q < NPATCH) P[q / PX][q % PX] = pre[u];
        }
        __syncthreads();
        if (i + 1 < VF_TZ + 2 * MM) load(z0 - MM + i + 1, pre);      // the next plane, in flight meanwhile
#pragma unroll
        for (int u = 0; u < NXP; ++u) {
            const int q = t + u * VF_THREADS;
            if (q < PY * VF_TX) {
                const int r = q / VF_TX, x = q % VF_TX;
                float acc = 0.f;
#pragma unroll
                for (int m = 0; m < NR; ++m) acc = fmaf(taps.t[m], P[r][x + m], acc);
                Sx[r][x] = acc;
            }
        }
        __syncthreads();
        float acc = 0.f;
#pragma unroll
        for (int m = 0; m < NR; ++m) acc = fmaf(taps.t[m], Sx[ty + m][tx], acc);
#pragma unroll
        for (int m = 0; m < NR - 1; ++m) ring[m] = ring[m + 1];
        ring[NR - 1] = acc;                  // the (x, y)-convolved value of plane z0 - MM + i
        if (i >= 2 * MM) {                   // plane zo = z0 + i - 2 MM has all its z neighbours
            const int zo = z0 + i - 2 * MM;
            float o = 0.f;
#pragma unroll
            for (int m = 0; m < NR; ++m) o = fmaf(taps.t[m], ring[m], o);
            if (own && zo < nz) out[zo * plane + (int64_t)(y0 + ty) * nx + x0 + tx] = o;
        }
    }
}

template <int MM>
static void vox_passes_fixed(const float* A, float* vol, float* tmp, const gpair_grid& og, const Taps& taps,
                             dim3 grid, cudaStream_t st) {
    const dim3 fgrid((og.nx + VF_TX - 1) / VF_TX, (og.ny + VF_TY - 1) / VF_TY, (og.nz + VF_TZ - 1) / VF_TZ);
    if (fgrid.y <= 65535 && fgrid.z <= 65535) {
        vox_fused_kernel<MM><<<fgrid, VF_THREADS, 0, st>>>(A, vol, og.nx, og.ny, og.nz, taps);
        return;
    }
    vox_pass_fixed_kernel<0, MM><<<grid, VOX_THREADS, 0, st>>>(A, vol, og.nx, og.ny, og.nz, taps);
    const int64_t gy = (int64_t)((og.ny + VOX_RUN - 1) / VOX_RUN) * og.nz;
    const int64_t gz = (int64_t)((og.nz + VOX_RUN - 1) / VOX_RUN) * og.ny;
    auto rgrid = [&](int64_t units) {
        const unsigned y = (unsigned)(units < 65535 ? units : 65535);
        const int64_t z = (units + y - 1) / y;
        return dim3(grid.x, y, (unsigned)(z < 65535 ? z : 65535));
    };
    vox_pass_run_kernel<1, MM><<<rgrid(gy), VOX_THREADS, 0, st>>>(vol, tmp, og.nx, og.ny, og.nz, taps);
    vox_pass_run_kernel<2, MM><<<rgrid(gz), VOX_THREADS, 0, st>>>(tmp, vol, og.nx, og.ny, og.nz, taps);
}

__global__ void zero_kernel(float* p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0.f;
}

// One thread per Gaussian: scatter A prod_a f_a into the box of voxels within k sigma per axis.
__global__ void vox_scatter_kernel(GaussDev g, gpair_grid og, float k, float* __restrict__ vol) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.M) return;
    const float A = g.A[i];
    if (A == 0.f) return;
    float cx, cy, cz, s;
    if (g.grid) {
        const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / ((int64_t)g.nx * g.ny));
        cx = (float)(g.ox + (ix + 0.5) * (double)g.h);
        cy = (float)(g.oy + (iy + 0.5) * (double)g.h);
        cz = (float)(g.oz + (iz + 0.5) * (double)g.h);
        s = g.sigma;
    } else {
        cx = g.cx[i]; cy = g.cy[i]; cz = g.cz[i]; s = g.sg[i];
    }
    const float half = k * s * (1.f + 1e-6f), c2 = -0.72134752044448170368f / (s * s);
    const float inv = 1.f / og.dx;
    const int xa = max(0, (int)floorf((cx - half - og.ox) * inv - 0.5f)), xb = min(og.nx - 1, (int)ceilf((cx + half - og.ox) * inv - 0.5f));
    const int ya = max(0, (int)floorf((cy - half - og.oy) * inv - 0.5f)), yb = min(og.ny - 1, (int)ceilf((cy + half - og.oy) * inv - 0.5f));
    const int za = max(0, (int)floorf((cz - half - og.oz) * inv - 0.5f)), zb = min(og.nz - 1, (int)ceilf((cz + half - og.oz) * inv - 0.5f));
    for (int iz = za; iz <= zb; ++iz) {
        const float rz = og.oz + (iz + 0.5f) * og.dx - cz;
        if (fabsf(rz) > half) continue;
        const float fz = A * ex2_approx(rz * rz * c2);
        for (int iy = ya; iy <= yb; ++iy) {
            const float ry = og.oy + (iy + 0.5f) * og.dx - cy;
            if (fabsf(ry) > half) continue;
            const float fyz = fz * ex2_approx(ry * ry * c2);
            for (int ix = xa; ix <= xb; ++ix) {
                const float rx = og.ox + (ix + 0.5f) * og.dx - cx;
                if (fabsf(rx) > half) continue;
                atomicAdd(&vol[((int64_t)iz * og.ny + iy) * og.nx + ix], fyz * ex2_approx(rx * rx * c2));
            }
        }
    }
}

static int vox_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)device_sms() * 32) b = (int64_t)device_sms() * 32;
    return (int)(b < 1 ? 1 : b);
}

bool vox_is_lattice(const GaussDev& g, const gpair_grid& og) {
    return g.grid && og.nx == g.nx && og.ny == g.ny && og.nz == g.nz && og.dx == g.h &&
           (double)og.ox == g.ox && (double)og.oy == g.oy && (double)og.oz == g.oz;
}

// tmp: scratch volume of the same size (lattice case).
cudaError_t launch_voxelize(const GaussDev& g, const gpair_grid& og, float k, float* vol, float* tmp, cudaStream_t st) {
    const int64_t nv = (int64_t)og.nx * og.ny * og.nz;
    if (vox_is_lattice(g, og)) {
        Taps taps;
        const double half = (double)k * g.sigma;
        int mm = (int)floor(half / g.h * (1.0 + 1e-9));
        if (mm > VOX_MAXTAP) return cudaErrorInvalidValue;
        taps.mm = mm;
        for (int m = -mm; m <= mm; ++m) {
            double r = m * (double)g.h;
            taps.t[m + mm] = (float)exp(-r * r / (2.0 * (double)g.sigma * g.sigma));
        }
        const dim3 grid((og.nx + VOX_THREADS - 1) / VOX_THREADS, og.ny < 65535 ? og.ny : 65535,
                        og.nz < 65535 ? og.nz : 65535);
        switch (mm) {
            case 1: vox_passes_fixed<1>(g.A, vol, tmp, og, taps, grid, st); break;
            case 2: vox_passes_fixed<2>(g.A, vol, tmp, og, taps, grid, st); break;
            case 3: vox_passes_fixed<3>(g.A, vol, tmp, og, taps, grid, st); break;
            case 4: vox_passes_fixed<4>(g.A, vol, tmp, og, taps, grid, st); break;
            case 5: vox_passes_fixed<5>(g.A, vol, tmp, og, taps, grid, st); break;
            case 6: vox_passes_fixed<6>(g.A, vol, tmp, og, taps, grid, st); break;
            default:
                vox_pass_kernel<0><<<grid, VOX_THREADS, 0, st>>>(g.A, vol, og.nx, og.ny, og.nz, taps);
                vox_pass_kernel<1><<<grid, VOX_THREADS, 0, st>>>(vol, tmp, og.nx, og.ny, og.nz, taps);
                vox_pass_kernel<2><<<grid, VOX_THREADS, 0, st>>>(tmp, vol, og.nx, og.ny, og.nz, taps);
        }
        return cudaGetLastError();
    }
    zero_kernel<<<vox_blocks(nv), 256, 0, st>>>(vol, nv);
    vox_scatter_kernel<<<(unsigned)((g.M + 255) / 256), 256, 0, st>>>(g, og, k, vol);
    return cudaGetLastError();
}

}  // namespace gp
