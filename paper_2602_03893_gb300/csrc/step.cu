// step.cu -- elementwise and reduction kernels of one reconstruction iteration (Algorithm 2):
// the nonnegative parameterisation x = (z + eps)^2 and its chain rule (Methods, NPC), the data
// loss |y - b|^2 / N and residual norm reduced in FP64, the Adam update, and the exact line
// search step of the steepest-descent variant.  All HBM-bound; FP64 is used only inside the
// reductions.
#include "gpair_internal.cuh"
#include "step_sched.cuh"

#include <atomic>
#include <cmath>

namespace gp {

constexpr int RED_THREADS = 256;
// Block partials of the FP64 reductions: 4 per SM of the current device; a second pass sums them in
// order.
int red_blocks();
#define RED_BLOCKS red_blocks()

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
// Per-step scalars of Algorithm 2 on the device, so that a step's launches do not change from one
// step to the next (and can be replayed as a CUDA graph): the CAWR step size of step t and Adam's
// bias corrections 1 / (1 - b1^(t+1)), 1 / sqrt(1 - b2^(t+1)), the powers kept as running
// products.  One thread; FP64 only for the products (GB300's FP64 pipe is slow, and a chain of
// FP64 pow / cos / divide took ~11 us).  schedule_kernel advances t.
__global__ void schedule_kernel(SchedParams p, StepSched* __restrict__ sd) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int t = sd->t;
    // SGDR: periods T0, T0 T_mult, ...; T_cur counts iterations since the last restart
    const int T0 = p.T0 > 0 ? p.T0 : 1;
    float phase;                                   // T_cur / T_i
    if (p.T_mult <= 1.0) {
        phase = (float)(t % T0) / (float)T0;
    } else {
        double Tcur = t, Ti = T0;
        for (int guard = 0; Tcur >= Ti && guard < 4096; ++guard) {   // O(log t) periods
            Tcur -= Ti;
            Ti *= p.T_mult;
        }
        phase = (float)(Tcur / Ti);
    }
    sd->eta = (float)p.eta_min + 0.5f * (float)(p.eta_max - p.eta_min) * (1.f + cospif(phase));
    const double b1t = sd->b1t * p.beta1, b2t = sd->b2t * p.beta2;   // beta^(t+1)
    sd->b1t = b1t;
    sd->b2t = b2t;
    sd->inv_c1 = 1.f / (float)(1.0 - b1t);
    sd->inv_sqrt_c2 = rsqrtf((float)(1.0 - b2t));
    sd->t = t + 1;
}

__global__ void set_step_kernel(StepSched* __restrict__ sd, int t, double b1t, double b2t) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sd->t = t;
        sd->b1t = b1t;
        sd->b2t = b2t;
    }
}

__global__ void adam_kernel(float* __restrict__ z, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ gx, int64_t M, int npc, float eps, float b1, float b2,
                            float adam_eps, const StepSched* __restrict__ sd) {
    const float eta = sd->eta, inv_c1 = sd->inv_c1, inv_sqrt_c2 = sd->inv_sqrt_c2;
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
    if (b > (int64_t)device_sms() * 32) b = (int64_t)device_sms() * 32;
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

cudaError_t launch_schedule(const SchedParams& p, StepSched* sd, cudaStream_t st) {
    schedule_kernel<<<1, 32, 0, st>>>(p, sd);
    return cudaGetLastError();
}

// t steps taken: the running products are beta^t.
cudaError_t launch_set_step(StepSched* sd, int t, const SchedParams& p, cudaStream_t st) {
    set_step_kernel<<<1, 32, 0, st>>>(sd, t, std::pow(p.beta1, (double)t), std::pow(p.beta2, (double)t));
    return cudaGetLastError();
}

cudaError_t launch_adam(float* z, float* m, float* v, const float* gx, int64_t M, int npc, float eps, float b1,
                        float b2, float adam_eps, const StepSched* sd, cudaStream_t st) {
    adam_kernel<<<ew_blocks(M), 256, 0, st>>>(z, m, v, gx, M, npc, eps, b1, b2, adam_eps, sd);
    return cudaGetLastError();
}

int red_blocks() { return 4 * device_sms(); }

int device_sms() {
    constexpr int MAXDEV = 64;
    static std::atomic<int> cache[MAXDEV];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 1; }
    if (dev < 0 || dev >= MAXDEV) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            cudaGetLastError();
            return 1;
        }
        return n;
    }
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 1;
    }
    cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

// ---- vessel continuity regulariser (Methods: R_VCR = R_H + beta R_TV) on a lattice image --------
// Readings of the unspecified parts: central first differences (x[i+1] - x[i-1]) / 2; second
// differences x[i+1] - 2 x[i] + x[i-1] and the four-point mixed stencil / 4 (counted twice in the
// Frobenius sum, D_pq = D_qp); Neumann boundaries (neighbour indices clamped per axis); unit voxel
// spacing; eps inside each square root.  Image x fastest.

__device__ __forceinline__ int64_t vox(int ix, int iy, int iz, int nx, int ny) {
    return ((int64_t)iz * ny + iy) * nx + ix;
}

// One fused pass marching along z.  A CTA owns a column of VM_TX x VM_TY voxels and a chunk of
// VM_ZC planes.  Per step it stages one plane of x with two voxels of halo in x and y (neighbour
// indices clamped per axis: the Neumann reading) into a ring of three planes, forms the weighted
// fields of the previous plane on the column plus one voxel per side,
//   F_k = m_k (D_k x) / sqrt(sH + eps)  (k = xx, yy, zz, xy, xz, yz; m = 1, 1, 1, 2, 2, 2),
//   F_{6+d} = beta (D_d x) / sqrt(sT + eps),
// sH = sum_{p,q} (D_pq x)^2, sT = sum_d (D_d x)^2, into a ring of three field planes, and adds
// lam (sum_k D_k^T F_k) to g on the plane before that.  (D^T F)[j] sums c F[i] over the stencil
// entries (o, c) and every i whose clamped neighbour i + o is j: inside the volume i = j - o, and
// on a face the clamp adds i = j.  Fields are zero outside the volume, so the gather over j - o
// needs no masks and a face voxel adds only the terms that take j itself.  Only x and g cross
// HBM; the fields stay in shared memory.  The value sum sqrt(sH + eps) + beta sqrt(sT + eps) over
// the CTA's own voxels is compensated FP32 per thread and FP64 per CTA (partial[blockIdx.x]).
constexpr int VM_TX = 32, VM_TY = 8, VM_ZC = 16;
constexpr int VM_XW = VM_TX + 4, VM_XH = VM_TY + 4, VM_XN = VM_XW * VM_XH;   // staged x plane
constexpr int VM_FW = VM_TX + 2, VM_FH = VM_TY + 2, VM_FN = VM_FW * VM_FH;   // field plane
static_assert(VM_TX * VM_TY == RED_THREADS, "one thread per column position");
struct VcrMarchSmem {
    float x[3][VM_XN];
    float F[3][9][VM_FN];
};

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

// Extra terms of (sum_k D_k^T F_k)[j] for a voxel on an edge or corner of the volume.  Along one
// axis the preimages of j under the clamped offset o are j - o (when inside) and j itself when
// j + o falls outside; the gather over j - o with zero fields outside the volume already holds
// the products of the first kind, so this adds every product that takes j itself along at least
// one axis.  Fplane[d + 1] is the field plane at z = jz + d ([9][VM_FN] each).
__device__ __noinline__ float vcr_fold_terms(const float* Fm, const float* F0, const float* Fp, int jx, int jy, int jz,
                                             int nx, int ny, int nz, int X0, int Y0) {
    const float* Fplane[3] = {Fm, F0, Fp};
    float s = 0.f;
    for (int e = 0; e < 27; ++e) {
        const VcrEntry E = c_vcr[e];
        const bool fx = jx + E.ox < 0 || jx + E.ox >= nx, fy = jy + E.oy < 0 || jy + E.oy >= ny,
                   fz = jz + E.oz < 0 || jz + E.oz >= nz;
        if (!(fx || fy || fz)) continue;
        float sum = 0.f;
        for (int m = 1; m < 8; ++m) {          // bit set: that axis takes j itself
            if (((m & 1) && !fx) || ((m & 2) && !fy) || ((m & 4) && !fz)) continue;
            const int px = (m & 1) ? jx : jx - E.ox, py = (m & 2) ? jy : jy - E.oy, pz = (m & 4) ? jz : jz - E.oz;
            // an axis that shifts outside the volume reads a zero field: skip it
            if (px < 0 || px >= nx || py < 0 || py >= ny || pz < 0 || pz >= nz) continue;
            sum += Fplane[pz - jz + 1][E.k * VM_FN + (py - Y0 + 1) * VM_FW + (px - X0 + 1)];
        }
        s = fmaf(E.c, sum, s);
    }
    return s;
}

template <bool GRAD>
__global__ void __launch_bounds__(RED_THREADS, 4)
vcr_march_kernel(const float* __restrict__ x, int nx, int ny, int nz, float beta, float eps, float lam,
                 float* __restrict__ g, double* __restrict__ partial, unsigned item_mul) {
    extern __shared__ __align__(16) unsigned char vcr_smem[];
    VcrMarchSmem& S = *reinterpret_cast<VcrMarchSmem*>(vcr_smem);
    __shared__ double red[RED_THREADS / 32];
    const int tx = threadIdx.x % VM_TX, ty = threadIdx.x / VM_TX;
    const unsigned ncx = (nx + VM_TX - 1) / VM_TX, ncy = (ny + VM_TY - 1) / VM_TY, ncz = (nz + VM_ZC - 1) / VM_ZC;
    const unsigned nitems = ncx * ncy * ncz;                  // < 2^31 (checked on the host)
    // Item k of this CTA is (blockIdx.x + k gridDim.x) item_mul mod nitems, stepped by one add:
    // item_mul is coprime to nitems, so every item is visited once, and the face columns, which
    // carry extra terms, spread over the CTAs.
    const unsigned step = (unsigned)(((unsigned long long)gridDim.x * item_mul) % nitems);
    unsigned it = (unsigned)(((unsigned long long)blockIdx.x * item_mul) % nitems);
    KahanF acc;    // this thread's own voxels; FP64 from the CTA sum on
    constexpr int SY = VM_FW;
    for (unsigned k = blockIdx.x; k < nitems; k += gridDim.x) {
        const unsigned cx = it % ncx, rest = it / ncx;
        const int X0 = (int)cx * VM_TX, Y0 = (int)(rest % ncy) * VM_TY, Z0 = (int)(rest / ncy) * VM_ZC;
        const int Z1 = min(Z0 + VM_ZC, nz);
        it += step;
        if (it >= nitems) it -= nitems;
        const int jx = X0 + tx, jy = Y0 + ty;
        // this thread's staging entries q = threadIdx.x + u RED_THREADS of a plane, loaded one step
        // ahead into registers so that the loads overlap the previous step's work
        constexpr int VM_STAGE = (VM_XN + RED_THREADS - 1) / RED_THREADS;
        float pre[VM_STAGE];
        auto load_plane = [&](int zi) {
            const int zc = min(max(zi, 0), nz - 1);
            const float* xp = x + (int64_t)zc * ny * nx;
#pragma unroll
            for (int u = 0; u < VM_STAGE; ++u) {
                const int q = threadIdx.x + u * RED_THREADS;
                const int a = q % VM_XW, b = q / VM_XW;
                const int ix = min(max(X0 - 2 + a, 0), nx - 1), iy = min(max(Y0 - 2 + b, 0), ny - 1);
                pre[u] = q < VM_XN ? __ldg(xp + (int64_t)iy * nx + ix) : 0.f;
            }
        };
        load_plane(Z0 - 2);
        // step s stages x plane Z0 - 2 + s, forms the fields of plane Z0 - 3 + s (s >= 2) and the
        // gradient of plane Z0 - 4 + s (s >= 4)
        for (int s = 0; Z0 - 4 + s < Z1; ++s) {
            const int zi = Z0 - 2 + s;
            __syncthreads();   // the readers of the slots overwritten below are done
            {
                float* xs = S.x[s % 3];
#pragma unroll
                for (int u = 0; u < VM_STAGE; ++u) {
                    const int q = threadIdx.x + u * RED_THREADS;
                    if (q < VM_XN) xs[q] = pre[u];
                }
            }
            if (Z0 - 4 + s + 1 < Z1) load_plane(zi + 1);
            __syncthreads();
            const int zf = zi - 1;
            if (s >= 2) {
                const float* xm = S.x[(s + 1) % 3];     // plane zf - 1
                const float* x0 = S.x[(s + 2) % 3];     // plane zf
                const float* xq = S.x[s % 3];           // plane zf + 1
                float* Fz = &S.F[s % 3][0][0];
                const bool zin = zf >= 0 && zf < nz;
                const bool zown = zf >= Z0 && zf < Z1;
                for (int q = threadIdx.x; q < VM_FN; q += RED_THREADS) {
                    const int a = q % VM_FW, b = q / VM_FW;
                    const int px = X0 - 1 + a, py = Y0 - 1 + b;
                    const bool inside = zin && px >= 0 && px < nx && py >= 0 && py < ny;
                    const bool own = inside && zown && a >= 1 && a <= VM_TX && b >= 1 && b <= VM_TY;
                    if (!inside) {
                        if (GRAD)
#pragma unroll
                            for (int f = 0; f < 9; ++f) Fz[f * VM_FN + q] = 0.f;
                        continue;
                    }
                    if (!GRAD && !own) continue;
                    const int o = (b + 1) * VM_XW + (a + 1);   // the position in the staged planes
                    const float c0 = x0[o];
                    const float vxp = x0[o + 1], vxm = x0[o - 1];
                    const float vyp = x0[o + VM_XW], vym = x0[o - VM_XW];
                    const float vzp = xq[o], vzm = xm[o];
                    const float d1x = 0.5f * (vxp - vxm), d1y = 0.5f * (vyp - vym), d1z = 0.5f * (vzp - vzm);
                    const float hxx = (vxp - c0) + (vxm - c0), hyy = (vyp - c0) + (vym - c0), hzz = (vzp - c0) + (vzm - c0);
                    const float hxy = 0.25f * ((x0[o + 1 + VM_XW] - x0[o + 1 - VM_XW]) - (x0[o - 1 + VM_XW] - x0[o - 1 - VM_XW]));
                    const float hxz = 0.25f * ((xq[o + 1] - xm[o + 1]) - (xq[o - 1] - xm[o - 1]));
                    const float hyz = 0.25f * ((xq[o + VM_XW] - xm[o + VM_XW]) - (xq[o - VM_XW] - xm[o - VM_XW]));
                    const float sH = hxx * hxx + hyy * hyy + hzz * hzz + 2.f * (hxy * hxy + hxz * hxz + hyz * hyz);
                    const float sT = d1x * d1x + d1y * d1y + d1z * d1z;
                    if (GRAD) {
                        const float wH = rsqrtf(sH + eps), wT = beta * rsqrtf(sT + eps);
                        Fz[0 * VM_FN + q] = wH * hxx;
                        Fz[1 * VM_FN + q] = wH * hyy;
                        Fz[2 * VM_FN + q] = wH * hzz;
                        Fz[3 * VM_FN + q] = 2.f * wH * hxy;
                        Fz[4 * VM_FN + q] = 2.f * wH * hxz;
                        Fz[5 * VM_FN + q] = 2.f * wH * hyz;
                        Fz[6 * VM_FN + q] = wT * d1x;
                        Fz[7 * VM_FN + q] = wT * d1y;
                        Fz[8 * VM_FN + q] = wT * d1z;
                    }
                    if (own) acc.add(sqrtf(sH + eps) + beta * sqrtf(sT + eps));
                }
            }
            if (!GRAD) continue;
            __syncthreads();
            const int jz = zi - 2;
            if (s >= 4 && jz >= Z0 && jx < nx && jy < ny) {
                const float* Fm = &S.F[(s + 1) % 3][0][0];    // fields of plane jz - 1
                const float* F0 = &S.F[(s + 2) % 3][0][0];    // plane jz
                const float* Fp = &S.F[s % 3][0][0];          // plane jz + 1
                const int f0 = (ty + 1) * VM_FW + (tx + 1);
                auto A = [&](const float* P, int f, int d) { return P[f * VM_FN + f0 + d]; };
                // the entries of c_vcr with i = j - o, written out
                float sg = (A(F0, 0, -1) + A(F0, 0, 1)) - 2.f * A(F0, 0, 0);
                sg += (A(F0, 1, -SY) + A(F0, 1, SY)) - 2.f * A(F0, 1, 0);
                sg += (A(Fm, 2, 0) + A(Fp, 2, 0)) - 2.f * A(F0, 2, 0);
                sg += 0.25f * ((A(F0, 3, -1 - SY) - A(F0, 3, -1 + SY)) - (A(F0, 3, 1 - SY) - A(F0, 3, 1 + SY)));
                sg += 0.25f * ((A(Fm, 4, -1) - A(Fp, 4, -1)) - (A(Fm, 4, 1) - A(Fp, 4, 1)));
                sg += 0.25f * ((A(Fm, 5, -SY) - A(Fp, 5, -SY)) - (A(Fm, 5, SY) - A(Fp, 5, SY)));
                sg += 0.5f * (A(F0, 6, -1) - A(F0, 6, 1));
                sg += 0.5f * (A(F0, 7, -SY) - A(F0, 7, SY));
                sg += 0.5f * (A(Fm, 8, 0) - A(Fp, 8, 0));
                const int fxs = jx == 0 ? -1 : (jx == nx - 1 ? 1 : 0);   // outward offset on a face, else 0
                const int fys = jy == 0 ? -1 : (jy == ny - 1 ? 1 : 0);
                const int fzs = jz == 0 ? -1 : (jz == nz - 1 ? 1 : 0);
                const int nf = (fxs != 0) + (fys != 0) + (fzs != 0);
                if (nf == 1 && (fxs ? nx : fys ? ny : nz) > 1) {
                    // one face, axis a with outward offset: the entries whose offset along a is that
                    // offset also take j itself along a (the other axes shift as inside)
                    const float h = 0.25f * (float)(fxs + fys + fzs);
                    if (fxs) sg += A(F0, 0, 0) + h * ((A(F0, 3, -SY) - A(F0, 3, SY)) + (A(Fm, 4, 0) - A(Fp, 4, 0)) + 2.f * A(F0, 6, 0));
                    else if (fys) sg += A(F0, 1, 0) + h * ((A(F0, 3, -1) - A(F0, 3, 1)) + (A(Fm, 5, 0) - A(Fp, 5, 0)) + 2.f * A(F0, 7, 0));
                    else sg += A(F0, 2, 0) + h * ((A(F0, 4, -1) - A(F0, 4, 1)) + (A(F0, 5, -SY) - A(F0, 5, SY)) + 2.f * A(F0, 8, 0));
                } else if (nf != 0) {
                    sg += vcr_fold_terms(Fm, F0, Fp, jx, jy, jz, nx, ny, nz, X0, Y0);
                }
                const int64_t j = vox(jx, jy, jz, nx, ny);
                g[j] = fmaf(lam, sg, g[j]);
            }
        }
    }
    const double tot = block_sum((double)acc.s - (double)acc.c, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

int64_t vcr_items(int nx, int ny, int nz) {
    return (int64_t)((nx + VM_TX - 1) / VM_TX) * ((ny + VM_TY - 1) / VM_TY) * ((nz + VM_ZC - 1) / VM_ZC);
}

// Multiplier of the item permutation: an odd prime that does not divide the item count.
unsigned vcr_item_mul(int nx, int ny, int nz) {
    const int64_t n = vcr_items(nx, ny, nz);
    const int64_t primes[] = {7919, 7927, 7933, 7937, 7949};
    for (int64_t p : primes)
        if (n % p != 0) return p % n == 0 ? 1u : (unsigned)p;
    return 1u;
}

size_t vcr_smem_bytes(bool grad) { return grad ? sizeof(VcrMarchSmem) : sizeof(float) * 3 * VM_XN; }

// value_out (device, may be NULL): R_VCR(x) in FP64.  g (may be NULL): g += lam grad R_VCR(x).
// partial: RED_BLOCKS doubles.
cudaError_t launch_vcr(const float* x, int nx, int ny, int nz, float beta, float eps, float lam, double* partial,
                       double* value_out, float* g, cudaStream_t st) {
    if (vcr_items(nx, ny, nz) >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    cudaError_t e;
    const unsigned mul = vcr_item_mul(nx, ny, nz);
    if (g) {
        const size_t sm = vcr_smem_bytes(true);
        if ((e = cudaFuncSetAttribute(vcr_march_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
            cudaSuccess)
            return e;
        vcr_march_kernel<true><<<RED_BLOCKS, RED_THREADS, sm, st>>>(x, nx, ny, nz, beta, eps, lam, g, partial, mul);
    } else {
        vcr_march_kernel<false><<<RED_BLOCKS, RED_THREADS, vcr_smem_bytes(false), st>>>(x, nx, ny, nz, beta, eps, lam,
                                                                                       nullptr, partial, mul);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (value_out) {
        finish_kernel<<<1, RED_THREADS, 0, st>>>(partial, RED_BLOCKS, 1, 1, value_out);
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
