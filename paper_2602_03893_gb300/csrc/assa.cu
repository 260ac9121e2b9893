// assa.cu -- the paper's discretised operator (Methods, adaptive supersampling alignment;
// Algorithm 1) for grid Gaussians sharing one width.  Each pair's time of flight is snapped to
// the nearest sample of a grid alpha times finer than fs, the pair's mass A / r accumulates at
// that sample, the impulse lines are convolved with the sampled pulse h and decimated back to
// fs.  The adjoint transposes each stage: zero filling, correlation with h, back-projection.
//
// Forward decomposition: as the exact forward (forward.cu), CTA = (slab of bricks, 8 sensors),
// one warp per sensor, bricks streamed through a ring of TMA-filled shared buffers.  Each warp
// keeps its sensor's impulse line over the slab's band on the fine grid in shared memory and
// adds every pair's mass there with a shared-memory atomic; after the slab it convolves and
// decimates the band into the slab's partial row (summed over slabs by slab_reduce_kernel).
// The adds are 32-bit integer adds of the mass in fixed point, which the shared-memory units
// execute at about twice the rate of float adds.  A warp scales its masses by
// q = ASSA_QMAX d_min / max|A|, d_min the sensor's distance to the slab's box, so that each
// scaled mass is below ASSA_QMAX = 2^19 in magnitude, and every ASSA_FLUSH bricks (at most
// 2^12 pairs) it converts the integer band into a float band and clears it: no band value can
// leave the int32 range, and each mass is rounded to 2^-19 of the largest.  A warp whose sensor
// touches the slab's box, or a non-finite max|A|, keeps float adds.
// Adjoint: the correlated residual dconv_j[k] = sum_n h[alpha n - k] delta_j[n] is formed once
// per sensor (assa_dconv_kernel); then one thread per Gaussian gathers dconv at its snapped
// samples over all sensors, Kahan-compensated, and writes its gradient once.
#include <cuda.h>

#include <cmath>
#include <cstring>

#include "gpair_internal.cuh"

namespace gp {

constexpr int ASSA_SPC = 8;
constexpr int ASSA_THREADS = 32 * ASSA_SPC;
constexpr int ASSA_RING = 4;
constexpr int ASSA_ADJ_SC = 32;
constexpr float ASSA_QMAX = 0.99f * 524288.f;      // 0.99 * 2^19: bound of a scaled mass
constexpr int ASSA_FLUSH = 16;                     // bricks per integer band (16 * 256 = 2^12 pairs)

struct AssaSmem {
    float tileA[ASSA_RING][TILE];
    uint64_t full[ASSA_RING];
    int released[ASSA_RING];
    int issued[ASSA_RING];
    int abort;
};
constexpr size_t ASSA_HDR = (sizeof(AssaSmem) + 127) & ~(size_t)127;

// Impulse band of one (slab, sensor) on the fine grid: samples alpha w - K .. alpha (w + LB - 1) + K.
__host__ __device__ __forceinline__ int assa_zb(int LB, int alpha, int K) { return (alpha * LB + 2 * K + 3) & ~3; }

// Snapping by the float representation: for |x| < 2^22, x + 1.5 * 2^23 rounds to the nearest
// integer in the float's mantissa, so its bits minus SNAP_BITS are that integer: round(x), which is
// floor(x + 1/2) except at exact ties (rounded to even there; the oracle bounds tie decisions).
constexpr float SNAP_MAGIC = 12582912.f;           // 1.5 * 2^23
constexpr unsigned SNAP_BITS = 0x4B400000u;         // its bits

// Snapped fine sample of a pair, alpha n0 + round(phi alpha / Delta): base = alpha n0 - SNAP_BITS
// (wrapping).
__device__ __forceinline__ int assa_snap(float phi, float aInvD, unsigned base) {
    return (int)((unsigned)__float_as_int(fmaf(phi, aInvD, SNAP_MAGIC)) + base);
}

// alpha n0, clamped far outside any record (the snapped sample then fails the range tests).
__device__ __forceinline__ int assa_an0(int alpha, int n0) {
    const long long an = (long long)alpha * n0;
    return (int)max(min(an, (long long)(1 << 30)), -(long long)(1 << 30));
}

// max |A| over the amplitudes, as the bits of a non-negative float (ordered like the floats;
// a NaN amplitude gives a NaN).  *out must be zero before the launch.
__global__ void assa_amax_kernel(const float* __restrict__ A, int64_t M, unsigned* __restrict__ out) {
    unsigned m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned)__float_as_int(fabsf(A[i])));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void __launch_bounds__(ASSA_THREADS)
assa_fwd_kernel(GaussDev g, ArrDev a, const SlabInfo* __restrict__ slabs, float* __restrict__ partial,
                int2* __restrict__ rows, int LB, int* status, int use_tma, const __grid_constant__ CUtensorMap tmap,
                const __grid_constant__ AssaTable T, const unsigned* __restrict__ amax_bits) {
    static_assert(BX == 8 && BY == 8 && BZ == 4 && TILE == 256,
                  "lane offsets below assume lane + 32 q -> (lane & 7, (lane >> 3) + 4 (q & 1), q >> 1)");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    AssaSmem& S = *reinterpret_cast<AssaSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int alpha = T.alpha, K = T.K;
    const int ZB = assa_zb(LB, alpha, K);
    float* zb = reinterpret_cast<float*>(smem_raw + ASSA_HDR) + (size_t)warp * 2 * ZB;   // float band
    int* zi = reinterpret_cast<int*>(zb + ZB);                                          // fixed-point band

    const int slab = blockIdx.y;
    const int j = blockIdx.x * ASSA_SPC + warp;
    const bool has_sensor = j < a.Nd;
    const SlabInfo sl = slabs[slab];
    const int nTiles = sl.t_end - sl.t_begin;
    const size_t row = (size_t)slab * a.Nd + (has_sensor ? j : 0);
    float* prow = partial + row * LB;
    const int Nup = alpha * a.Nt;

    // the slab's sample band for this sensor; a.k * sigma covers the pulse half-width plus half
    // a fine step of snapping
    float sx = 0.f, sy = 0.f, sz = 0.f;
    int n_lo = 0, n_hi = -1;
    float qscale = 0.f;                    // 0: float adds
    if (has_sensor) {
        sx = a.xyz[3 * j]; sy = a.xyz[3 * j + 1]; sz = a.xyz[3 * j + 2];
        if (nTiles > 0) {
            double dmin, dmax;
            box_distance(sl, sx, sy, sz, dmin, dmax);
            const float amax = __int_as_float((int)*amax_bits);
            if (amax > 0.f && amax <= 3.0e38f && dmin > 0.0) qscale = (float)((double)ASSA_QMAX * dmin / (double)amax);
            double ks = (double)a.k * sl.smax;
            double lo = floor(((dmin - ks) / a.v - a.t0) * a.fs) - 2.0;
            double hi = ceil(((dmax + ks) / a.v - a.t0) * a.fs) + 2.0;
            if (lo < 0) lo = 0;
            if (hi > a.Nt - 1) hi = a.Nt - 1;
            if (lo <= hi) { n_lo = (int)lo; n_hi = (int)hi; }
        }
    }
    const int w = n_lo & ~3;
    bool active = has_sensor && n_lo <= n_hi;
    if (active && n_hi + 1 - w > LB) {     // cannot happen with the host's band bound
        set_status(status, DEV_CAPACITY);
        n_hi = w + LB - 1;
    }
    if (lane == 0 && has_sensor) rows[row] = make_int2(w, active ? min(LB, a.Nt - w) : 0);
    if (threadIdx.x == 0) {
        S.abort = 0;
        for (int b = 0; b < ASSA_RING; ++b) {
            S.released[b] = 0;
            S.issued[b] = -1;
            mbar_init(&S.full[b], 1);
        }
        fence_mbar_init();
    }
    for (int q = lane; q < ZB; q += 32) {
        zb[q] = 0.f;
        zi[q] = 0;
    }
    const bool fixedp = qscale > 0.f;     // warp-uniform
    const float inv_q = fixedp ? 1.f / qscale : 0.f;
    // integer band -> float band, cleared for the next bricks
    auto flush = [&]() {
        __syncwarp();
        for (int q = lane; q < ZB; q += 32) {
            const int v = zi[q];
            if (v != 0) {
                zb[q] = fmaf((float)v, inv_q, zb[q]);
                zi[q] = 0;
            }
        }
        __syncwarp();
    };
    __syncthreads();

    const bool tma = use_tma != 0;
    auto fill = [&](int TT) {
        const int b = TT % ASSA_RING;
        int tx, ty, tz;
        slab_brick(sl, TT, tx, ty, tz);
        if (tma) {
            if (lane == 0) {
                S.issued[b] = TT;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_expect_tx(&S.full[b], TILE * sizeof(float));
                tma_load_3d(&S.tileA[b][0], &tmap, tx * BX, ty * BY, tz * BZ, &S.full[b]);
            }
        } else {
            for (int q = lane; q < TILE; q += 32) {
                const int gx = tx * BX + (q & (BX - 1)), gy = ty * BY + ((q / BX) & (BY - 1)), gz = tz * BZ + q / (BX * BY);
                const bool ok = gx < g.nx && gy < g.ny && gz < g.nz;
                S.tileA[b][q] = ok ? g.A[((int64_t)gz * g.ny + gy) * g.nx + gx] : 0.f;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.full[b]);
        }
    };
    if (warp == 0)
        for (int TT = 0; TT < ASSA_RING && TT < nTiles; ++TT) fill(TT);

    const float aInvD = (float)alpha * a.invDelta;     // fine samples per metre
    const int kb0 = alpha * w - K;                     // fine sample at zb[0]
    const float h = g.h;
    const float ox = ((float)(lane & 7) - 0.5f * (BX - 1)) * h;
    const float oy0 = ((float)(lane >> 3) - 0.5f * (BY - 1)) * h;
    const float oy1 = ((float)((lane >> 3) + 4) - 0.5f * (BY - 1)) * h;

    PairRef refs;
    int t = 0;
    bool ok = true;
    for (; t < nTiles; ++t) {
        const int b = t % ASSA_RING;
        if (!mbar_wait(&S.full[b], (uint32_t)((t / ASSA_RING) & 1))) {
            ok = false;
            break;
        }
        if (active) {
            if ((t & 31) == 0 && t + lane < nTiles) {
                int tx, ty, tz;
                slab_brick(sl, t + lane, tx, ty, tz);
                refs = make_ref(g.ox + (tx * BX + BX / 2) * (double)g.h, g.oy + (ty * BY + BY / 2) * (double)g.h,
                                g.oz + (tz * BZ + BZ / 2) * (double)g.h, sx, sy, sz, a);
            }
            const int src = t & 31;
            PairRef r;
            r.v0x = __shfl_sync(0xffffffffu, refs.v0x, src);
            r.v0y = __shfl_sync(0xffffffffu, refs.v0y, src);
            r.v0z = __shfl_sync(0xffffffffu, refs.v0z, src);
            r.R0 = __shfl_sync(0xffffffffu, refs.R0, src);
            r.phi0 = __shfl_sync(0xffffffffu, refs.phi0, src);
            r.n0 = __shfl_sync(0xffffffffu, refs.n0, src);
            const unsigned base = (unsigned)assa_an0(alpha, r.n0) - SNAP_BITS;
            const float ax = ox * (2.f * r.v0x + ox);
            const float ay0 = oy0 * (2.f * r.v0y + oy0), ay1 = oy1 * (2.f * r.v0y + oy1);
#pragma unroll
            for (int q = 0; q < TILE / 32; ++q) {
                const float Ai = S.tileA[b][lane + 32 * q];
                const float oz = ((float)(q >> 1) - 0.5f * (BZ - 1)) * h;
                const float num = (ax + ((q & 1) ? ay1 : ay0)) + oz * (2.f * r.v0z + oz);
                float invR, phi;
                pair_phase_num(r, num, invR, phi);
                // snapped fine sample: floor((R / v - t0) alpha fs + 1/2) = alpha n0 + floor(phi alpha / Delta + 1/2)
                const int k = assa_snap(phi, aInvD, base);
                const int kb = k - kb0;
                if (Ai != 0.f && k >= 0 && k < Nup && kb >= 0 && kb < ZB) {
                    if (fixedp)   // round(A / r q): |.| < 2^19, so the float representation gives it
                        atomicAdd(&zi[kb], __float_as_int(fmaf(Ai * invR, qscale, SNAP_MAGIC)) - (int)SNAP_BITS);
                    else
                        atomicAdd(&zb[kb], Ai * invR);
                }
            }
            if (fixedp && (t + 1) % ASSA_FLUSH == 0) flush();
        }
        // release the slot; the warp that releases it last refills it with tile t + ASSA_RING
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = (atomicAdd(&S.released[b], 1) + 1) % ASSA_SPC == 0;
            if (last) __threadfence_block();
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last && t + ASSA_RING < nTiles) fill(t + ASSA_RING);
    }
    if (!ok && lane == 0) {
        set_status(status, DEV_TIMEOUT);
        S.abort = 1;
    }
    __syncthreads();
    if (S.abort) {
        if (tma && threadIdx.x == 0)
            for (int b = 0; b < ASSA_RING; ++b)
                if (S.issued[b] >= 0) mbar_wait(&S.full[b], (uint32_t)((S.issued[b] / ASSA_RING) & 1));
        return;
    }
    if (active) {
        if (fixedp) flush();
        // y[n] = sum_m z[m] h[alpha n - m]; sample n = w + q needs zb[alpha q .. alpha q + 2K]
        const int wend = min(a.Nt, w + LB);
        for (int q = lane; q < wend - w; q += 32) {
            const float* zq = zb + (size_t)alpha * q;
            float y = 0.f;
            for (int tt = 0; tt <= 2 * K; ++tt) y = fmaf(zq[tt], T.hr[tt], y);   // h[alpha n - m] = h[K - tt]
            prow[q] = y;
        }
    }
}

// dconv_j[k] = sum_n h[alpha n - k] delta_j[n], k = 0 .. alpha Nt - 1 (zero filling and the
// correlation with the flipped pulse in one pass).  Block: 256 fine samples of one sensor.
__device__ __forceinline__ int floor_div(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

__global__ void assa_dconv_kernel(const float* __restrict__ delta, int Nt, const __grid_constant__ AssaTable T,
                                  float* __restrict__ dconv) {
    extern __shared__ float sd[];
    const int j = blockIdx.y;
    const int alpha = T.alpha, K = T.K;
    const int Nup = alpha * Nt;
    const int k0 = blockIdx.x * 256;
    const int na = -floor_div(-(k0 - K), alpha);            // ceil((k0 - K) / alpha)
    const int nb = floor_div(k0 + 255 + K, alpha);
    const float* dj = delta + (size_t)j * Nt;
    for (int q = threadIdx.x; q <= nb - na; q += blockDim.x) {
        const int n = na + q;
        sd[q] = (n >= 0 && n < Nt) ? dj[n] : 0.f;
    }
    __syncthreads();
    const int k = k0 + (int)threadIdx.x;
    if (k >= Nup) return;
    const int n1 = -floor_div(-(k - K), alpha), n2 = floor_div(k + K, alpha);
    float acc = 0.f;
    for (int n = n1; n <= n2; ++n) acc = fmaf(T.hr[K - (alpha * n - k)], sd[n - na], acc);
    dconv[(size_t)j * Nup + k] = acc;
}

size_t assa_dconv_smem(const AssaTable& T) { return (size_t)((255 + 2 * T.K) / T.alpha + 3) * sizeof(float); }

// g_i = sum_j dconv_j[k_ij] / r_ij.  One CTA per brick, one thread per Gaussian, all sensors in
// chunks of 32 with FP64 references prepared one chunk ahead by the last warp.
__global__ void __launch_bounds__(TILE)
assa_adj_kernel(GaussDev g, ArrDev a, const float* __restrict__ dconv, const __grid_constant__ AssaTable T,
                float* __restrict__ gA) {
    __shared__ AdjRef refs2[2][ASSA_ADJ_SC];
    const int64_t t = blockIdx.x;
    const int l = threadIdx.x, warp = l >> 5, lane = l & 31;
    const int tx = (int)(t % g.ntx), ty = (int)((t / g.ntx) % g.nty), tz = (int)(t / ((int64_t)g.ntx * g.nty));
    // warp w takes a 4 x 4 x 2 block of the 8 x 8 x 4 brick, so that the snapped positions of its
    // 32 Gaussians for one sensor -- the residual entries it gathers -- stay close together
    static_assert(BX == 8 && BY == 8 && BZ == 4 && TILE == 256, "brick of 8 x 8 x 4, 8 warps");
    const int lx = (l & 3) | (((l >> 5) & 1) << 2), ly = ((l >> 2) & 3) | (((l >> 6) & 1) << 2),
              lz = ((l >> 4) & 1) | (((l >> 7) & 1) << 1);
    const int gx = tx * BX + lx, gy = ty * BY + ly, gz = tz * BZ + lz;
    const bool valid = gx < g.nx && gy < g.ny && gz < g.nz;
    const int64_t i = ((int64_t)gz * g.ny + gy) * g.nx + gx;
    const float dx = ((float)lx - 0.5f * (BX - 1)) * g.h, dy = ((float)ly - 0.5f * (BY - 1)) * g.h,
                dz = ((float)lz - 0.5f * (BZ - 1)) * g.h;
    const double c0x = g.ox + (tx * BX + BX / 2) * (double)g.h;
    const double c0y = g.oy + (ty * BY + BY / 2) * (double)g.h;
    const double c0z = g.oz + (tz * BZ + BZ / 2) * (double)g.h;
    const int alpha = T.alpha;
    const int Nup = alpha * a.Nt;
    const float aInvD = (float)alpha * a.invDelta;
    constexpr int LASTW = TILE / 32 - 1;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    // the shared references carry alpha n0 (clamped) and the sensor's row j alpha Nt of dconv
    auto ref_fine = [&](int j) {
        const PairRef r = make_ref(c0x, c0y, c0z, a.xyz[3 * j], a.xyz[3 * j + 1], a.xyz[3 * j + 2], a);
        return adj_ref(r, (int)((unsigned)assa_an0(alpha, r.n0) - SNAP_BITS), j * Nup);   // see assa_snap
    };
    KahanF kA;                       // across chunks; FP32 within a chunk of 32 sensors
    if (warp == LASTW && lane < min(ASSA_ADJ_SC, a.Nd)) refs2[0][lane] = ref_fine(lane);
    int cur = 0;
    for (int j0 = 0; j0 < a.Nd; j0 += ASSA_ADJ_SC, cur ^= 1) {
        const int nsc = min(ASSA_ADJ_SC, a.Nd - j0);
        __syncthreads();
        if (warp == LASTW && j0 + ASSA_ADJ_SC + lane < a.Nd) refs2[cur ^ 1][lane] = ref_fine(j0 + ASSA_ADJ_SC + lane);
        const AdjRef* refs = refs2[cur];
        if (valid) {
            float acc = 0.f;
#pragma unroll 4
            for (int q = 0; q < nsc; ++q) {
                const AdjRef r = refs[q];
                float invR, phi;
                pair_phase_r(r, dx, dy, dz, d2, invR, phi);
                const int k = assa_snap(phi, aInvD, (unsigned)r.n0);
                if ((unsigned)k < (unsigned)Nup) acc = fmaf(__ldg(dconv + (size_t)(unsigned)(r.row + k)), invR, acc);
            }
            kA.add(acc);
        }
    }
    if (valid) gA[i] = kA.s;
}

// ---- host side -----------------------------------------------------------------------------

size_t assa_fwd_smem(int LB, const AssaTable& T) {
    return ASSA_HDR + (size_t)ASSA_SPC * 2 * assa_zb(LB, T.alpha, T.K) * sizeof(float);
}

// ev (optional): two events recorded immediately before and after the main kernel.  amax: 4 bytes
// of device scratch for max |A|.
cudaError_t launch_assa_forward(const GaussDev& g, const ArrDev& a, const SlabInfo* si, int S, float* partial,
                                int2* rows, int LB, int* status, const CUtensorMap* tmap, const AssaTable& T,
                                unsigned* amax, const cudaEvent_t* ev, cudaStream_t st) {
    static const CUtensorMap zero_map = [] { CUtensorMap z; memset(&z, 0, sizeof(z)); return z; }();
    const size_t smem = assa_fwd_smem(LB, T);
    cudaError_t e = cudaFuncSetAttribute(assa_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(amax, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    assa_amax_kernel<<<4 * device_sms(), 256, 0, st>>>(g.A, g.M, amax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid((a.Nd + ASSA_SPC - 1) / ASSA_SPC, S);
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    assa_fwd_kernel<<<grid, ASSA_THREADS, smem, st>>>(g, a, si, partial, rows, LB, status, tmap != nullptr,
                                                      tmap ? *tmap : zero_map, T, amax);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
    return e;
}

size_t assa_dconv_bytes(const ArrDev& a, const AssaTable& T) { return (size_t)a.Nd * T.alpha * a.Nt * sizeof(float); }

cudaError_t launch_assa_adjoint(const GaussDev& g, const ArrDev& a, const float* delta, float* gA, const AssaTable& T,
                                float* dconv, const cudaEvent_t* ev, cudaStream_t st) {
    dim3 dgrid((T.alpha * a.Nt + 255) / 256, a.Nd);
    assa_dconv_kernel<<<dgrid, 256, assa_dconv_smem(T), st>>>(delta, a.Nt, T, dconv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    assa_adj_kernel<<<(unsigned)g.ntiles, TILE, 0, st>>>(g, a, dconv, T, gA);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
    return e;
}

}  // namespace gp
