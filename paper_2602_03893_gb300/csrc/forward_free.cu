// forward_free.cu -- the forward operator for free-centre Gaussians (each with its own centre and
// width; Methods, Eq. single_forward with the window |d| <= k sigma_i), with the 32 lanes of a
// warp owning 32 sensors.
//
// Work decomposition.  Gaussians come in tiles of 256 consecutive ones (with a reference point
// and radius per tile, tile_info_soa_kernel) and tiles in slabs (contiguous tile ranges).  A CTA
// owns one slab and NW x 32 sensors.  The CTA stages each tile's Gaussians in shared memory with
// the per-Gaussian constants of the window (offset from the tile reference, A / 2, the
// exponent scale -log2(e) / 2 sigma^2, k sigma / Delta, the positions to walk), double
// buffered.  All lanes then take the same Gaussian: a lane forms its pair's phase from the FP64
// (tile, sensor) reference and the window's first and last samples, and walks the window,
// adding (A / 2R) d_q exp(-d_q^2 / 2 sigma^2) at d_q = d_0 - q Delta into its own signal band,
// laid out [sample][lane] so that the 32 lanes' read-modify-writes fall in 32 banks whatever
// samples they address.  After the slab each lane writes its band as the slab's banded partial
// row (start sample, length); the slab reduction sums the rows per sample in fixed slab order.
// No atomics.  A sensor whose band is longer than the shared-memory band takes several passes
// over the slab, each keeping the next LB samples.
#include <cuda.h>

#include <climits>
#include <cmath>

#include "gpair_internal.cuh"

namespace gp {

constexpr int FF_MAXW = 8;            // warps per CTA, at most
constexpr int FF_THREADS_MAX = FF_MAXW * 32;

// Staged constants of one Gaussian (uniform over the lanes): 8 floats as two float4.
struct FfGauss {
    float4 o;    // dx, dy, dz (offset from the tile reference), |offset|^2
    float4 e;    // A / 2, c2 = -log2(e) / (2 sigma^2), k sigma / Delta, positions to walk (as float)
};
struct FfHdr {
    FfGauss tile[2][TILE];
    int npass;
};
constexpr size_t FF_HDR = (sizeof(FfHdr) + 127) & ~(size_t)127;

__host__ __device__ __forceinline__ size_t ff_smem_bytes(int NW, int LB) { return FF_HDR + (size_t)NW * LB * 32 * 4; }

constexpr float FF_MAGIC = 12582912.0f;     // 1.5 * 2^23: x + MAGIC, rounded up, is MAGIC + ceil(x)
constexpr int FF_MAGIC_BITS = 0x4B400000;

__global__ void __launch_bounds__(FF_THREADS_MAX, 1)
fwd_free_lanes_kernel(GaussDev g, ArrDev a, const TileInfo* __restrict__ ti, const SlabInfo* __restrict__ slabs,
                      float* __restrict__ partial, int2* __restrict__ rows, int PL, int LB) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FfHdr& S = *reinterpret_cast<FfHdr*>(smem_raw);
    const int NW = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* Y = reinterpret_cast<float*>(smem_raw + FF_HDR) + (size_t)warp * LB * 32;   // [LB][32]

    const int slab = blockIdx.y;
    const int j = (blockIdx.x * NW + warp) * 32 + lane;
    const bool has_sensor = j < a.Nd;
    const SlabInfo sl = slabs[slab];
    const int nTiles = sl.t_end - sl.t_begin;
    const size_t row = (size_t)slab * a.Nd + (has_sensor ? j : 0);
    float* prow = partial + row * PL;

    // this lane's samples for the slab: [n_lo, n_hi], band start w a multiple of 4
    float sx = 0.f, sy = 0.f, sz = 0.f;
    int n_lo = 0, n_hi = -1;
    if (has_sensor) {
        sx = a.xyz[3 * j]; sy = a.xyz[3 * j + 1]; sz = a.xyz[3 * j + 2];
        if (nTiles > 0) {
            double dmin, dmax;
            box_distance(sl, sx, sy, sz, dmin, dmax);
            const double ksd = (double)a.k * sl.smax;
            double lo = floor(((dmin - ksd) / a.v - a.t0) * a.fs) - 2.0;
            double hi = ceil(((dmax + ksd) / a.v - a.t0) * a.fs) + 2.0;
            if (lo < 0) lo = 0;
            if (hi > a.Nt - 1) hi = a.Nt - 1;
            if (lo <= hi) { n_lo = (int)lo; n_hi = (int)hi; }
        }
    }
    const int wa = n_lo & ~3;
    const int npass_j = n_lo <= n_hi ? (n_hi + 1 - wa + LB - 1) / LB : 0;
    if (threadIdx.x == 0) S.npass = 0;
    __syncthreads();
    if (has_sensor && npass_j > 0) atomicMax(&S.npass, npass_j);
    // banded row: samples [wa, wa + len) at row positions [0, len)
    if (has_sensor) rows[row] = make_int2(wa, npass_j > 0 ? min(a.Nt, n_hi + 1) - wa : 0);
    __syncthreads();
    const int npass = S.npass;

    const float Delta = a.Delta, invDelta = a.invDelta;
    // staging of tile t into buffer b: the constants of its Gaussians, by all threads of the CTA
    auto stage = [&](int t, int b) {
        const TileInfo r = ti[sl.t_begin + t];
        for (int l = threadIdx.x; l < TILE; l += blockDim.x) {
            const int64_t i = (int64_t)(sl.t_begin + t) * TILE + l;
            FfGauss q;
            if (i < g.M && g.A[i] != 0.f) {
                const float dx = g.cx[i] - r.c0x, dy = g.cy[i] - r.c0y, dz = g.cz[i] - r.c0z;
                const float sg = g.sg[i];
                const float c2 = __fdividef(-0.72134752044448170368f, sg * sg);   // -log2(e) / (2 sigma^2)
                const float ksi = a.k * sg * invDelta;
                q.o = make_float4(dx, dy, dz, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                q.e = make_float4(0.5f * g.A[i], c2, ksi, floorf(2.f * ksi) + 2.f);
            } else {
                q.o = make_float4(0.f, 0.f, 0.f, 0.f);
                q.e = make_float4(0.f, 0.f, 0.f, 0.f);    // zero positions: skipped
            }
            S.tile[b][l] = q;
        }
    };

    for (int pass = 0; pass < npass; ++pass) {
        const int w = wa + pass * LB;
        const bool active = has_sensor && pass < npass_j;
        const int LBe = active ? min(LB, min(a.Nt, n_hi + 1) - w) : 0;     // band entries this pass keeps
        for (int q = 0; q < LB; ++q) Y[q * 32 + lane] = 0.f;
        if (nTiles > 0) stage(0, 0);
        __syncthreads();
        for (int t = 0; t < nTiles; ++t) {
            const int b = t & 1;
            if (t + 1 < nTiles) stage(t + 1, b ^ 1);      // the next tile, while this one is used
            if (active) {
                const TileInfo rt = ti[sl.t_begin + t];
                const PairRef r = ref_doubled(make_ref(rt.c0x, rt.c0y, rt.c0z, sx, sy, sz, a));
                const int ybase = r.n0 - w;                    // band index of sample n0 + m is ybase + m
                // one window: positions to walk Q (0: skip), its first sample's band row y0, the
                // positions [qa, qa + span) this pass keeps (its band, inside the record; none when
                // the window lies wholly in another pass's band), d_0, A / 2R and the exponent scale
                struct Win { int Q, y0, qa, span; float d, wR, c2; };
                auto window = [&](int l) {
                    const FfGauss G = S.tile[b][l];
                    Win w;
                    w.Q = (int)G.e.w;
                    float invR, phi;
                    pair_phase_pre(r, G.o.x, G.o.y, G.o.z, G.o.w, invR, phi);
                    const float tt = phi * invDelta;
                    const float ulo = __fadd_ru(tt - G.e.z, FF_MAGIC);      // MAGIC + first window sample
                    const float uhi = __fadd_rd(tt + G.e.z, FF_MAGIC);      // MAGIC + last window sample
                    const int m0 = __float_as_int(ulo) - FF_MAGIC_BITS;
                    const int cnt = __float_as_int(uhi) - __float_as_int(ulo) + 1;
                    w.d = fmaf(-(ulo - FF_MAGIC), Delta, phi);
                    w.y0 = ybase + m0;
                    w.qa = max(0, -w.y0);
                    w.span = max(0, min(cnt, LBe - w.y0) - w.qa);
                    w.wR = G.e.x * invR;
                    w.c2 = G.e.y;
                    return w;
                };
                // the next Gaussian's window is formed while this one is walked
                Win cur = window(0);
#pragma unroll 1
                for (int l = 0; l < TILE; ++l) {
                    const Win nxt = window(l + 1 < TILE ? l + 1 : l);
                    if (cur.Q > 0) {
                        float d = cur.d;
#pragma unroll 4
                        for (int q = 0; q < cur.Q; ++q) {
                            const float v = cur.wR * d * ex2_approx(d * d * cur.c2);
                            if ((unsigned)(q - cur.qa) < (unsigned)cur.span) Y[(cur.y0 + q) * 32 + lane] += v;
                            d -= Delta;
                        }
                    }
                    cur = nxt;
                }
            }
            __syncthreads();      // tile t's buffer is free; tile t + 1 is staged
        }
        if (active) {      // row positions [pass LB, pass LB + LB): LB and PL are multiples of 4
            float4* dst = reinterpret_cast<float4*>(prow + pass * LB);
            for (int q = 0; q < LBe; q += 4)
                dst[q >> 2] = make_float4(Y[q * 32 + lane], Y[(q + 1) * 32 + lane], Y[(q + 2) * 32 + lane],
                                          Y[(q + 3) * 32 + lane]);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Host side.

size_t fwd_free_smem(int NW, int LB) { return ff_smem_bytes(NW, LB); }

cudaError_t launch_forward_free(const GaussDev& g, const ArrDev& a, const TileInfo* ti, const SlabInfo* si, int S,
                                float* partial, int2* rows, int PL, int LB, int NW, cudaStream_t st) {
    const size_t smem = ff_smem_bytes(NW, LB);
    cudaError_t e = cudaFuncSetAttribute(fwd_free_lanes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.Nd + 32 * NW - 1) / (32 * NW), S);
    fwd_free_lanes_kernel<<<grid, 32 * NW, smem, st>>>(g, a, ti, si, partial, rows, PL, LB);
    return cudaGetLastError();
}

}  // namespace gp
