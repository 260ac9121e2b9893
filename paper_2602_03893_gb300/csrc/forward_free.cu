// forward_free.cu -- the forward operator for free-centre Gaussians (each with its own centre and
// width; Methods, Eq. single_forward with the window |d| <= k sigma_i), with the 32 lanes of a
// warp owning 32 sensors.
//
// Work decomposition.  Gaussians come in tiles of 256 consecutive ones (with a reference point
// and radius per tile, tile_info_soa_kernel) and tiles in slabs (contiguous tile ranges).  A CTA
// owns one slab and NW x 32 sensors.  The CTA stages each tile's Gaussians in shared memory with
// the per-Gaussian constants of the window (offset from the tile reference, the scaled weight
// A / 2 sc, the phase scale sc = sqrt(log2(e) / 2) / sigma, k sigma / Delta, the sample pairs to
// walk), double buffered.  All lanes then take the same Gaussian: a lane forms its pair's phase
// from the FP64 (tile, sensor) reference and the window's first and last samples, and walks the
// window adding (A / 2R) d_q exp(-d_q^2 / 2 sigma^2) at d_q = d_0 - q Delta into its own signal
// band.  In the scaled phase s = sc d the term is (A / 2R sc) s 2^(-s^2).
//
// Band layout.  A warp's band holds rows (samples) 2i and 2i + 1 of lane l as one float2 at
// [i][l]: the 32 lanes' 8-byte accesses fall in distinct banks whatever rows they address, and a
// lane walks its window two samples per step with packed FP32 arithmetic (one 8-byte
// read-modify-write, one FMUL2 for s^2, one for the weight, one FFMA2 into the band, one FADD2 for
// the phase, two ex2).  The walk starts at the even row at or below the window's first sample;
// only its first pair and last three pairs can hold samples outside the window, and only those
// are masked.  When a lane's walked rows do not all lie in its band (a window across a pass
// boundary or the record's start), the warp walks that Gaussian with every pair tested against
// the band and the window; a window that lies wholly in another pass's samples is skipped.  Rows
// past the band's kept entries are never written out.  The windows of the next FF_G Gaussians
// (phase, bounds and weight: a chain of about twenty dependent operations with two MUFU
// operations each) are formed together while the current FF_G are walked, so that their
// latencies overlap.
//
// After the slab each lane writes its band as the slab's banded partial row (start sample,
// length); the slab reduction sums the rows per sample in a fixed order.  No atomics.  A
// sensor whose band is longer than the shared-memory band takes several passes over the slab,
// each keeping the next LB samples.
#include <cuda.h>

#include <climits>
#include <cmath>

#include "gpair_internal.cuh"

namespace gp {

constexpr int FF_MAXW = 8;            // warps per CTA, at most
constexpr int FF_THREADS_MAX = FF_MAXW * 32;
constexpr int FF_G = 4;               // Gaussians whose windows are formed together (divides TILE)
static_assert(TILE % FF_G == 0, "FF_G divides the tile");

// Staged constants of one Gaussian (uniform over the lanes): 8 floats as two float4.
struct FfGauss {
    float4 o;    // dx, dy, dz (offset from the tile reference), |offset|^2
    float4 e;    // A / (2 sc), sc = sqrt(log2(e) / 2) / sigma, k sigma / Delta, sample pairs to walk (0: skip)
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
    // rows 2i, 2i + 1 of this lane at Y2[i * 32] (LB is a multiple of 4)
    float2* Y2 = reinterpret_cast<float2*>(smem_raw + FF_HDR) + (size_t)warp * (LB / 2) * 32 + lane;

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
                const float sc = __fdividef(0.84932180028801904272f, sg);   // sqrt(log2(e) / 2) / sigma
                const float ksi = a.k * sg * invDelta;
                q.o = make_float4(dx, dy, dz, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                // pairs: a window holds at most floor(2 ksi) + 2 samples (rounding of its ends
                // included) and the walk may start one row early
                q.e = make_float4(__fdividef(0.5f * g.A[i], sc), sc, ksi, (float)(((int)floorf(2.f * ksi) + 4) >> 1));
            } else {
                q.o = make_float4(0.f, 0.f, 0.f, 0.f);
                q.e = make_float4(0.f, 0.f, 0.f, 0.f);    // zero pairs: skipped
            }
            S.tile[b][l] = q;
        }
    };

    for (int pass = 0; pass < npass; ++pass) {
        const int w = wa + pass * LB;
        const bool active = has_sensor && pass < npass_j;
        const int LBe = active ? min(LB, min(a.Nt, n_hi + 1) - w) : 0;     // band entries this pass keeps
        for (int q = 0; q < LB / 2; ++q) Y2[q * 32] = make_float2(0.f, 0.f);
        if (nTiles > 0) stage(0, 0);
        __syncthreads();
        for (int t = 0; t < nTiles; ++t) {
            const int b = t & 1;
            if (t + 1 < nTiles) stage(t + 1, b ^ 1);      // the next tile, while this one is used
            if (active) {
                const TileInfo rt = ti[sl.t_begin + t];
                const PairRef r = ref_doubled(make_ref(rt.c0x, rt.c0y, rt.c0z, sx, sy, sz, a));
                const int ybase = r.n0 - w;                    // band row of sample n0 + m is ybase + m
                // one window: sample pairs to walk NP (0: skip), the band row y0 of its first sample,
                // its sample count, the scaled phase s and its step at that sample, the scaled weight
                struct Win { int NP, y0, cnt; float s, step, wt; };
                auto window = [&](int l) {
                    const FfGauss G = S.tile[b][l];
                    Win c;
                    c.NP = (int)G.e.w;
                    float invR, phi;
                    pair_phase_pre(r, G.o.x, G.o.y, G.o.z, G.o.w, invR, phi);
                    const float tt = phi * invDelta;
                    const float ulo = __fadd_ru(tt - G.e.z, FF_MAGIC);      // MAGIC + first window sample
                    const float uhi = __fadd_rd(tt + G.e.z, FF_MAGIC);      // MAGIC + last window sample
                    const int m0 = __float_as_int(ulo) - FF_MAGIC_BITS;
                    c.cnt = max(0, __float_as_int(uhi) - __float_as_int(ulo) + 1);
                    c.y0 = ybase + m0;
                    c.s = G.e.y * fmaf(-(ulo - FF_MAGIC), Delta, phi);
                    c.step = G.e.y * Delta;
                    c.wt = G.e.x * invR;
                    return c;
                };
                // two samples per step: rows 2i + 2p, 2i + 2p + 1 from the even row 2i at or below y0
                auto walk_pairs = [&](const Win& c) {
                    const int off = c.y0 & 1;
                    float2* Yp = Y2 + ((c.y0 - off) >> 1) * 32;
                    const float sa = fmaf((float)off, c.step, c.s);
                    float2 s = make_float2(sa, sa - c.step);
                    const float2 ds = make_float2(-2.f * c.step, -2.f * c.step);
                    const float2 wt = make_float2(c.wt, c.wt);
                    const unsigned cnt = (unsigned)c.cnt;
                    auto pair = [&](int p, bool masked) {
                        const float2 q = __fmul2_rn(s, s);
                        float2 v = __fmul2_rn(s, wt);
                        const float2 e = make_float2(ex2_approx(-q.x), ex2_approx(-q.y));
                        if (masked) {      // window position of the pair's first sample: 2p - off
                            const int m = 2 * p - off;
                            v.x = (unsigned)m < cnt ? v.x : 0.f;
                            v.y = (unsigned)(m + 1) < cnt ? v.y : 0.f;
                        }
                        Yp[p * 32] = __ffma2_rn(v, e, Yp[p * 32]);
                        s = __fadd2_rn(s, ds);
                    };
                    const int NP = c.NP;
                    pair(0, true);
#pragma unroll 4
                    for (int p = 1; p < NP - 3; ++p) pair(p, false);
                    for (int p = max(1, NP - 3); p < NP; ++p) pair(p, true);
                };
                // the same walk with every pair tested against the window and the band: a pair
                // outside the band [0, LB) (pairs never straddle its ends: the walk starts at an
                // even row and LB is even) adds zero to the lane's first pair of rows instead
                auto walk_pairs_banded = [&](const Win& c) {
                    const int off = c.y0 & 1, ya = c.y0 - off;
                    const float sa = fmaf((float)off, c.step, c.s);
                    float2 s = make_float2(sa, sa - c.step);
                    const float2 ds = make_float2(-2.f * c.step, -2.f * c.step);
                    const float2 wt = make_float2(c.wt, c.wt);
                    const unsigned cnt = (unsigned)c.cnt;
#pragma unroll 2
                    for (int p = 0; p < c.NP; ++p) {
                        const float2 q = __fmul2_rn(s, s);
                        float2 v = __fmul2_rn(s, wt);
                        const float2 e = make_float2(ex2_approx(-q.x), ex2_approx(-q.y));
                        const int row = ya + 2 * p, m = 2 * p - off;
                        const bool inb = (unsigned)row < (unsigned)LB;
                        v.x = inb && (unsigned)m < cnt ? v.x : 0.f;
                        v.y = inb && (unsigned)(m + 1) < cnt ? v.y : 0.f;
                        float2* yp = Y2 + (inb ? (row >> 1) : 0) * 32;
                        *yp = __ffma2_rn(v, e, *yp);
                        s = __fadd2_rn(s, ds);
                    }
                };
                // per Gaussian, one path for the whole warp: the plain paired walk when every lane's
                // walked rows lie in its band, none when every lane's window lies wholly in another
                // pass's samples, else the banded walk (a window across a pass boundary)
                auto walk = [&](const Win& c) {
                    if (c.NP > 0) {
                        const int ya = c.y0 - (c.y0 & 1);      // first walked row
                        const bool in = ya >= 0 && ya + 2 * c.NP <= LB;
                        const bool out = ya >= LB || ya + 2 * c.NP <= 0;
                        const unsigned am = __activemask();
                        if (__all_sync(am, in)) walk_pairs(c);
                        else if (!__all_sync(am, out)) walk_pairs_banded(c);
                    }
                };
                // the windows of the next FF_G Gaussians are formed while the current FF_G are walked:
                // independent chains of phase, bounds and weight that hide one another's latency
                Win cur[FF_G];
#pragma unroll
                for (int u = 0; u < FF_G; ++u) cur[u] = window(u);
#pragma unroll 1
                for (int l = 0; l < TILE; l += FF_G) {
                    Win nxt[FF_G];
#pragma unroll
                    for (int u = 0; u < FF_G; ++u) nxt[u] = window(min(l + FF_G + u, TILE - 1));
#pragma unroll
                    for (int u = 0; u < FF_G; ++u) walk(cur[u]);
#pragma unroll
                    for (int u = 0; u < FF_G; ++u) cur[u] = nxt[u];
                }
            }
            __syncthreads();      // tile t's buffer is free; tile t + 1 is staged
        }
        if (active) {      // row positions [pass LB, pass LB + LB): LB and PL are multiples of 4
            float4* dst = reinterpret_cast<float4*>(prow + pass * LB);
            for (int q = 0; q < LBe; q += 4) {
                const float2 u0 = Y2[(q >> 1) * 32], u1 = Y2[((q >> 1) + 1) * 32];
                dst[q >> 2] = make_float4(u0.x, u0.y, u1.x, u1.y);
            }
        }
        __syncthreads();
    }
}

// Longest slabs first: the slab descriptors permuted in place by decreasing box diagonal (ties
// by index), so that the CTAs of the slabs with the longest sample bands -- those that may need
// several passes, such as a tile range that jumps across the Morton order -- start in the first
// wave instead of extending the last.  The slab reduction sums the rows of all slabs, so only the
// order of its (fixed-order) sum changes.  One CTA; S <= FF_ORDER_MAX.
constexpr int FF_ORDER_THREADS = 1024;
constexpr int FF_ORDER_MAX = 2048;
constexpr int FF_ORDER_PER = FF_ORDER_MAX / FF_ORDER_THREADS;

__global__ void __launch_bounds__(FF_ORDER_THREADS)
slab_order_kernel(SlabInfo* __restrict__ si, int S) {
    __shared__ float key[FF_ORDER_MAX];
    SlabInfo mine[FF_ORDER_PER];
    int rank[FF_ORDER_PER];
#pragma unroll
    for (int u = 0; u < FF_ORDER_PER; ++u) {
        const int s = threadIdx.x + u * FF_ORDER_THREADS;
        if (s < S) {
            mine[u] = si[s];
            const float dx = mine[u].hi[0] - mine[u].lo[0], dy = mine[u].hi[1] - mine[u].lo[1],
                        dz = mine[u].hi[2] - mine[u].lo[2];
            key[s] = (mine[u].t_end > mine[u].t_begin) ? dx * dx + dy * dy + dz * dz : -1.f;
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < FF_ORDER_PER; ++u) {
        const int s = threadIdx.x + u * FF_ORDER_THREADS;
        rank[u] = 0;
        if (s < S) {
            const float k = key[s];
            int r = 0;
            for (int t = 0; t < S; ++t) {
                const float kt = key[t];
                r += (kt > k) || (kt == k && t < s);
            }
            rank[u] = r;
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < FF_ORDER_PER; ++u) {
        const int s = threadIdx.x + u * FF_ORDER_THREADS;
        if (s < S) si[rank[u]] = mine[u];
    }
}

// ------------------------------------------------------------------------------------------
// Host side.

size_t fwd_free_smem(int NW, int LB) { return ff_smem_bytes(NW, LB); }

cudaError_t launch_slab_order(SlabInfo* si, int S, cudaStream_t st) {
    if (S <= 1 || S > FF_ORDER_MAX) return cudaSuccess;     // more slabs: kept in tile order
    slab_order_kernel<<<1, FF_ORDER_THREADS, 0, st>>>(si, S);
    return cudaGetLastError();
}

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
