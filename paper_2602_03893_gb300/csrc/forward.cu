// forward.cu -- the forward operator y = A(x) by direct windowed evaluation
// (Methods, Eq. single_forward; the pair enumeration over |d| <= k sigma).
//
// Work decomposition.  Gaussians are cut into tiles (grid: 8x8x4 bricks, each loaded by one 3-D
// TMA copy; SoA: 256 consecutive Gaussians) and tiles into slabs (grid: compact blocks of
// bricks; SoA: contiguous tile ranges).  One CTA owns (slab, group of 8 sensors); each warp owns
// one sensor.  For every tile the warp's lanes take Gaussians, evaluate each pair's window and add
// the samples into a short per-tile float band with shared-memory atomics; the tile band is then
// added into the slab's FP64 band, so long sums never accumulate in FP32.  The slab band is
// flushed once into a per-slab partial signal (coalesced stores; grid mode stores only the band
// and its offset), and a second kernel sums the slabs in a fixed order.  No global atomics.
#include <cuda.h>

#include <cstring>

#include "gpair_internal.cuh"

namespace gp {

constexpr int FWD_SPC = 8;        // sensors per CTA (one per warp)
constexpr int FWD_THREADS = 256;

// ------------------------------------------------------------------------------------------
// Tile summaries.  Grid mode: analytic (reference = brick centre).  SoA mode: bounding box of
// the tile's Gaussians; the reference is the box centre rounded to float.

__global__ void tile_info_grid_kernel(GaussDev g, TileInfo* ti) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= g.ntiles) return;
    int tx = (int)(t % g.ntx), ty = (int)((t / g.ntx) % g.nty), tz = (int)(t / ((int64_t)g.ntx * g.nty));
    TileInfo r;
    r.c0x = (float)(g.ox + (tx * BX + BX / 2) * (double)g.h);   // informational in grid mode
    r.c0y = (float)(g.oy + (ty * BY + BY / 2) * (double)g.h);
    r.c0z = (float)(g.oz + (tz * BZ + BZ / 2) * (double)g.h);
    r.rad = brick_radius(g.h);
    r.smax = g.sigma;
    int cx = min(BX, g.nx - tx * BX), cy = min(BY, g.ny - ty * BY), cz = min(BZ, g.nz - tz * BZ);
    r.count = cx * cy * cz;
    r.pad0 = r.pad1 = 0;
    ti[t] = r;
}

__global__ void __launch_bounds__(TILE) tile_info_soa_kernel(GaussDev g, TileInfo* ti) {
    __shared__ float red[7][TILE / 32];
    __shared__ float s_c0[3];
    const int64_t t = blockIdx.x;
    const int64_t i = t * TILE + threadIdx.x;
    const bool ok = i < g.M;
    const float x = ok ? g.cx[i] : 0.f, y = ok ? g.cy[i] : 0.f, z = ok ? g.cz[i] : 0.f;
    float v[7] = {ok ? x : 3e38f, ok ? y : 3e38f, ok ? z : 3e38f, ok ? -x : 3e38f, ok ? -y : 3e38f,
                  ok ? -z : 3e38f, ok ? -g.sg[i] : 3e38f};
    for (int q = 0; q < 7; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] = fminf(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) for (int q = 0; q < 7; ++q) red[q][w] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        float b[7];
        for (int q = 0; q < 7; ++q) { b[q] = red[q][0]; for (int k = 1; k < TILE / 32; ++k) b[q] = fminf(b[q], red[q][k]); }
        s_c0[0] = 0.5f * (b[0] - b[3]); s_c0[1] = 0.5f * (b[1] - b[4]); s_c0[2] = 0.5f * (b[2] - b[5]);
        red[0][0] = -b[6];
    }
    __syncthreads();
    const float c0x = s_c0[0], c0y = s_c0[1], c0z = s_c0[2], smax = red[0][0];
    const float dx = x - c0x, dy = y - c0y, dz = z - c0z;
    float r2 = ok ? dx * dx + dy * dy + dz * dz : 0.f;
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    __syncthreads();
    if (lane == 0) red[1][w] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = red[1][0];
        for (int k = 1; k < TILE / 32; ++k) m = fmaxf(m, red[1][k]);
        TileInfo r;
        r.c0x = c0x; r.c0y = c0y; r.c0z = c0z;
        r.rad = sqrtf(m) * 1.0001f + 1e-9f;
        r.smax = smax;
        int64_t cnt = g.M - t * TILE;
        r.count = (int)(cnt > TILE ? TILE : cnt);
        r.pad0 = r.pad1 = 0;
        ti[t] = r;
    }
}

// Grid mode: slab s is block (sx, sy, sz) of the block lattice; its bounding box is the box of
// its node centres.
__global__ void slab_info_grid_kernel(GaussDev g, int sbx, int sby, int sbz, int nsx, int nsy, int S,
                                      SlabInfo* si) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int sx = s % nsx, sy = (s / nsx) % nsy, sz = s / (nsx * nsy);
    SlabInfo o;
    o.bx0 = sx * sbx; o.by0 = sy * sby; o.bz0 = sz * sbz;
    o.bdx = min(sbx, g.ntx - o.bx0); o.bdy = min(sby, g.nty - o.by0); o.bdz = min(sbz, g.ntz - o.bz0);
    const int ax = o.bx0 * BX, bxn = min(g.nx, (o.bx0 + o.bdx) * BX);
    const int ay = o.by0 * BY, byn = min(g.ny, (o.by0 + o.bdy) * BY);
    const int az = o.bz0 * BZ, bzn = min(g.nz, (o.bz0 + o.bdz) * BZ);
    o.lo[0] = (float)(g.ox + (ax + 0.5) * g.h); o.hi[0] = (float)(g.ox + (bxn - 0.5) * g.h);
    o.lo[1] = (float)(g.oy + (ay + 0.5) * g.h); o.hi[1] = (float)(g.oy + (byn - 0.5) * g.h);
    o.lo[2] = (float)(g.oz + (az + 0.5) * g.h); o.hi[2] = (float)(g.oz + (bzn - 0.5) * g.h);
    // widen by a few ulp so that float rounding of the box never cuts a centre off
    for (int q = 0; q < 3; ++q) {
        float pad = 1e-6f * (fabsf(o.lo[q]) + fabsf(o.hi[q])) + 1e-9f;
        o.lo[q] -= pad; o.hi[q] += pad;
    }
    o.smax = g.sigma;
    o.t_begin = 0; o.t_end = o.bdx * o.bdy * o.bdz;
    o.pad = 0;
    si[s] = o;
}

// SoA mode: the axis-aligned box of the Gaussian centres and the widest sigma of each contiguous
// tile range (exact over the range's Gaussians, so that a slab of elongated tiles keeps a short
// sample band).
__global__ void slab_info_soa_kernel(GaussDev g, int64_t ntiles, int64_t tiles_per_slab, SlabInfo* si) {
    __shared__ float red[7][FWD_THREADS / 32];
    const int s = blockIdx.x;
    int64_t tb = s * tiles_per_slab, te = tb + tiles_per_slab;
    if (te > ntiles) te = ntiles;
    float v[7] = {3e38f, 3e38f, 3e38f, 3e38f, 3e38f, 3e38f, 0.f};
    const int64_t ie = te * TILE < g.M ? te * TILE : g.M;
    for (int64_t i = tb * TILE + threadIdx.x; i < ie; i += blockDim.x) {
        const float x = g.cx[i], y = g.cy[i], z = g.cz[i];
        v[0] = fminf(v[0], x); v[1] = fminf(v[1], y); v[2] = fminf(v[2], z);
        v[3] = fminf(v[3], -x); v[4] = fminf(v[4], -y); v[5] = fminf(v[5], -z);
        v[6] = fmaxf(v[6], g.sg[i]);
    }
    for (int q = 0; q < 6; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] = fminf(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
    for (int o = 16; o > 0; o >>= 1) v[6] = fmaxf(v[6], __shfl_xor_sync(0xffffffffu, v[6], o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) for (int q = 0; q < 7; ++q) red[q][w] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x / 32;
        SlabInfo o;
        for (int q = 0; q < 3; ++q) {
            float a = red[q][0], b = red[q + 3][0];
            for (int k = 1; k < nw; ++k) { a = fminf(a, red[q][k]); b = fminf(b, red[q + 3][k]); }
            o.lo[q] = a; o.hi[q] = -b;
            const float pad = 1e-6f * (fabsf(o.lo[q]) + fabsf(o.hi[q])) + 1e-9f;   // rounding slack
            o.lo[q] -= pad; o.hi[q] += pad;
        }
        float sm = red[6][0];
        for (int k = 1; k < nw; ++k) sm = fmaxf(sm, red[6][k]);
        o.smax = sm;
        o.t_begin = (int)tb; o.t_end = (int)te;
        o.bx0 = o.by0 = o.bz0 = 0; o.bdx = o.bdy = o.bdz = 0; o.pad = 0;
        si[s] = o;
    }
}

// ------------------------------------------------------------------------------------------
// Forward slab kernel.

struct FwdSmem {
    float tile[2][5][TILE];   // [buffer][A, cx, cy, cz, sigma][Gaussian]; grid mode uses A only
    uint64_t mbar[2];
    int npass;
    int abort;
};
// Bands follow the header at a 128-byte boundary: per warp a float tile band of TB entries,
// then per warp an FP64 slab band of LB entries.
constexpr size_t FWD_HDR = (sizeof(FwdSmem) + 127) & ~(size_t)127;



// banded = 1 (grid mode): the partial row of (slab, sensor) holds only the slab's band window,
// at offset rows[].x, length rows[].y; PL = LB.  banded = 0: full rows of PL = N_t samples,
// written completely (zeros outside the band).
template <bool GRID>
__global__ void __launch_bounds__(FWD_THREADS)
fwd_slab_kernel(GaussDev g, ArrDev a, const TileInfo* __restrict__ ti, const SlabInfo* __restrict__ slabs,
                float* __restrict__ partial, int2* __restrict__ rows, int PL, int LB, int TB, int banded,
                int* status, int use_tma, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FwdSmem& S = *reinterpret_cast<FwdSmem*>(smem_raw);
    float* tbands = reinterpret_cast<float*>(smem_raw + FWD_HDR);
    double* lbands = reinterpret_cast<double*>(smem_raw + FWD_HDR + (((size_t)FWD_SPC * TB * 4 + 127) & ~(size_t)127));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slab = blockIdx.y;
    const int j = blockIdx.x * FWD_SPC + warp;
    const bool has_sensor = j < a.Nd;
    const SlabInfo sl = slabs[slab];
    const int nTiles = sl.t_end - sl.t_begin;
    float* tband = tbands + (size_t)warp * TB;
    double* lband = lbands + (size_t)warp * LB;
    const size_t row = (size_t)slab * a.Nd + (has_sensor ? j : 0);
    float* prow = partial + row * PL;

    // Band of samples this (slab, sensor) can touch.
    float sx = 0.f, sy = 0.f, sz = 0.f;
    int n_lo = 0, n_hi = -1;
    if (has_sensor) {
        sx = a.xyz[3 * j]; sy = a.xyz[3 * j + 1]; sz = a.xyz[3 * j + 2];
        if (nTiles > 0) {
            double dmin, dmax;
            box_distance(sl, sx, sy, sz, dmin, dmax);
            double ks = (double)a.k * sl.smax;
            double lo = floor(((dmin - ks) / a.v - a.t0) * a.fs) - 2.0;
            double hi = ceil(((dmax + ks) / a.v - a.t0) * a.fs) + 2.0;
            if (lo < 0) lo = 0;
            if (hi > a.Nt - 1) hi = a.Nt - 1;
            if (lo <= hi) { n_lo = (int)lo; n_hi = (int)hi; }
        }
    }
    const int wa = n_lo & ~3;
    int npass_j = (n_lo <= n_hi) ? (n_hi + 1 - wa + LB - 1) / LB : 0;
    if (banded && npass_j > 1) {      // cannot happen with the host's band bound; keep memory safe
        set_status(status, DEV_CAPACITY);
        npass_j = 1;
    }
    if (threadIdx.x == 0) { S.npass = 0; S.abort = 0; }
    __syncthreads();
    if (lane == 0 && has_sensor) {
        atomicMax(&S.npass, npass_j);
        if (banded) rows[row] = make_int2(wa, npass_j > 0 ? min(LB, a.Nt - wa) : 0);
    }

    // Full-row mode: zero the partial row outside the windows the passes will write.
    if (has_sensor && !banded) {
        int wend = (npass_j > 0) ? min(a.Nt, wa + npass_j * LB) : 0;
        int zb = (npass_j > 0) ? wa : a.Nt;
        for (int n = lane; n < zb; n += 32) prow[n] = 0.f;
        for (int n = wend + lane; n < a.Nt; n += 32) prow[n] = 0.f;
    }
    const bool tma = GRID && use_tma;
    if (tma && threadIdx.x == 0) {
        mbar_init(&S.mbar[0], 1);
        mbar_init(&S.mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int npass = S.npass;
    const int64_t total = (int64_t)npass * nTiles;

    auto issue = [&](int64_t T) {
        // grid mode: one 3-D TMA box (8 x 8 x 4 floats of A) per tile
        int tx, ty, tz;
        slab_brick(sl, (int)(T % nTiles), tx, ty, tz);
        const int b = (int)(T & 1);
        mbar_arrive_expect_tx(&S.mbar[b], TILE * sizeof(float));
        tma_load_3d(&S.tile[b][0][0], &tmap, tx * BX, ty * BY, tz * BZ, &S.mbar[b]);
    };
    if (tma && threadIdx.x == 0) {
        if (total > 0) issue(0);
        if (total > 1) issue(1);
    }

    const float Delta = a.Delta, invDelta = a.invDelta;
    const float c2g = GRID ? -0.72134752044448170368f / (g.sigma * g.sigma) : 0.f;  // -log2(e)/2/s^2
    const float reach_g = GRID ? brick_radius(g.h) + a.k * g.sigma : 0.f;

    int64_t T = 0;
    for (int pass = 0; pass < npass; ++pass) {
        const int w = wa + pass * LB;
        const bool active = has_sensor && pass < npass_j;
        for (int q = lane; q < LB; q += 32) lband[q] = 0.0;
        __syncwarp();
        PairRef refs;            // lane q holds the reference of tile (t & ~31) + q
        for (int t = 0; t < nTiles; ++t, ++T) {
            const int b = (int)(T & 1);
            if (tma) {
                bool ok = mbar_wait(&S.mbar[b], (uint32_t)((T >> 1) & 1));
                if (!ok) S.abort = 1;
                __syncthreads();
                if (S.abort) goto aborted;
            } else if (GRID) {
                // brick without a TMA descriptor (row pitch not 16-byte aligned): plain loads
                int tx, ty, tz;
                slab_brick(sl, t, tx, ty, tz);
                for (int q = threadIdx.x; q < TILE; q += FWD_THREADS) {
                    const int gx = tx * BX + (q & (BX - 1)), gy = ty * BY + ((q / BX) & (BY - 1)), gz = tz * BZ + q / (BX * BY);
                    const bool ok = gx < g.nx && gy < g.ny && gz < g.nz;
                    S.tile[b][0][q] = ok ? g.A[((int64_t)gz * g.ny + gy) * g.nx + gx] : 0.f;
                }
                __syncthreads();
            } else {
                const int64_t base = (int64_t)(sl.t_begin + t) * TILE;
                for (int q = threadIdx.x; q < TILE; q += FWD_THREADS) {
                    int64_t i = base + q;
                    bool ok = i < g.M;
                    S.tile[b][0][q] = ok ? g.A[i] : 0.f;
                    S.tile[b][1][q] = ok ? g.cx[i] : 0.f;
                    S.tile[b][2][q] = ok ? g.cy[i] : 0.f;
                    S.tile[b][3][q] = ok ? g.cz[i] : 0.f;
                    S.tile[b][4][q] = ok ? g.sg[i] : 1.f;
                }
                __syncthreads();
            }
            if (active) {
                if ((t & 31) == 0 && t + lane < nTiles) {
                    if (GRID) {
                        int tx, ty, tz;
                        slab_brick(sl, t + lane, tx, ty, tz);
                        refs = make_ref(g.ox + (tx * BX + BX / 2) * (double)g.h, g.oy + (ty * BY + BY / 2) * (double)g.h,
                                        g.oz + (tz * BZ + BZ / 2) * (double)g.h, sx, sy, sz, a);
                    } else {
                        const TileInfo r = ti[sl.t_begin + t + lane];
                        refs = make_ref(r.c0x, r.c0y, r.c0z, sx, sy, sz, a);
                    }
                }
                const int src = t & 31;
                PairRef r;
                r.v0x = __shfl_sync(0xffffffffu, refs.v0x, src);
                r.v0y = __shfl_sync(0xffffffffu, refs.v0y, src);
                r.v0z = __shfl_sync(0xffffffffu, refs.v0z, src);
                r.R0 = __shfl_sync(0xffffffffu, refs.R0, src);
                r.phi0 = __shfl_sync(0xffffffffu, refs.phi0, src);
                r.n0 = __shfl_sync(0xffffffffu, refs.n0, src);
                float rc0x = 0.f, rc0y = 0.f, rc0z = 0.f, reach = reach_g;
                if (!GRID) {
                    const TileInfo rt = ti[sl.t_begin + t];
                    rc0x = rt.c0x; rc0y = rt.c0y; rc0z = rt.c0z;
                    reach = rt.rad + a.k * rt.smax;
                }
                // samples this tile can touch, inside this pass's window and the record
                int ta = r.n0 + (int)floorf((r.phi0 - reach) * invDelta) - 2;
                int tb = r.n0 + (int)ceilf((r.phi0 + reach) * invDelta) + 2;
                ta = max(ta, max(w, 0));
                tb = min(tb, min(w + LB - 1, a.Nt - 1));
                for (int sw = ta; sw <= tb; sw += TB) {
                    const int se = min(sw + TB - 1, tb);
                    for (int q = lane; q < TB; q += 32) tband[q] = 0.f;
                    __syncwarp();
                    const int mlo_cap = sw - r.n0, mhi_cap = se - r.n0;
                    const int bofs = r.n0 - sw;
                    for (int l = lane; l < TILE; l += 32) {
                        const float Ai = S.tile[b][0][l];
                        if (Ai == 0.f) continue;
                        float dx, dy, dz, sig, c2;
                        if (GRID) {
                            brick_offset(l, g.h, dx, dy, dz);
                            sig = g.sigma;
                            c2 = c2g;
                        } else {
                            dx = S.tile[b][1][l] - rc0x;
                            dy = S.tile[b][2][l] - rc0y;
                            dz = S.tile[b][3][l] - rc0z;
                            sig = S.tile[b][4][l];
                            c2 = -0.72134752044448170368f / (sig * sig);
                        }
                        float R, phi;
                        pair_phase(r, dx, dy, dz, R, phi);
                        const float ks = a.k * sig;
                        const int m_lo = max((int)ceilf((phi - ks) * invDelta), mlo_cap);
                        const int m_hi = min((int)floorf((phi + ks) * invDelta), mhi_cap);
                        const float wgt = Ai * 0.5f / R;
                        for (int m = m_lo; m <= m_hi; ++m) {
                            const float d = fmaf(-(float)m, Delta, phi);
                            const float e = ex2_approx(d * d * c2);
                            atomicAdd(&tband[bofs + m], wgt * d * e);
                        }
                    }
                    __syncwarp();
                    for (int q = lane; q <= se - sw; q += 32) lband[sw - w + q] += (double)tband[q];
                    __syncwarp();
                }
            }
            __syncthreads();   // every warp is done with buffer b
            if (tma && threadIdx.x == 0 && T + 2 < total) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(T + 2);
            }
        }
        __syncwarp();
        if (active) {
            const int wend = min(a.Nt, w + LB);
            float* dst = banded ? prow : prow + w;
            for (int q = lane; q < wend - w; q += 32) dst[q] = (float)lband[q];
        }
        __syncwarp();
    }
    return;
aborted:
    set_status(status, DEV_TIMEOUT);
    // Let the copies this CTA issued land before its shared memory is released.
    if (tma && threadIdx.x == 0) {
        for (int64_t U = T; U < total && U < T + 2; ++U) mbar_wait(&S.mbar[U & 1], (uint32_t)((U >> 1) & 1));
    }
}

// ------------------------------------------------------------------------------------------
// Grid-mode forward with per-(tile, sensor) binning.
//
// For one brick and one sensor every pair's window starts at some sample of the tile band.
// The warp sorts the brick's 256 pairs by that start -- a counting sort whose ranks come from
// __match_any_sync -- and then walks the bins: lanes take window positions m (G lanes per bin,
// 32/G bins at a time) and loop over the bin's Gaussians, accumulating sample start + m in a
// register.  Each (bin, position) sum is added into the warp's tile band once, by plain
// read-modify-writes ordered group by group (no atomics, deterministic order), and every tile
// band is added into the slab band with Kahan compensation.

struct FwdGridSmem {
    float tileA[2][TILE];
    uint64_t mbar[2];
    int npass;
    int abort;
};
constexpr size_t FWDG_HDR = (sizeof(FwdGridSmem) + 127) & ~(size_t)127;
constexpr int FWDG_NCH = 4;      // window chunks of G positions per lane (L <= 4 G)

// Per-warp shared memory of the binned kernel: sorted records (d0, w) | bin offsets [TB + 2] |
// float tile band [TB] | Kahan slab band (hi, lo) [LB].
__host__ __device__ __forceinline__ size_t fwdg_warp_bytes(int TB, int LB) {
    return (size_t)TILE * 8 + (((size_t)(TB + 2) * 4 + 15) & ~(size_t)15) + (((size_t)TB * 4 + 15) & ~(size_t)15) +
           (size_t)LB * 8;
}

template <int G>
__global__ void __launch_bounds__(FWD_THREADS, 3)
fwd_grid_kernel(GaussDev g, ArrDev a, const SlabInfo* __restrict__ slabs, float* __restrict__ partial,
                int2* __restrict__ rows, int LB, int TB, int* status, int use_tma,
                const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FwdGridSmem& S = *reinterpret_cast<FwdGridSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* wbase = smem_raw + FWDG_HDR + (size_t)warp * fwdg_warp_bytes(TB, LB);
    float2* rec = reinterpret_cast<float2*>(wbase);
    int* off = reinterpret_cast<int*>(wbase + (size_t)TILE * 8);
    float* tband = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(off) + (((size_t)(TB + 2) * 4 + 15) & ~(size_t)15));
    float2* lband = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(tband) + (((size_t)TB * 4 + 15) & ~(size_t)15));

    const int slab = blockIdx.y;
    const int j = blockIdx.x * FWD_SPC + warp;
    const bool has_sensor = j < a.Nd;
    const SlabInfo sl = slabs[slab];
    const int nTiles = sl.t_end - sl.t_begin;
    const size_t row = (size_t)slab * a.Nd + (has_sensor ? j : 0);
    float* prow = partial + row * LB;

    // band of samples this (slab, sensor) can touch; one pass by construction of LB
    float sx = 0.f, sy = 0.f, sz = 0.f;
    int n_lo = 0, n_hi = -1;
    if (has_sensor) {
        sx = a.xyz[3 * j]; sy = a.xyz[3 * j + 1]; sz = a.xyz[3 * j + 2];
        if (nTiles > 0) {
            double dmin, dmax;
            box_distance(sl, sx, sy, sz, dmin, dmax);
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
    if (threadIdx.x == 0) { S.abort = 0; }
    const bool tma = use_tma != 0;
    if (tma && threadIdx.x == 0) {
        mbar_init(&S.mbar[0], 1);
        mbar_init(&S.mbar[1], 1);
        fence_mbar_init();
    }
    for (int q = lane; q < LB; q += 32) lband[q] = make_float2(0.f, 0.f);
    __syncthreads();

    auto issue = [&](int T) {
        int tx, ty, tz;
        slab_brick(sl, T, tx, ty, tz);
        const int b = T & 1;
        mbar_arrive_expect_tx(&S.mbar[b], TILE * sizeof(float));
        tma_load_3d(&S.tileA[b][0], &tmap, tx * BX, ty * BY, tz * BZ, &S.mbar[b]);
    };
    if (tma && threadIdx.x == 0) {
        if (nTiles > 0) issue(0);
        if (nTiles > 1) issue(1);
    }

    const float Delta = a.Delta, invDelta = a.invDelta;
    const float c2 = -0.72134752044448170368f / (g.sigma * g.sigma);   // -log2(e) / (2 sigma^2)
    const float ks = a.k * g.sigma;
    const float reach = brick_radius(g.h) + ks;
    const int grp = lane / G, mpos = lane % G;
    const unsigned lt_mask = (1u << lane) - 1u;

    PairRef refs;
    int t = 0;
    for (; t < nTiles; ++t) {
        const int b = t & 1;
        if (tma) {
            bool ok = mbar_wait(&S.mbar[b], (uint32_t)((t >> 1) & 1));
            if (!ok) S.abort = 1;
            __syncthreads();
            if (S.abort) break;
        } else {
            int tx, ty, tz;
            slab_brick(sl, t, tx, ty, tz);
            for (int q = threadIdx.x; q < TILE; q += FWD_THREADS) {
                const int gx = tx * BX + (q & (BX - 1)), gy = ty * BY + ((q / BX) & (BY - 1)), gz = tz * BZ + q / (BX * BY);
                const bool ok = gx < g.nx && gy < g.ny && gz < g.nz;
                S.tileA[b][q] = ok ? g.A[((int64_t)gz * g.ny + gy) * g.nx + gx] : 0.f;
            }
            __syncthreads();
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
            int ta = r.n0 + (int)floorf((r.phi0 - reach) * invDelta) - 2;
            int tb = r.n0 + (int)ceilf((r.phi0 + reach) * invDelta) + 2;
            ta = max(ta, w);
            tb = min(tb, n_hi);
            if (ta <= tb) {
                int NB = tb - ta + 1;
                if (NB > TB) {             // cannot happen with the host's bound on TB
                    if (lane == 0) set_status(status, DEV_CAPACITY);
                    NB = TB;
                    tb = ta + TB - 1;
                }
                for (int q = lane; q <= NB; q += 32) off[q] = 0;
                __syncwarp();
                // ---- pass 1: one lane per Gaussian; window start (key), rank within the key
                int key[TILE / 32], rnk[TILE / 32];
                float d0v[TILE / 32], wv[TILE / 32];
                int Lmax = 0;
#pragma unroll
                for (int q = 0; q < TILE / 32; ++q) {
                    const int l = lane + 32 * q;
                    const float Ai = S.tileA[b][l];
                    float dx, dy, dz, invR, phi;
                    brick_offset(l, g.h, dx, dy, dz);
                    pair_phase_fast(r, dx, dy, dz, invR, phi);
                    const int m_lo = max((int)ceilf((phi - ks) * invDelta), ta - r.n0);
                    const int m_hi = min((int)floorf((phi + ks) * invDelta), tb - r.n0);
                    const bool valid = Ai != 0.f && m_lo <= m_hi;
                    key[q] = valid ? r.n0 + m_lo - ta : NB;
                    d0v[q] = fmaf(-(float)m_lo, Delta, phi);
                    wv[q] = Ai * 0.5f * invR;
                    if (valid) Lmax = max(Lmax, m_hi - m_lo + 1);
                    const unsigned grpmask = __match_any_sync(0xffffffffu, key[q]);
                    const int before = __popc(grpmask & lt_mask);
                    const int base = off[key[q]];
                    __syncwarp();
                    if (before == 0) off[key[q]] = base + __popc(grpmask);
                    __syncwarp();
                    rnk[q] = base + before;
                }
                // ---- exclusive scan of the bin counts (each lane owns a run of bins)
                {
                    const int per = (NB + 31) / 32;
                    const int b0 = lane * per;
                    int run = 0;
                    for (int q = 0; q < per; ++q)
                        if (b0 + q < NB) run += off[b0 + q];
                    int incl = run;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v;
                    }
                    int acc = incl - run;
                    __syncwarp();
                    for (int q = 0; q < per; ++q)
                        if (b0 + q < NB) {
                            const int c = off[b0 + q];
                            off[b0 + q] = acc;
                            acc += c;
                        }
                    if (lane == 31) off[NB] = incl;
                    __syncwarp();
                }
#pragma unroll
                for (int q = 0; q < TILE / 32; ++q)
                    if (key[q] < NB) rec[off[key[q]] + rnk[q]] = make_float2(d0v[q], wv[q]);
                for (int o = 16; o > 0; o >>= 1) Lmax = max(Lmax, __shfl_xor_sync(0xffffffffu, Lmax, o));
                int nch = (Lmax + G - 1) / G;
                if (nch > FWDG_NCH) {      // cannot happen: the host picks the direct kernel then
                    if (lane == 0) set_status(status, DEV_CAPACITY);
                    nch = FWDG_NCH;
                }
                for (int q = lane; q < NB; q += 32) tband[q] = 0.f;
                __syncwarp();
                // ---- pass 2: lanes = window positions, loop over each bin's Gaussians
                float mD[FWDG_NCH];
#pragma unroll
                for (int c = 0; c < FWDG_NCH; ++c) mD[c] = (float)(mpos + c * G) * Delta;
                for (int b0 = 0; b0 < NB; b0 += 32 / G) {
                    const int bb = b0 + grp;
                    const bool bv = bb < NB;
                    const int start = bv ? off[bb] : 0;
                    const int cnt = bv ? off[bb + 1] - start : 0;
                    int niter = cnt;
                    for (int o = G; o < 32; o <<= 1) niter = max(niter, __shfl_xor_sync(0xffffffffu, niter, o));
                    if (niter == 0) continue;    // empty bins add nothing (warp-uniform)
                    float acc[FWDG_NCH];
#pragma unroll
                    for (int c = 0; c < FWDG_NCH; ++c) acc[c] = 0.f;
                    if (nch == 1) {        // every window fits one chunk (the usual case)
                        const float mD0 = mD[0];
                        const float2* rp = rec + start;
                        for (int i = 0; i < niter; ++i) {
                            // groups with fewer records read a zero record (finite, weight 0)
                            const float2 rr = (i < cnt) ? rp[i] : make_float2(0.f, 0.f);
                            const float d = rr.x - mD0;
                            const float e = ex2_approx(d * d * c2);
                            const float v = (d >= -ks) ? rr.y * d : 0.f;
                            acc[0] = fmaf(v, e, acc[0]);
                        }
                    } else {
                        for (int i = 0; i < niter; ++i) {
                            if (i < cnt) {
                                const float2 rr = rec[start + i];
#pragma unroll
                                for (int c = 0; c < FWDG_NCH; ++c) {
                                    if (c < nch) {
                                        const float d = rr.x - mD[c];
                                        if (d >= -ks) {
                                            const float e = ex2_approx(d * d * c2);
                                            acc[c] = fmaf(rr.y * d, e, acc[c]);
                                        }
                                    }
                                }
                            }
                        }
                    }
                    // groups write overlapping samples: one group at a time
#pragma unroll
                    for (int gg = 0; gg < 32 / G; ++gg) {
                        if (grp == gg && bv) {
#pragma unroll
                            for (int c = 0; c < FWDG_NCH; ++c) {
                                const int p = bb + mpos + c * G;
                                if (c < nch && p < NB) tband[p] += acc[c];
                            }
                        }
                        __syncwarp();
                    }
                }
                // ---- tile band -> slab band (Kahan)
                for (int q = lane; q < NB; q += 32) {
                    float2 s = lband[ta - w + q];
                    const float y = tband[q] - s.y;
                    const float tt = s.x + y;
                    s.y = (tt - s.x) - y;
                    s.x = tt;
                    lband[ta - w + q] = s;
                }
                __syncwarp();
            }
        }
        __syncthreads();   // every warp is done with buffer b
        if (tma && threadIdx.x == 0 && t + 2 < nTiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(t + 2);
        }
    }
    if (t < nTiles) {      // a bounded wait ran out
        set_status(status, DEV_TIMEOUT);
        if (tma && threadIdx.x == 0)
            for (int U = t; U < nTiles && U < t + 2; ++U) mbar_wait(&S.mbar[U & 1], (uint32_t)((U >> 1) & 1));
        return;
    }
    if (active) {
        const int wend = min(a.Nt, w + LB);
        for (int q = lane; q < wend - w; q += 32) {
            const float2 s = lband[q];
            prow[q] = s.x + s.y;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Grid-mode forward through the sub-sample expansion (MomentTable).  Binning as above, but each
// pair is reduced to its window-start bin b and offset e: the slab keeps, per bin, the moments
//     Z_p[b] = sum over the slab's pairs starting at b of w e^p     (p < MOM_P)
// and the signal is their correlation with the table, y[n] = sum_{m<L} sum_p c[m][p] Z_p[n - m],
// plus the direct edge terms of the few pairs the table misses at position E.  Lanes own bins:
// a lane sums the moments of its bin's records in registers and adds them into the slab's
// moment band (moment-major, so a warp's adds hit consecutive banks); no atomics except the
// ranks within a bin and the rare direct terms.
//
// Tiles stream through a ring of FWDM_RING shared buffers.  Each slot has a "full" barrier
// (completed by the TMA's byte count, or by the arrive of the warp that loaded it with plain
// loads) and a release counter; the last of the CTA's warps to release a slot refills it.  The
// warps (one sensor each) thus drift apart by up to FWDM_RING tiles instead of meeting at a CTA
// barrier every tile.
constexpr int FWDM_RING = 4;
struct FwdMomSmem {
    float tileA[FWDM_RING][TILE];
    uint64_t full[FWDM_RING];
    int released[FWDM_RING];     // release count of the slot, all phases (never reset)
    int issued[FWDM_RING];       // last tile copied into the slot by TMA (-1: none)
    int abort;
};
constexpr size_t FWDM_HDR = (sizeof(FwdMomSmem) + 127) & ~(size_t)127;

// Per-warp shared memory: sorted records (e, w) [TILE] | bin offsets [TB + 2] | moment band
// [P][LB + L] | direct-term band [LB], each part a multiple of 16 bytes so that every warp's
// records stay 8-byte aligned (with P = 7 and LB + L odd the band alone is not).
__host__ __device__ __forceinline__ size_t fwdm_band_floats(int LB, int L, int P) {
    return (((size_t)(LB + L) * P + 3) & ~(size_t)3);
}
__host__ __device__ __forceinline__ size_t fwdm_warp_bytes(int TB, int LB, int L, int P) {
    return (size_t)TILE * 8 + (((size_t)(TB + 2) * 4 + 15) & ~(size_t)15) + fwdm_band_floats(LB, L, P) * 4 +
           (((size_t)LB * 4 + 15) & ~(size_t)15);
}

template <int P>
__global__ void __launch_bounds__(FWD_THREADS, 3)
fwd_moment_kernel(GaussDev g, ArrDev a, const SlabInfo* __restrict__ slabs, float* __restrict__ partial,
                  int2* __restrict__ rows, int LB, int TB, int* status, int use_tma,
                  const __grid_constant__ CUtensorMap tmap, const __grid_constant__ MomentTable T) {
    static_assert(BX == 8 && BY == 8 && BZ == 4 && TILE == 256,
                  "lane offsets below assume lane + 32 q -> (lane & 7, (lane >> 3) + 4 (q & 1), q >> 1)");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FwdMomSmem& S = *reinterpret_cast<FwdMomSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = T.L;
    const int ZS = LB + L;                 // bins of the moment band
    static_assert(P >= 6 && P <= 8, "6 to 8 moments");
    unsigned char* wbase = smem_raw + FWDM_HDR + (size_t)warp * fwdm_warp_bytes(TB, LB, L, P);
    float2* rec = reinterpret_cast<float2*>(wbase);
    int* off = reinterpret_cast<int*>(wbase + (size_t)TILE * 8);
    float* Z = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(off) + (((size_t)(TB + 2) * 4 + 15) & ~(size_t)15));
    float* xband = Z + fwdm_band_floats(LB, L, P);

    const int slab = blockIdx.y;
    const int j = blockIdx.x * FWD_SPC + warp;
    const bool has_sensor = j < a.Nd;
    const SlabInfo sl = slabs[slab];
    const int nTiles = sl.t_end - sl.t_begin;
    const size_t row = (size_t)slab * a.Nd + (has_sensor ? j : 0);
    float* prow = partial + row * LB;

    float sx = 0.f, sy = 0.f, sz = 0.f;
    int n_lo = 0, n_hi = -1;
    if (has_sensor) {
        sx = a.xyz[3 * j]; sy = a.xyz[3 * j + 1]; sz = a.xyz[3 * j + 2];
        if (nTiles > 0) {
            double dmin, dmax;
            box_distance(sl, sx, sy, sz, dmin, dmax);
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
        for (int b = 0; b < FWDM_RING; ++b) {
            S.released[b] = 0;
            S.issued[b] = -1;
            mbar_init(&S.full[b], 1);
        }
        fence_mbar_init();
    }
    for (int q = lane; q < ZS * P; q += 32) Z[q] = 0.f;
    for (int q = lane; q < LB; q += 32) xband[q] = 0.f;
    __syncthreads();

    const bool tma = use_tma != 0;
    // Warp-cooperative fill of the slot of tile TT: one TMA copy issued by lane 0, or plain loads
    // by the warp's lanes followed by one release arrive.
    auto fill = [&](int TT) {
        const int b = TT % FWDM_RING;
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
        for (int TT = 0; TT < FWDM_RING && TT < nTiles; ++TT) fill(TT);

    const float Delta = a.Delta, invDelta = a.invDelta;
    const float c2 = -0.72134752044448170368f / (g.sigma * g.sigma);
    const float ks = a.k * g.sigma;
    const float rad = brick_radius(g.h);
    const float ED = (float)T.E * Delta;
    const float efac = edge_factor(T);
    const float ksi = ks * invDelta;       // k sigma in samples (same rounding as the adjoint)
    const int zlo = w - L;                 // first bin of the moment band
    // this lane's lattice offsets from the brick centre (Gaussian l = lane + 32 q)
    const float h = g.h;
    const float ox = ((float)(lane & 7) - 0.5f * (BX - 1)) * h;
    const float oy0 = ((float)(lane >> 3) - 0.5f * (BY - 1)) * h;
    const float oy1 = ((float)((lane >> 3) + 4) - 0.5f * (BY - 1)) * h;

    PairRef refs;
    int t = 0;
    bool ok = true;
    for (; t < nTiles; ++t) {
        const int b = t % FWDM_RING;
        if (!mbar_wait(&S.full[b], (uint32_t)((t / FWDM_RING) & 1))) {
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
            // window-start bins of the brick: its phases lie within rad of phi0
            int ta = r.n0 + (int)floorf((r.phi0 - rad - ks) * invDelta) - 2;
            int tb = r.n0 + (int)ceilf((r.phi0 + rad - ks) * invDelta) + 2;
            ta = max(ta, zlo);
            tb = min(tb, n_hi);
            if (ta <= tb) {
                int NB = tb - ta + 1;
                if (NB > TB) {
                    if (lane == 0) set_status(status, DEV_CAPACITY);
                    NB = TB;
                    tb = ta + TB - 1;
                }
                for (int q = lane; q <= NB; q += 32) off[q] = 0;
                __syncwarp();
                // num = 2 (c0 - s) . delta + |delta|^2, separable over the lane's offsets
                const float ax = ox * (2.f * r.v0x + ox);
                const float ay0 = oy0 * (2.f * r.v0y + oy0), ay1 = oy1 * (2.f * r.v0y + oy1);
                int key[TILE / 32], rnk[TILE / 32];
                float ev[TILE / 32], wv[TILE / 32];
#pragma unroll
                for (int q = 0; q < TILE / 32; ++q) {
                    const int l = lane + 32 * q;
                    const float Ai = S.tileA[b][l];
                    const float oz = ((float)(q >> 1) - 0.5f * (BZ - 1)) * h;
                    const float num = (ax + ((q & 1) ? ay1 : ay0)) + oz * (2.f * r.v0z + oz);
                    float invR, phi;
                    pair_phase_num(r, num, invR, phi);
                    const float mf = ceilf(fmaf(phi, invDelta, -ksi));   // first sample with d <= k sigma
                    const int bin = r.n0 + (int)mf;
                    const unsigned rel = (unsigned)(bin - ta);
                    const bool valid = Ai != 0.f && rel <= (unsigned)(tb - ta);
                    key[q] = valid ? (int)rel : NB;
                    const float d0 = fmaf(-mf, Delta, phi);
                    ev[q] = (d0 - T.dstar) * T.inv_half;
                    wv[q] = Ai * invR;             // the table carries the 1/2
                    // edge position E: the rare pairs the table does not account for, directly
                    if (valid && edge_corrected(T, ev[q])) {
                        const float dE = d0 - ED;
                        const int nE = bin + T.E;
                        if (nE >= w && nE <= n_hi)
                            atomicAdd(&xband[nE - w], efac * wv[q] * dE * ex2_approx(dE * dE * c2));
                    }
                    // rank within the bin (the order inside a bin only affects rounding)
                    rnk[q] = valid ? atomicAdd(&off[key[q]], 1) : 0;
                }
                __syncwarp();
                {   // exclusive scan of the bin counts
                    const int per = (NB + 31) / 32;
                    const int b0 = lane * per;
                    int run = 0;
                    for (int q = 0; q < per; ++q)
                        if (b0 + q < NB) run += off[b0 + q];
                    int incl = run;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v;
                    }
                    int acc = incl - run;
                    __syncwarp();
                    for (int q = 0; q < per; ++q)
                        if (b0 + q < NB) {
                            const int c = off[b0 + q];
                            off[b0 + q] = acc;
                            acc += c;
                        }
                    if (lane == 31) off[NB] = incl;
                    __syncwarp();
                }
#pragma unroll
                for (int q = 0; q < TILE / 32; ++q)
                    if (key[q] < NB) rec[off[key[q]] + rnk[q]] = make_float2(ev[q], wv[q]);
                __syncwarp();
                // lanes own bins: moments in registers, then one add into the moment band
                for (int bb = lane; bb < NB; bb += 32) {
                    const int start = off[bb], end = off[bb + 1];
                    if (start == end) continue;
                    float M[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) M[p] = 0.f;
#pragma unroll 2
                    for (int i = start; i < end; ++i) {
                        const float2 rr = rec[i];
                        const float e1 = rr.x, wq = rr.y;
                        const float e2 = e1 * e1, e4 = e2 * e2;
                        const float e3 = e2 * e1, e5 = e4 * e1, e6 = e4 * e2;
                        M[0] += wq;
                        M[1] = fmaf(wq, e1, M[1]);
                        M[2] = fmaf(wq, e2, M[2]);
                        M[3] = fmaf(wq, e3, M[3]);
                        M[4] = fmaf(wq, e4, M[4]);
                        M[5] = fmaf(wq, e5, M[5]);
                        if constexpr (P >= 7) M[6] = fmaf(wq, e6, M[6]);
                        if constexpr (P == 8) M[P - 1] = fmaf(wq, e4 * e3, M[P - 1]);
                    }
                    float* zp = Z + (ta + bb - zlo);
#pragma unroll
                    for (int p = 0; p < P; ++p) zp[(size_t)p * ZS] += M[p];
                }
                __syncwarp();
            }
        }
        // release the slot; the warp that releases it last refills it with tile t + FWDM_RING
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = (atomicAdd(&S.released[b], 1) + 1) % FWD_SPC == 0;
            if (last) __threadfence_block();
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last && t + FWDM_RING < nTiles) fill(t + FWDM_RING);
    }
    if (!ok && lane == 0) {   // a bounded wait ran out
        set_status(status, DEV_TIMEOUT);
        S.abort = 1;
    }
    __syncthreads();
    if (S.abort) {
        // wait (bounded) for the last copy issued into each slot before the CTA exits
        if (tma && threadIdx.x == 0)
            for (int b = 0; b < FWDM_RING; ++b)
                if (S.issued[b] >= 0) mbar_wait(&S.full[b], (uint32_t)((S.issued[b] / FWDM_RING) & 1));
        return;
    }
    if (active) {
        // y[n] = sum_{m<L} sum_p c[m][p] Z_p[n - m] + direct terms, for the slab's samples
        const int wend = min(a.Nt, w + LB);
        for (int q = lane; q < wend - w; q += 32) {
            float y = xband[q];
            const float* zb = Z + q + L;       // bin n = w + q sits at index q + L
            for (int m = 0; m < L; ++m) {
                const float* zm = zb - m;
#pragma unroll
                for (int p = 0; p < P; ++p) y = fmaf(T.c[m][p], zm[(size_t)p * ZS], y);
            }
            prow[q] = y;
        }
    }
}

// y[j][n] = sum over slabs of the partial rows, fixed slab order.  Banded rows cover
// [rows.x, rows.x + rows.y); full rows (banded = 0) cover the whole record.
__global__ void slab_reduce_kernel(const float* __restrict__ partial, const int2* __restrict__ rows, int S, int Nd,
                                   int Nt, int PL, int banded, float* __restrict__ y) {
    const int j = blockIdx.y;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < Nt; n += gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < S; ++s) {
            const size_t r = (size_t)s * Nd + j;
            if (banded) {
                const int2 ri = rows[r];
                const int q = n - ri.x;
                if (q >= 0 && q < ri.y) acc += partial[r * PL + q];
            } else {
                acc += partial[r * PL + n];
            }
        }
        y[(size_t)j * Nt + n] = acc;
    }
}

// Banded rows with the sensor's row descriptors staged in shared memory (S of them): a block
// covers 256 samples of one sensor, leaves at once when no band reaches them, and skips the
// slabs whose band misses them without touching their rows.  Each sample sums its slabs in
// slab order, as slab_reduce_kernel does.
constexpr int SLAB_RED_THREADS = 256;
constexpr int SLAB_RED_MAX_S = 6144;        // 48 KB of row descriptors
__global__ void __launch_bounds__(SLAB_RED_THREADS)
slab_reduce_banded_kernel(const float* __restrict__ partial, const int2* __restrict__ rows, int S, int Nd, int Nt,
                          int PL, float* __restrict__ y) {
    extern __shared__ int2 srow[];
    __shared__ int ext[2];
    const int j = blockIdx.y;
    const int n0 = blockIdx.x * SLAB_RED_THREADS;
    if (threadIdx.x == 0) {
        ext[0] = INT_MAX;
        ext[1] = INT_MIN;
    }
    __syncthreads();
    int lo = INT_MAX, hi = INT_MIN;
    for (int q = threadIdx.x; q < S; q += SLAB_RED_THREADS) {
        const int2 ri = rows[(size_t)q * Nd + j];
        srow[q] = ri;
        if (ri.y > 0) {
            lo = min(lo, ri.x);
            hi = max(hi, ri.x + ri.y);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&ext[0], lo);
        atomicMax(&ext[1], hi);
    }
    __syncthreads();
    const int n = n0 + (int)threadIdx.x;
    float acc = 0.f;
    if (ext[0] < n0 + SLAB_RED_THREADS && ext[1] > n0) {
        const int nend = n0 + SLAB_RED_THREADS;
        for (int q = 0; q < S; ++q) {
            const int2 ri = srow[q];
            if (ri.x >= nend || ri.x + ri.y <= n0) continue;     // the same for the whole block
            const unsigned d = (unsigned)(n - ri.x);
            if (d < (unsigned)ri.y) acc += partial[((size_t)q * Nd + j) * PL + d];
        }
    }
    if (n < Nt) y[(size_t)j * Nt + n] = acc;
}

// Banded rows, one block per (sensor, group of four 256-sample chunks): the sensor's row
// descriptors are sorted by band start (bitonic sort of (start, slab) keys in shared memory), and
// each chunk walks only the slabs whose bands can reach it -- those starting after the chunk's
// first sample minus the longest band and before its end, a contiguous run of the sorted keys --
// instead of testing every slab, eight slabs' loads at a time.  Each sample sums its slabs in the
// order of their band starts, ties by slab index: a fixed order, so the result is deterministic.
constexpr int SRS_THREADS = 256;
constexpr int SRS_MAX_S = 2048;             // sorted keys and descriptors: 32 KB
constexpr int SRS_CHUNKS = 4;               // 256-sample chunks per block (blockIdx.y: chunk group)
constexpr int SRS_UNROLL = 8;
__global__ void __launch_bounds__(SRS_THREADS)
slab_reduce_sorted_kernel(const float* __restrict__ partial, const int2* __restrict__ rows, int S, int Nd, int Nt,
                          int PL, float* __restrict__ y) {
    extern __shared__ unsigned long long srs_key[];     // [Sp] keys, then S descriptors
    __shared__ int red[2][SRS_THREADS / 32];
    const int j = blockIdx.x, t = threadIdx.x;
    int Sp = 1;
    while (Sp < S) Sp <<= 1;
    int2* srow = reinterpret_cast<int2*>(srs_key + Sp);
    int lbmax = 0, nvalid = 0;
    for (int q = t; q < Sp; q += SRS_THREADS) {
        unsigned long long k = ~0ull;                     // empty rows sort last
        if (q < S) {
            const int2 ri = rows[(size_t)q * Nd + j];
            srow[q] = ri;
            if (ri.y > 0) {
                k = ((unsigned long long)(unsigned)ri.x << 32) | (unsigned)q;
                lbmax = max(lbmax, ri.y);
                ++nvalid;
            }
        }
        srs_key[q] = k;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lbmax = max(lbmax, __shfl_xor_sync(0xffffffffu, lbmax, o));
        nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
    }
    if ((t & 31) == 0) { red[0][t >> 5] = lbmax; red[1][t >> 5] = nvalid; }
    __syncthreads();
    lbmax = 0; nvalid = 0;
#pragma unroll
    for (int w = 0; w < SRS_THREADS / 32; ++w) { lbmax = max(lbmax, red[0][w]); nvalid += red[1][w]; }
    for (int k = 2; k <= Sp; k <<= 1)                     // bitonic sort, ascending
        for (int h = k >> 1; h > 0; h >>= 1) {
            for (int i = t; i < Sp; i += SRS_THREADS) {
                const int p = i ^ h;
                if (p > i) {
                    const unsigned long long a = srs_key[i], b = srs_key[p];
                    if ((a > b) == ((i & k) == 0)) { srs_key[i] = b; srs_key[p] = a; }
                }
            }
            __syncthreads();
        }
    const int c_end = min(Nt, (blockIdx.y + 1) * SRS_CHUNKS * SRS_THREADS);
    for (int n0 = blockIdx.y * SRS_CHUNKS * SRS_THREADS; n0 < c_end; n0 += SRS_THREADS) {
        // the run of keys whose bands can reach the chunk: start in [n0 - lbmax + 1, n0 + 256)
        auto lower = [&](long long wv) {
            int lo = 0, hi = nvalid;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((long long)(srs_key[mid] >> 32) < wv) lo = mid + 1; else hi = mid;
            }
            return lo;
        };
        const int i0 = lower((long long)n0 - lbmax + 1), i1 = lower((long long)n0 + SRS_THREADS);
        const int n = n0 + t;
        float acc = 0.f;
        // SRS_UNROLL slabs at a time, so that their loads are in flight together; a slab past the
        // run or missing the sample contributes an exact zero, so the sum is the slab-by-slab one
        for (int i = i0; i < i1; i += SRS_UNROLL) {
            float v[SRS_UNROLL];
#pragma unroll
            for (int u = 0; u < SRS_UNROLL; ++u) {
                const int ii = min(i + u, i1 - 1);
                const unsigned long long k = srs_key[ii];
                const int q = (int)(k & 0xffffffffu);
                const unsigned d = (unsigned)(n - (int)(k >> 32));
                const bool use = i + u < i1 && d < (unsigned)srow[q].y;
                v[u] = use ? partial[((size_t)q * Nd + j) * PL + (use ? d : 0u)] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < SRS_UNROLL; ++u) acc += v[u];
        }
        if (n < Nt) y[(size_t)j * Nt + n] = acc;
    }
}

// ------------------------------------------------------------------------------------------
// Host side.

size_t fwd_smem_bytes(int LB, int TB) {
    return FWD_HDR + (((size_t)FWD_SPC * TB * 4 + 127) & ~(size_t)127) + (size_t)FWD_SPC * LB * 8;
}

static const CUtensorMap& null_tmap() {
    static CUtensorMap m = [] { CUtensorMap z; memset(&z, 0, sizeof(z)); return z; }();
    return m;
}

cudaError_t launch_tile_info(const GaussDev& g, TileInfo* ti, cudaStream_t st) {
    if (g.grid) {
        int blocks = (int)((g.ntiles + 255) / 256);
        tile_info_grid_kernel<<<blocks, 256, 0, st>>>(g, ti);
    } else {
        tile_info_soa_kernel<<<(unsigned)g.ntiles, TILE, 0, st>>>(g, ti);
    }
    return cudaGetLastError();
}

cudaError_t launch_slab_info_grid(const GaussDev& g, int sbx, int sby, int sbz, int S, SlabInfo* si,
                                  cudaStream_t st) {
    const int nsx = (g.ntx + sbx - 1) / sbx, nsy = (g.nty + sby - 1) / sby;
    slab_info_grid_kernel<<<(S + 127) / 128, 128, 0, st>>>(g, sbx, sby, sbz, nsx, nsy, S, si);
    return cudaGetLastError();
}

cudaError_t launch_slab_info_soa(const GaussDev& g, int64_t ntiles, int64_t tiles_per_slab, int S, SlabInfo* si,
                                 cudaStream_t st) {
    slab_info_soa_kernel<<<S, FWD_THREADS, 0, st>>>(g, ntiles, tiles_per_slab, si);
    return cudaGetLastError();
}

cudaError_t launch_forward(const GaussDev& g, const ArrDev& a, const TileInfo* ti, const SlabInfo* si, int S,
                           float* partial, int2* rows, int PL, int LB, int TB, bool binned, int* status,
                           const CUtensorMap* tmap, const MomentTable* mom, cudaStream_t st) {
    const size_t smem = fwd_smem_bytes(LB, TB);
    const int banded = g.grid ? 1 : 0;
    dim3 grid((a.Nd + FWD_SPC - 1) / FWD_SPC, S);
    cudaError_t e;
    if (g.grid && binned && mom) {
        // window-start bins of one brick: phases within its radius of phi0, so at most
        // 2 rad / Delta + 7 bins (floor/ceil and the -2/+2 margins)
        const int TBm = ((int)std::ceil(2.0 * brick_radius(g.h) * a.invDelta) + 8 + 3) & ~3;
        const size_t msm = FWDM_HDR + (size_t)FWD_SPC * fwdm_warp_bytes(TBm, LB, mom->L, mom->P);
        if (msm <= 227 * 1024) {
            auto kern = mom->P == 6 ? fwd_moment_kernel<6> : (mom->P == 7 ? fwd_moment_kernel<7> : fwd_moment_kernel<8>);
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm);
            if (e != cudaSuccess) return e;
            kern<<<grid, FWD_THREADS, msm, st>>>(g, a, si, partial, rows, LB, TBm, status, tmap != nullptr,
                                                 *(tmap ? tmap : &null_tmap()), *mom);
            return cudaGetLastError();
        }
    }
    const int Lmain = (int)floor(2.0 * a.k * g.sigma * a.invDelta) + 1;   // longest window, samples
    if (g.grid && binned) {
        const size_t gsm = FWDG_HDR + (size_t)FWD_SPC * fwdg_warp_bytes(TB, LB);
        const int use_tma = tmap != nullptr;
        const CUtensorMap& tm = *(tmap ? tmap : &null_tmap());
        if (Lmain <= 16) {
            e = cudaFuncSetAttribute(fwd_grid_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
            if (e != cudaSuccess) return e;
            fwd_grid_kernel<16><<<grid, FWD_THREADS, gsm, st>>>(g, a, si, partial, rows, LB, TB, status, use_tma, tm);
        } else {
            e = cudaFuncSetAttribute(fwd_grid_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
            if (e != cudaSuccess) return e;
            fwd_grid_kernel<32><<<grid, FWD_THREADS, gsm, st>>>(g, a, si, partial, rows, LB, TB, status, use_tma, tm);
        }
        return cudaGetLastError();
    }
    if (g.grid) {
        e = cudaFuncSetAttribute(fwd_slab_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fwd_slab_kernel<true><<<grid, FWD_THREADS, smem, st>>>(g, a, ti, si, partial, rows, PL, LB, TB, banded, status,
                                                               tmap != nullptr, *(tmap ? tmap : &null_tmap()));
    } else {
        e = cudaFuncSetAttribute(fwd_slab_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fwd_slab_kernel<false><<<grid, FWD_THREADS, smem, st>>>(g, a, ti, si, partial, rows, PL, LB, TB, banded,
                                                                status, 0, null_tmap());
    }
    return cudaGetLastError();
}

static dim3 slab_reduce_sorted_grid(const ArrDev& a) {
    return dim3(a.Nd, (a.Nt + SRS_CHUNKS * SRS_THREADS - 1) / (SRS_CHUNKS * SRS_THREADS));
}

static size_t slab_reduce_sorted_smem(int S) {
    size_t Sp = 1;
    while (Sp < (size_t)S) Sp <<= 1;
    return Sp * sizeof(unsigned long long) + (size_t)S * sizeof(int2);
}

// Banded rows (start sample, length; row capacity PL) of any Gaussian set.
cudaError_t launch_slab_reduce_rows(const ArrDev& a, const float* partial, const int2* rows, int S, int PL, float* y,
                                    cudaStream_t st) {
    dim3 rgrid((a.Nt + 255) / 256, a.Nd);
    if (S <= SRS_MAX_S && slab_reduce_sorted_grid(a).y <= 65535)
        slab_reduce_sorted_kernel<<<slab_reduce_sorted_grid(a), SRS_THREADS, slab_reduce_sorted_smem(S), st>>>(
            partial, rows, S, a.Nd, a.Nt, PL, y);
    else if (S <= SLAB_RED_MAX_S)
        slab_reduce_banded_kernel<<<rgrid, SLAB_RED_THREADS, (size_t)S * sizeof(int2), st>>>(partial, rows, S, a.Nd,
                                                                                             a.Nt, PL, y);
    else
        slab_reduce_kernel<<<rgrid, 256, 0, st>>>(partial, rows, S, a.Nd, a.Nt, PL, 1, y);
    return cudaGetLastError();
}

cudaError_t launch_slab_reduce(const GaussDev& g, const ArrDev& a, const float* partial, const int2* rows, int S,
                               int PL, float* y, cudaStream_t st) {
    dim3 rgrid((a.Nt + 255) / 256, a.Nd);
    if (g.grid && S <= SRS_MAX_S && slab_reduce_sorted_grid(a).y <= 65535)
        slab_reduce_sorted_kernel<<<slab_reduce_sorted_grid(a), SRS_THREADS, slab_reduce_sorted_smem(S), st>>>(
            partial, rows, S, a.Nd, a.Nt, PL, y);
    else if (g.grid && S <= SLAB_RED_MAX_S)
        slab_reduce_banded_kernel<<<rgrid, SLAB_RED_THREADS, (size_t)S * sizeof(int2), st>>>(partial, rows, S, a.Nd,
                                                                                             a.Nt, PL, y);
    else
        slab_reduce_kernel<<<rgrid, 256, 0, st>>>(partial, rows, S, a.Nd, a.Nt, PL, g.grid ? 1 : 0, y);
    return cudaGetLastError();
}

}  // namespace gp
