// forward_lanes.cu -- the forward operator for grid Gaussians with a shared sigma (Methods,
// Eq. single_forward with its window |d| <= k sigma), through the sub-sample expansion of the
// pulse (MomentTable), with the 32 lanes of a warp owning 32 sensors.
//
// Work decomposition.  The lattice is cut into cubes of 8 x 8 x 8 nodes (one 3-D TMA box each)
// and cubes into slabs (compact blocks of cubes).  A CTA owns one slab and NW x 32 sensors; the
// warps share the slab's cubes, which stream through a ring of shared buffers, and each lane owns
// one sensor.  For every cube all lanes take the same Gaussian at the same time, so that a lane
// evaluates the pair (Gaussian, its sensor): phase, window-start sample, offset e and weight
// w = A / R.  It adds the pair's P moments w e^p into its own moment band, indexed by the
// window-start sample relative to a per-(cube, sensor) base.  The band is laid out
// [bin][lane], so the 32 lanes of a warp hit 32 different banks whatever bins they address:
// there is no sort, no atomic and no divergence.  After the cube each lane correlates its band
// with the expansion table,
//     y[n] += sum_{m < L} sum_p c[m][p] Z_p[n - m],
// into its signal band for the slab ([sample][lane], also conflict free), then clears the
// moment band.  After the slab the signal bands become the slab's partial rows, which the slab
// reduction sums per sample in a fixed order: no global atomics, deterministic.
#include <cuda.h>

#include <climits>
#include <cmath>
#include <cstring>

#include "gpair_internal.cuh"

namespace gp {

constexpr int CUBE = 8;                        // cube side, lattice nodes
constexpr int CUBE_N = CUBE * CUBE * CUBE;     // Gaussians per cube
constexpr int FL_RING = 4;                     // cube buffers in flight
constexpr int FL_MAXW = 8;                     // warps per CTA, at most
constexpr int FL_Q = 8;                        // outputs per correlation chunk

struct FlHdr {
    float tileA[FL_RING][CUBE_N];
    uint64_t full[FL_RING];
    int released[FL_RING];       // release count of the slot over all phases (never reset)
    int issued[FL_RING];         // last cube copied into the slot by TMA (-1: none)
    int abort;
};
constexpr size_t FL_HDR = (sizeof(FlHdr) + 127) & ~(size_t)127;

// Moment band of a warp: per (bin, lane) P floats as a float4 (p = 0..3) plus the rest (p = 4, 5
// as a float2 for P = 6; a float2 and a float for P = 7; a float4 for P = 8), each part its own
// [bin][lane] array so that every access of a warp is conflict free.
// The band has NZ + 1 bins: bin NZ is never written and stays zero, so that reads of bins outside
// [0, NZ) in the correlation take it instead of a select per value.
__host__ __device__ __forceinline__ size_t fl_zbytes(int NZ, int P) { return (size_t)(NZ + 1) * 32 * 4 * (P <= 8 ? P : 8); }
__host__ __device__ __forceinline__ size_t fl_warp_bytes(int NZ, int LB, int P) {
    return fl_zbytes(NZ, P) + (size_t)LB * 32 * 4;
}
__host__ __device__ __forceinline__ int fl_lpad(int L) { return (L + FL_Q - 1) & ~(FL_Q - 1); }
__host__ __device__ __forceinline__ size_t fl_smem_bytes(int NW, int NZ, int LB, int P, int L) {
    return FL_HDR + (size_t)fl_lpad(L) * 8 * 4 + (size_t)NW * fl_warp_bytes(NZ, LB, P);
}

// Radius of a cube about its centre, with a little slack for rounding.
__host__ __device__ __forceinline__ float cube_radius(float h) {
    return sqrtf(3.f) * 0.5f * (CUBE - 1) * h * 1.0001f + 1e-9f;
}

// Bins of a (cube, sensor) moment band: the cube's phases lie within cube_radius of the
// reference phase, so the window-start samples span at most 2 rad / Delta + 1; the base is one
// sample below the lowest and one more covers the ceiling.
__host__ __device__ __forceinline__ int fl_nz(float h, float invDelta) {
    return (int)ceilf(2.f * cube_radius(h) * invDelta) + 4;
}

template <int P>
struct ZBand {
    float4* a;      // p = 0..3
    float2* b2;     // p = 4, 5 (P = 6, 7)
    float* c1;      // p = 6 (P = 7)
    float4* b4;     // p = 4..7 (P = 8)
    __device__ __forceinline__ void init(unsigned char* base, int NZ) {
        a = reinterpret_cast<float4*>(base);
        unsigned char* rest = base + (size_t)(NZ + 1) * 32 * 16;
        b2 = reinterpret_cast<float2*>(rest);
        c1 = reinterpret_cast<float*>(rest + (size_t)(NZ + 1) * 32 * 8);
        b4 = reinterpret_cast<float4*>(rest);
    }
    // Z[bin][lane] += (m0 .. m_{P-1})
    __device__ __forceinline__ void add(int idx, const float* m) {
        float4 z = a[idx];
        z.x += m[0]; z.y += m[1]; z.z += m[2]; z.w += m[3];
        a[idx] = z;
        if constexpr (P == 8) {
            float4 y = b4[idx];
            y.x += m[4]; y.y += m[5]; y.z += m[6]; y.w += m[7];
            b4[idx] = y;
        } else {
            float2 y = b2[idx];
            y.x += m[4]; y.y += m[5];
            b2[idx] = y;
            if constexpr (P == 7) c1[idx] += m[6];
        }
    }
    // Two pairs at once: Z[i1] += m1 and Z[i2] += m2.  All loads come before all stores, so the two
    // read-modify-writes (and the parts of each) form one dependency step instead of a chain of
    // four; when i1 == i2 the second store, which lands last, carries both pairs.
    __device__ __forceinline__ void add2(int i1, int i2, const float* m1, const float* m2) {
        const bool eq = i1 == i2;
        const float4 za1 = a[i1], za2 = a[i2];
        float s1[8], s2[8];
        float z1[8], z2[8];
        z1[0] = za1.x; z1[1] = za1.y; z1[2] = za1.z; z1[3] = za1.w;
        z2[0] = za2.x; z2[1] = za2.y; z2[2] = za2.z; z2[3] = za2.w;
        if constexpr (P == 8) {
            const float4 y1 = b4[i1], y2 = b4[i2];
            z1[4] = y1.x; z1[5] = y1.y; z1[6] = y1.z; z1[7] = y1.w;
            z2[4] = y2.x; z2[5] = y2.y; z2[6] = y2.z; z2[7] = y2.w;
        } else {
            const float2 y1 = b2[i1], y2 = b2[i2];
            z1[4] = y1.x; z1[5] = y1.y;
            z2[4] = y2.x; z2[5] = y2.y;
            if constexpr (P == 7) { z1[6] = c1[i1]; z2[6] = c1[i2]; }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            s1[p] = z1[p] + m1[p];
            s2[p] = (eq ? s1[p] : z2[p]) + m2[p];
        }
        a[i1] = make_float4(s1[0], s1[1], s1[2], s1[3]);
        a[i2] = make_float4(s2[0], s2[1], s2[2], s2[3]);
        if constexpr (P == 8) {
            b4[i1] = make_float4(s1[4], s1[5], s1[6], s1[7]);
            b4[i2] = make_float4(s2[4], s2[5], s2[6], s2[7]);
        } else {
            b2[i1] = make_float2(s1[4], s1[5]);
            b2[i2] = make_float2(s2[4], s2[5]);
            if constexpr (P == 7) { c1[i1] = s1[6]; c1[i2] = s2[6]; }
        }
    }
    // Z[bin][lane]
    __device__ __forceinline__ void load(int idx, float* m) const {
        const float4 z = a[idx];
        m[0] = z.x; m[1] = z.y; m[2] = z.z; m[3] = z.w;
        if constexpr (P == 8) {
            const float4 y = b4[idx];
            m[4] = y.x; m[5] = y.y; m[6] = y.z; m[7] = y.w;
        } else {
            const float2 y = b2[idx];
            m[4] = y.x; m[5] = y.y;
            if constexpr (P == 7) m[6] = c1[idx];
        }
    }
    __device__ __forceinline__ void clear(int idx) {
        a[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (P == 8) {
            b4[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            b2[idx] = make_float2(0.f, 0.f);
            if constexpr (P == 7) c1[idx] = 0.f;
        }
    }
};

// Slab descriptors in cube units: a block of scx x scy x scz cubes; lo/hi bound its Gaussian
// centres (for the sample band of each sensor).
__global__ void slab_info_cube_kernel(GaussDev g, int ncx, int ncy, int ncz, int scx, int scy, int scz, int nsx,
                                      int nsy, int S, SlabInfo* si) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int sx = s % nsx, sy = (s / nsx) % nsy, sz = s / (nsx * nsy);
    SlabInfo o;
    o.bx0 = sx * scx; o.by0 = sy * scy; o.bz0 = sz * scz;
    o.bdx = min(scx, ncx - o.bx0); o.bdy = min(scy, ncy - o.by0); o.bdz = min(scz, ncz - o.bz0);
    const int ax = o.bx0 * CUBE, bxn = min(g.nx, (o.bx0 + o.bdx) * CUBE);
    const int ay = o.by0 * CUBE, byn = min(g.ny, (o.by0 + o.bdy) * CUBE);
    const int az = o.bz0 * CUBE, bzn = min(g.nz, (o.bz0 + o.bdz) * CUBE);
    o.lo[0] = (float)(g.ox + (ax + 0.5) * g.h); o.hi[0] = (float)(g.ox + (bxn - 0.5) * g.h);
    o.lo[1] = (float)(g.oy + (ay + 0.5) * g.h); o.hi[1] = (float)(g.oy + (byn - 0.5) * g.h);
    o.lo[2] = (float)(g.oz + (az + 0.5) * g.h); o.hi[2] = (float)(g.oz + (bzn - 0.5) * g.h);
    for (int q = 0; q < 3; ++q) {      // widen by a few ulp so that rounding never cuts a centre off
        const float pad = 1e-6f * (fabsf(o.lo[q]) + fabsf(o.hi[q])) + 1e-9f;
        o.lo[q] -= pad; o.hi[q] += pad;
    }
    o.smax = g.sigma;
    o.t_begin = 0; o.t_end = o.bdx * o.bdy * o.bdz;
    o.pad = 0;
    si[s] = o;
}

// 1.5 * 2^23: adding it to |x| < 2^22 with rounding toward +inf leaves ceil(x) in the low bits.
constexpr float FL_MAGIC = 12582912.0f;
constexpr int FL_MAGIC_BITS = 0x4B400000;

// LF > 0: the correlation for windows of at most LF positions with the outputs in a register
// ring of LF (the table's coefficients are compile-time operands); LF = 0: any window length.
template <int P, int LF>
__global__ void __launch_bounds__(FL_MAXW * 32, 1)
fwd_lanes_kernel(GaussDev g, ArrDev a, const SlabInfo* __restrict__ slabs, float* __restrict__ partial,
                 int2* __restrict__ rows, int LB, int NZ, int* status, int use_tma,
                 const __grid_constant__ CUtensorMap tmap, const __grid_constant__ MomentTable T) {
    static_assert(P >= 6 && P <= 8, "6 to 8 moments");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FlHdr& S = *reinterpret_cast<FlHdr*>(smem_raw);
    const int NW = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = T.L, Lp = fl_lpad(L);
    float* cs = reinterpret_cast<float*>(smem_raw + FL_HDR);                     // [Lp][8]
    unsigned char* wbase = smem_raw + FL_HDR + (size_t)Lp * 32 + (size_t)warp * fl_warp_bytes(NZ, LB, P);
    ZBand<P> Z;
    Z.init(wbase, NZ);
    float* Y = reinterpret_cast<float*>(wbase + fl_zbytes(NZ, P));              // [LB][32]

    const int slab = blockIdx.y;
    const int j = (blockIdx.x * NW + warp) * 32 + lane;
    const bool has_sensor = j < a.Nd;
    const SlabInfo sl = slabs[slab];
    const int nCubes = sl.t_end;
    const size_t row = (size_t)slab * a.Nd + (has_sensor ? j : 0);

    // this lane's sample band for the slab: [w, w + LB), w a multiple of 4
    float sx = 0.f, sy = 0.f, sz = 0.f;
    int n_lo = 0, n_hi = -1;
    if (has_sensor) {
        sx = a.xyz[3 * j]; sy = a.xyz[3 * j + 1]; sz = a.xyz[3 * j + 2];
        if (nCubes > 0) {
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
    const int w = n_lo & ~3;
    const bool active = has_sensor && n_lo <= n_hi;
    if (active && n_hi + 1 - w > LB) set_status(status, DEV_CAPACITY);   // cannot happen with the host's LB
    const int LBe = active ? min(min(LB, a.Nt - w), n_hi + 1 - w) : 0;     // Y entries this lane keeps
    // the row keeps the band's own samples only (the rest of the signal band stays zero)
    if (has_sensor) rows[row] = make_int2(w, LBe);

    if (threadIdx.x == 0) {
        S.abort = 0;
        for (int b = 0; b < FL_RING; ++b) {
            S.released[b] = 0;
            S.issued[b] = -1;
            mbar_init(&S.full[b], 1);
        }
        fence_mbar_init();
    }
    for (int q = threadIdx.x; q < Lp * 8; q += blockDim.x) {
        const int m = q >> 3, p = q & 7;
        cs[q] = (m < L && p < P) ? T.c[m][p] : 0.f;
    }
    for (int i = 0; i <= NZ; ++i) Z.clear(i * 32 + lane);
    for (int q = 0; q < LB; ++q) Y[q * 32 + lane] = 0.f;
    __syncthreads();

    const bool tma = use_tma != 0;
    auto fill = [&](int TT) {      // warp-cooperative fill of the slot of cube TT
        const int b = TT % FL_RING;
        const int cx = sl.bx0 + TT % sl.bdx, cy = sl.by0 + (TT / sl.bdx) % sl.bdy, cz = sl.bz0 + TT / (sl.bdx * sl.bdy);
        if (tma) {
            if (lane == 0) {
                S.issued[b] = TT;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_expect_tx(&S.full[b], CUBE_N * sizeof(float));
                tma_load_3d(&S.tileA[b][0], &tmap, cx * CUBE, cy * CUBE, cz * CUBE, &S.full[b]);
            }
        } else {
            for (int q = lane; q < CUBE_N; q += 32) {
                const int gx = cx * CUBE + (q & 7), gy = cy * CUBE + ((q >> 3) & 7), gz = cz * CUBE + (q >> 6);
                const bool ok = gx < g.nx && gy < g.ny && gz < g.nz;
                S.tileA[b][q] = ok ? g.A[((int64_t)gz * g.ny + gy) * g.nx + gx] : 0.f;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.full[b]);
        }
    };
    if (warp == 0)
        for (int TT = 0; TT < FL_RING && TT < nCubes; ++TT) fill(TT);

    const float Delta = a.Delta, invDelta = a.invDelta;
    const float c2 = -0.72134752044448170368f / (g.sigma * g.sigma);     // -1 / (2 sigma^2 ln 2)
    const float ks = a.k * g.sigma;
    const float ksi = ks * invDelta;
    const float radc = cube_radius(g.h);
    const float ED = (float)T.E * Delta;
    const float efac = edge_factor(T);
    const bool edge_in = T.edge_in != 0;
    const float h = g.h;
    const int NO = NZ + L - 1;                 // outputs of one cube's band

    bool ok = true;
    for (int t = 0; t < nCubes; ++t) {
        const int b = t % FL_RING;
        if (!mbar_wait(&S.full[b], (uint32_t)((t / FL_RING) & 1))) {
            ok = false;
            break;
        }
        const int cx = sl.bx0 + t % sl.bdx, cy = sl.by0 + (t / sl.bdx) % sl.bdy, cz = sl.bz0 + t / (sl.bdx * sl.bdy);
        // FP64 reference of (cube centre, this lane's sensor)
        const PairRef r = make_ref(g.ox + (cx * CUBE + CUBE / 2) * (double)h, g.oy + (cy * CUBE + CUBE / 2) * (double)h,
                                   g.oz + (cz * CUBE + CUBE / 2) * (double)h, sx, sy, sz, a);
        // band base: zb = n0 + fl0, fl0 one below the lowest window-start offset of the cube
        const float fl0 = floorf((r.phi0 - radc - ks) * invDelta) - 1.f;
        const float magk = FL_MAGIC - fl0;     // exact: |fl0| is small
        const int zb = r.n0 + (int)fl0;
        const int yoff = zb - w;               // signal-band index of output o is yoff + o
        // separable parts of num = 2 (c0 - s) . delta + |delta|^2 over the cube's lattice offsets
        float ax[CUBE];
#pragma unroll
        for (int l = 0; l < CUBE; ++l) {
            const float o = ((float)l - 0.5f * (CUBE - 1)) * h;
            ax[l] = o * fmaf(2.f, r.v0x, o);
        }
        const float* tile = S.tileA[b];
        unsigned relmax = 0;       // largest band offset of the cube's pairs (as unsigned: negatives too)
        // a cube without amplitudes adds nothing (sparse images): the warp skips it
        bool any = false;
#pragma unroll
        for (int q = 0; q < CUBE_N / 32 / 4; ++q) {
            const float4 v = reinterpret_cast<const float4*>(tile)[lane * (CUBE_N / 32 / 4) + q];
            any |= (v.x != 0.f) | (v.y != 0.f) | (v.z != 0.f) | (v.w != 0.f);
        }
        const bool cube_on = __any_sync(0xffffffffu, any);
        // The pairs of lattice row `row` (= 8 lz + ly, 8 Gaussians along x) without branches: their
        // moments, band slots and the row's extreme e on the edge's side.
        auto row_pairs = [&](int row, float (&mom)[CUBE][P], int (&idx)[CUBE], float (&ev)[CUBE], float& eext) {
            const int lz = row >> 3, ly = row & (CUBE - 1);
            const float4 a0 = *reinterpret_cast<const float4*>(tile + row * CUBE);
            const float4 a1 = *reinterpret_cast<const float4*>(tile + row * CUBE + 4);
            const float Arow[CUBE] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float oy = ((float)ly - 0.5f * (CUBE - 1)) * h, oz = ((float)lz - 0.5f * (CUBE - 1)) * h;
            const float ayz = fmaf(oy, fmaf(2.f, r.v0y, oy), oz * fmaf(2.f, r.v0z, oz));
            eext = edge_in ? 3.f : -3.f;
#pragma unroll
            for (int lx = 0; lx < CUBE; ++lx) {
                const float num = ax[lx] + ayz;
                float invR, phi;
                pair_phase_num(r, num, invR, phi);
                const float tt = fmaf(phi, invDelta, -ksi);      // window start: first d <= k sigma
                const float u = __fadd_ru(tt, magk);              // magk + ceil(tt)
                const float mf = u - magk;
                const int rel = __float_as_int(u) - FL_MAGIC_BITS;   // ceil(tt) - fl0
                const float d0 = fmaf(-mf, Delta, phi);
                const float e = (d0 - T.dstar) * T.inv_half;
                // rel lies in [0, NZ) by the band's bound; a clamp keeps any other value inside the
                // band, and the kernel then reports the capacity status
                const unsigned ur = (unsigned)rel;
                relmax = max(relmax, ur);
                idx[lx] = (int)min(ur, (unsigned)(NZ - 1)) * 32 + lane;
                mom[lx][0] = Arow[lx] * invR;                      // the table carries the 1/2
#pragma unroll
                for (int p = 1; p < P; ++p) mom[lx][p] = mom[lx][p - 1] * e;
                ev[lx] = e;
                eext = edge_in ? fminf(eext, e) : fmaxf(eext, e);
            }
        };
        if (active && cube_on) {
            // Software pipeline over the cube's 64 rows, two per step: the next row's pairs are
            // formed while the current row's read-modify-writes (a chain through shared memory)
            // are in flight.  Rows needing the edge correction are marked and redone afterwards.
            float momA[CUBE][P], momB[CUBE][P], evA[CUBE], evB[CUBE], eA, eB;
            int idxA[CUBE], idxB[CUBE];
            unsigned long long emask = 0;
            row_pairs(0, momA, idxA, evA, eA);
#pragma unroll 1
            for (int row = 0; row < CUBE * CUBE; row += 2) {
                row_pairs(row + 1, momB, idxB, evB, eB);
#pragma unroll
                for (int k = 0; k < CUBE; k += 2) Z.add2(idxA[k], idxA[k + 1], momA[k], momA[k + 1]);
                emask |= (unsigned long long)edge_corrected(T, eA) << row;
                row_pairs((row + 2) & (CUBE * CUBE - 1), momA, idxA, evA, eA);   // row 64: a dummy row 0
#pragma unroll
                for (int k = 0; k < CUBE; k += 2) Z.add2(idxB[k], idxB[k + 1], momB[k], momB[k + 1]);
                emask |= (unsigned long long)edge_corrected(T, eB) << (row + 1);
            }
            // edge position E (rare at the benchmark's geometry): the direct term of the marked rows
            while (emask) {
                const int row = __ffsll(emask) - 1;
                emask &= emask - 1;
                row_pairs(row, momA, idxA, evA, eA);
#pragma unroll
                for (int lx = 0; lx < CUBE; ++lx)
                    if (edge_corrected(T, evA[lx])) {
                        const float dE = fmaf(evA[lx], 0.5f * Delta, T.dstar) - ED;   // d0 - E Delta
                        const int yi = yoff + (idxA[lx] >> 5) + T.E;
                        if ((unsigned)yi < (unsigned)LBe)
                            Y[yi * 32 + lane] += efac * momA[lx][0] * dE * ex2_approx(dE * dE * c2);
                    }
            }
        }
        if (relmax >= (unsigned)NZ) set_status(status, DEV_CAPACITY);   // a pair outside its band: not reached
        // release the slot; the warp that releases it last refills it with cube t + FL_RING
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = (atomicAdd(&S.released[b], 1) + 1) % NW == 0;
            if (last) __threadfence_block();
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last && t + FL_RING < nCubes) fill(t + FL_RING);
        if (active && cube_on) {
        if constexpr (LF > 0) {
        // correlation of the cube's moment band into the signal band, bin by bin: bin b adds
        // c[m] . Z[b] to output b + m for m < LF; acc[m] holds output b + m, so output b (acc[0])
        // is complete once bin b is in, and the ring shifts by one (the bin loop unrolled by 2, so
        // that half of the shift is register renaming).  Each bin is cleared as it is read.
        float acc[LF];
#pragma unroll
        for (int q = 0; q < LF; ++q) acc[q] = 0.f;
#pragma unroll 2
        for (int b = 0; b < NZ; ++b) {
            float z[8];
            Z.load(b * 32 + lane, z);
            Z.clear(b * 32 + lane);
#pragma unroll
            for (int m = 0; m < LF; ++m) {
                float v = acc[m];
#pragma unroll
                for (int p = 0; p < P; ++p) v = fmaf(T.c[m][p], z[p], v);
                acc[m] = v;
            }
            const int yi = yoff + b;
            if ((unsigned)yi < (unsigned)LBe) Y[yi * 32 + lane] += acc[0];
#pragma unroll
            for (int m = 0; m < LF - 1; ++m) acc[m] = acc[m + 1];
            acc[LF - 1] = 0.f;
        }
        // outputs NZ .. NZ + L - 2 are in acc[0 .. L - 2]
#pragma unroll
        for (int q = 0; q < LF - 1; ++q) {
            const int n = NZ + q;
            const int yi = yoff + n;
            if (n < NO && (unsigned)yi < (unsigned)LBe) Y[yi * 32 + lane] += acc[q];
        }
        } else {
        // correlation of the cube's moment band into the signal band, FL_Q outputs at a time:
        // acc[q] = sum_m c[m] . Z[c0 + q - m]; a ring of FL_Q bins in registers, slot (q - m) mod FL_Q
        for (int c0 = 0; c0 < NO; c0 += FL_Q) {
            float acc[FL_Q];
            float zw[FL_Q][P];
#pragma unroll
            for (int q = 0; q < FL_Q; ++q) {
                acc[q] = 0.f;
                float mm8[8];
                const int i = c0 + q;
                Z.load((i < NZ ? i : NZ) * 32 + lane, mm8);
#pragma unroll
                for (int p = 0; p < P; ++p) zw[q][p] = mm8[p];
            }
            for (int m0 = 0; m0 < Lp; m0 += FL_Q) {
#pragma unroll
                for (int mm = 0; mm < FL_Q; ++mm) {
                    const int m = m0 + mm;
                    const float4 ca = *reinterpret_cast<const float4*>(cs + m * 8);
                    const float4 cb = *reinterpret_cast<const float4*>(cs + m * 8 + 4);
                    const float cm[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
#pragma unroll
                    for (int q = 0; q < FL_Q; ++q) {
                        const int s = (q - mm) & (FL_Q - 1);
                        float v = acc[q];
#pragma unroll
                        for (int p = 0; p < P; ++p) v = fmaf(cm[p], zw[s][p], v);
                        acc[q] = v;
                    }
                    // the slot of bin c0 + 7 - m takes bin c0 - m - 1 for the next step
                    const int i = c0 - m - 1;
                    float mm8[8];
                    Z.load(((unsigned)i < (unsigned)NZ ? i : NZ) * 32 + lane, mm8);
#pragma unroll
                    for (int p = 0; p < P; ++p) zw[(FL_Q - 1 - mm) & (FL_Q - 1)][p] = mm8[p];
                }
            }
#pragma unroll
            for (int q = 0; q < FL_Q; ++q) {
                const int yi = yoff + c0 + q;
                if (c0 + q < NO && (unsigned)yi < (unsigned)LBe) Y[yi * 32 + lane] += acc[q];
            }
        }
        for (int i = 0; i < NZ; ++i) Z.clear(i * 32 + lane);
        }
        }
    }
    if (!ok && lane == 0) {   // a bounded wait ran out
        set_status(status, DEV_TIMEOUT);
        S.abort = 1;
    }
    __syncthreads();
    if (S.abort) {
        // wait (bounded) for the last copy issued into each slot before the CTA exits
        if (tma && threadIdx.x == 0)
            for (int b = 0; b < FL_RING; ++b)
                if (S.issued[b] >= 0) mbar_wait(&S.full[b], (uint32_t)((S.issued[b] / FL_RING) & 1));
        return;
    }
    if (active) {
        float4* prow = reinterpret_cast<float4*>(partial + row * LB);
        for (int q = 0; q < LBe; q += 4)      // LB is a multiple of 4, entries past LBe are zero
            prow[q >> 2] = make_float4(Y[q * 32 + lane], Y[(q + 1) * 32 + lane], Y[(q + 2) * 32 + lane],
                                       Y[(q + 3) * 32 + lane]);
    }
}

// ------------------------------------------------------------------------------------------
// Host side.

size_t fwd_lanes_smem(int NW, int NZ, int LB, int P, int L) { return fl_smem_bytes(NW, NZ, LB, P, L); }
int fwd_lanes_nz(float h, float invDelta) { return fl_nz(h, invDelta); }
float fwd_lanes_cube_radius(float h) { return cube_radius(h); }

cudaError_t launch_slab_info_cubes(const GaussDev& g, int scx, int scy, int scz, int S, SlabInfo* si, cudaStream_t st) {
    const int ncx = (g.nx + CUBE - 1) / CUBE, ncy = (g.ny + CUBE - 1) / CUBE, ncz = (g.nz + CUBE - 1) / CUBE;
    const int nsx = (ncx + scx - 1) / scx, nsy = (ncy + scy - 1) / scy;
    slab_info_cube_kernel<<<(S + 127) / 128, 128, 0, st>>>(g, ncx, ncy, ncz, scx, scy, scz, nsx, nsy, S, si);
    return cudaGetLastError();
}

cudaError_t launch_forward_lanes(const GaussDev& g, const ArrDev& a, const SlabInfo* si, int S, float* partial,
                                 int2* rows, int LB, int NZ, int NW, int* status, const CUtensorMap* tmap,
                                 const MomentTable& T, cudaStream_t st) {
    static const CUtensorMap zero_map = [] { CUtensorMap z; memset(&z, 0, sizeof(z)); return z; }();
    const size_t smem = fl_smem_bytes(NW, NZ, LB, T.P, T.L);
    dim3 grid((a.Nd + 32 * NW - 1) / (32 * NW), S);
    const bool l16 = T.L <= 16;     // the table is zero beyond L: a 16-slot ring serves any L <= 16
    auto kern = T.P == 6 ? (l16 ? fwd_lanes_kernel<6, 16> : fwd_lanes_kernel<6, 0>)
              : T.P == 7 ? (l16 ? fwd_lanes_kernel<7, 16> : fwd_lanes_kernel<7, 0>)
                         : (l16 ? fwd_lanes_kernel<8, 16> : fwd_lanes_kernel<8, 0>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 32 * NW, smem, st>>>(g, a, si, partial, rows, LB, NZ, status, tmap != nullptr,
                                      tmap ? *tmap : zero_map, T);
    return cudaGetLastError();
}

}  // namespace gp
