// adjoint.cu -- exact transpose of the windowed forward operator and the closed-form
// gradients with respect to amplitude, centre and width (Methods, adjoint operator; the
// derivatives of Eq. single_forward).
//
// Work decomposition: one CTA per tile of 256 Gaussians, one thread per Gaussian.  The CTA
// walks all sensors in chunks of 32: warp 0 forms the 32 FP64 (tile, sensor) references, the
// CTA stages each sensor's residual band (the samples the tile can touch) in shared memory,
// and every thread gathers its own pair windows from those bands.  Each Gaussian's sums over a
// chunk's sensors are FP32, Kahan-compensated across chunks in registers, and written once: no
// global atomics.  Free-centre Gaussians are taken in the order of their window length (a
// counting sort of the tile in shared memory), so the 32 threads of a warp walk windows of about
// the same length.
#include "gpair_internal.cuh"

namespace gp {

constexpr int ADJ_THREADS = TILE;
constexpr int ADJ_SC = 32;   // sensors staged per chunk
constexpr int ADJ_KEYS = 64; // window-length keys of the free-centre ordering
constexpr float ADJ_MAGIC = 12582912.0f;    // 1.5 * 2^23: x + MAGIC, rounded up (down), holds ceil(x) (floor(x))
constexpr int ADJ_MAGIC_BITS = 0x4B400000;



// Window sums of one pair: s1 = sum dl d e (amplitude gradient); with FULL also s0 = sum dl e,
// s2 = sum dl d^2 e, s3 = sum dl d^3 e (centre and width gradients).  src[m] is the residual at
// sample n0 + m; d = phi - m Delta is the pair's phase there.  Samples go two at a time through
// packed FP32 pairs (mul/add/fma .f32x2), the even and odd samples in the two halves of each
// accumulator; an odd window's last pair has its second residual set to zero.
template <bool FULL>
__device__ __forceinline__ void window_sums(const float* __restrict__ src, int m_lo, int m_hi, float phi,
                                            float Delta, float c2, float& s0, float& s1, float& s2, float& s3) {
    float2 fm = make_float2((float)m_lo, (float)(m_lo + 1));     // m as floats, stepped exactly
    const float2 two = make_float2(2.f, 2.f), nD = make_float2(-Delta, -Delta), cc = make_float2(c2, c2);
    const float2 ph = make_float2(phi, phi);
    float2 S0 = make_float2(0.f, 0.f), S1 = S0, S2 = S0, S3 = S0;
    for (int m = m_lo; m <= m_hi; m += 2, fm = __fadd2_rn(fm, two)) {
        const float2 d = __ffma2_rn(fm, nD, ph);
        const float2 E = __fmul2_rn(__fmul2_rn(d, d), cc);
        const float x0 = src[m], x1 = m + 1 <= m_hi ? src[m + 1] : 0.f;
        const float2 u = __fmul2_rn(make_float2(x0, x1), make_float2(ex2_approx(E.x), ex2_approx(E.y)));
        if (FULL) {
            const float2 ud = __fmul2_rn(u, d);
            const float2 udd = __fmul2_rn(ud, d);
            S0 = __fadd2_rn(S0, u);
            S1 = __fadd2_rn(S1, ud);
            S2 = __fadd2_rn(S2, udd);
            S3 = __ffma2_rn(udd, d, S3);
        } else {
            S1 = __ffma2_rn(u, d, S1);
        }
    }
    s1 += S1.x + S1.y;
    if (FULL) {
        s0 += S0.x + S0.y;
        s2 += S2.x + S2.y;
        s3 += S3.x + S3.y;
    }
}

// The same sums over a window held in a staged band, in the scaled phase s = sc d
// (sc = sqrt(log2(e) / 2) / sigma, so that exp(-d^2 / 2 sigma^2) = 2^(-s^2)): S0 = sum dl e,
// S1 = sum dl s e, S2 = sum dl s^2 e, S3 = sum dl s^3 e.  band[c] is the residual at band index
// c; the window is [c_lo, c_hi] with s_lo the scaled phase at c_lo and step = sc Delta.  The walk
// reads the band two samples at a time as one aligned float2, from the even index at or below
// c_lo up to the pair holding c_hi (band[c_hi + 1] must exist): only the first and the last pair
// can hold a sample outside the window, and only those two are masked.
template <bool FULL>
__device__ __forceinline__ void band_sums(const float* __restrict__ band, int c_lo, int c_hi, float s_lo, float step,
                                          float& s0, float& s1, float& s2, float& s3) {
    const int ca = c_lo & ~1;
    const int NI = ((c_hi - ca) >> 1) + 1;                      // pairs walked (c_hi >= c_lo)
    const float2* bp = reinterpret_cast<const float2*>(band + ca);
    const float sa = (c_lo & 1) ? s_lo + step : s_lo;           // scaled phase at index ca
    float2 s = make_float2(sa, sa - step);
    const float2 ds = make_float2(-2.f * step, -2.f * step);
    float2 S0 = make_float2(0.f, 0.f), S1 = S0, S2 = S0, S3 = S0;
    auto pair = [&](float2 x) {
        const float2 ss = __fmul2_rn(s, s);
        const float2 u = __fmul2_rn(x, make_float2(ex2_approx(-ss.x), ex2_approx(-ss.y)));
        if (FULL) {
            const float2 us = __fmul2_rn(u, s);
            const float2 uss = __fmul2_rn(us, s);
            S0 = __fadd2_rn(S0, u);
            S1 = __fadd2_rn(S1, us);
            S2 = __fadd2_rn(S2, uss);
            S3 = __ffma2_rn(uss, s, S3);
        } else {
            S1 = __ffma2_rn(u, s, S1);
        }
        s = __fadd2_rn(s, ds);
    };
    const int last_hi = ca + 2 * (NI - 1) + 1;                  // second index of the last pair
    float2 x = bp[0];
    if (c_lo & 1) x.x = 0.f;
    if (NI == 1 && last_hi > c_hi) x.y = 0.f;
    pair(x);
    for (int q = 1; q < NI - 1; ++q) pair(bp[q]);
    if (NI > 1) {
        x = bp[NI - 1];
        if (last_hi > c_hi) x.y = 0.f;
        pair(x);
    }
    s1 += S1.x + S1.y;
    if (FULL) {
        s0 += S0.x + S0.y;
        s2 += S2.x + S2.y;
        s3 += S3.x + S3.y;
    }
}

template <bool GRID, bool FULL>
__global__ void __launch_bounds__(ADJ_THREADS, 4)
adj_kernel(GaussDev g, ArrDev a, const TileInfo* __restrict__ ti, const float* __restrict__ delta,
           float* __restrict__ gA, float* __restrict__ gc, float* __restrict__ gs, int LBA) {
    extern __shared__ __align__(16) float bands[];   // [ADJ_SC][LBA]
    __shared__ PairRef refs[ADJ_SC];
    __shared__ int nbs[ADJ_SC];
    __shared__ int hist[ADJ_KEYS], perm[ADJ_THREADS];

    const int64_t t = blockIdx.x;
    const int l0 = threadIdx.x, warp = l0 >> 5, lane = l0 & 31;
    const TileInfo rt = ti[t];
    // free centres: thread l0 takes the tile's Gaussian perm[l0], in the order of window length
    // (2 k sigma / Delta, clamped to the key range; invalid entries last)
    int l = l0;
    if (!GRID) {
        const int64_t i0 = t * TILE + l0;
        const int key = i0 < g.M ? min(ADJ_KEYS - 1, (int)(2.f * a.k * g.sg[i0] * a.invDelta)) : ADJ_KEYS - 1;
        for (int q = l0; q < ADJ_KEYS; q += ADJ_THREADS) hist[q] = 0;
        __syncthreads();
        const int rank = atomicAdd(&hist[key], 1);
        __syncthreads();
        if (l0 == 0)
            for (int q = 0, acc = 0; q < ADJ_KEYS; ++q) { const int c = hist[q]; hist[q] = acc; acc += c; }
        __syncthreads();
        perm[hist[key] + rank] = l0;
        __syncthreads();
        l = perm[l0];
    }

    // This thread's Gaussian: index, amplitude, width and offset from the tile reference.
    bool valid;
    int64_t i;
    float Ai, sig, dx, dy, dz;
    double c0x, c0y, c0z;
    if (GRID) {
        const int tx = (int)(t % g.ntx), ty = (int)((t / g.ntx) % g.nty), tz = (int)(t / ((int64_t)g.ntx * g.nty));
        const int gx = tx * BX + (l & (BX - 1)), gy = ty * BY + ((l / BX) & (BY - 1)), gz = tz * BZ + l / (BX * BY);
        valid = gx < g.nx && gy < g.ny && gz < g.nz;
        i = ((int64_t)gz * g.ny + gy) * g.nx + gx;
        Ai = valid ? g.A[i] : 0.f;
        sig = g.sigma;
        brick_offset(l, g.h, dx, dy, dz);
        c0x = g.ox + (tx * BX + BX / 2) * (double)g.h;
        c0y = g.oy + (ty * BY + BY / 2) * (double)g.h;
        c0z = g.oz + (tz * BZ + BZ / 2) * (double)g.h;
    } else {
        i = t * TILE + l;
        valid = i < g.M;
        Ai = valid ? g.A[i] : 0.f;
        sig = valid ? g.sg[i] : 1.f;
        dx = valid ? g.cx[i] - rt.c0x : 0.f;
        dy = valid ? g.cy[i] - rt.c0y : 0.f;
        dz = valid ? g.cz[i] - rt.c0z : 0.f;
        c0x = rt.c0x; c0y = rt.c0y; c0z = rt.c0z;
    }
    const float c2 = -0.72134752044448170368f / (sig * sig);   // -log2(e) / (2 sigma^2)
    const float inv_s2 = 1.f / (sig * sig), inv_s3 = inv_s2 / sig;
    const float ks = a.k * sig;
    const float Delta = a.Delta, invDelta = a.invDelta;
    const float sc = 0.84932180028801904272f / sig;             // sqrt(log2(e) / 2) / sigma
    const float isc = 1.f / sc, step = sc * Delta;
    const float ksi = ks * invDelta;
    const float reach = rt.rad + a.k * rt.smax;                // farthest |d| offset in the tile

    KahanF kA, kX, kY, kZ, kS;
    for (int j0 = 0; j0 < a.Nd; j0 += ADJ_SC) {
        const int nsc = min(ADJ_SC, a.Nd - j0);
        if (warp == 0 && lane < nsc) {
            const int j = j0 + lane;
            const PairRef r = make_ref(c0x, c0y, c0z, a.xyz[3 * j], a.xyz[3 * j + 1], a.xyz[3 * j + 2], a);
            refs[lane] = r;
            nbs[lane] = (r.n0 + (int)floorf((r.phi0 - reach) * invDelta) - 2) & ~3;
        }
        __syncthreads();
        for (int q = 0; q < nsc; ++q) {
            const float* dj = delta + (size_t)(j0 + q) * a.Nt;
            for (int c = l0; c < LBA; c += ADJ_THREADS) {
                const int n = nbs[q] + c;
                bands[q * LBA + c] = (n >= 0 && n < a.Nt) ? dj[n] : 0.f;
            }
        }
        __syncthreads();
        if (valid) {
            float aA = 0.f, aX = 0.f, aY = 0.f, aZ = 0.f, aS = 0.f;   // FP32 over the chunk
            for (int q = 0; q < nsc; ++q) {
                const PairRef r = refs[q];
                float invR, phi;
                pair_phase_fast(r, dx, dy, dz, invR, phi);
                // window [w_lo, w_hi] in samples from n0 (the forward's rounding of its ends)
                const float tt = phi * invDelta;
                const float ulo = __fadd_ru(tt - ksi, ADJ_MAGIC), uhi = __fadd_rd(tt + ksi, ADJ_MAGIC);
                const int w_lo = __float_as_int(ulo) - ADJ_MAGIC_BITS, w_hi = __float_as_int(uhi) - ADJ_MAGIC_BITS;
                const int off = r.n0 - nbs[q];
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
                if (w_lo <= w_hi) {
                    if ((off + w_lo >= 0) && (off + w_hi + 1 < LBA)) {
                        // the band is zero outside the record: no clamp; sums in the scaled phase
                        band_sums<FULL>(bands + q * LBA, off + w_lo, off + w_hi,
                                        sc * fmaf(-(ulo - ADJ_MAGIC), Delta, phi), step, s0, s1, s2, s3);
                        s1 *= isc;
                        if (FULL) { s2 *= isc * isc; s3 *= isc * isc * isc; }
                    } else {
                        const int m_lo = max(w_lo, -r.n0), m_hi = min(w_hi, a.Nt - 1 - r.n0);
                        window_sums<FULL>(delta + (size_t)(j0 + q) * a.Nt + r.n0, m_lo, m_hi, phi, Delta, c2, s0, s1,
                                          s2, s3);
                    }
                }
                const float inv2R = 0.5f * invR;
                aA = fmaf(s1, inv2R, aA);
                if (FULL) {
                    const float wA = Ai * inv2R;
                    const float gR = wA * (s0 - s2 * inv_s2) - wA * s1 * invR;
                    const float gRi = gR * invR;
                    aX = fmaf(gRi, r.v0x + dx, aX);
                    aY = fmaf(gRi, r.v0y + dy, aY);
                    aZ = fmaf(gRi, r.v0z + dz, aZ);
                    aS = fmaf(wA * s3, inv_s3, aS);
                }
            }
            kA.add(aA);
            if (FULL) { kX.add(aX); kY.add(aY); kZ.add(aZ); kS.add(aS); }
        }
        __syncthreads();
    }
    if (valid) {
        gA[i] = kA.s;
        if (FULL) {
            if (gc) {
                gc[i] = kX.s;
                gc[g.M + i] = kY.s;
                gc[2 * g.M + i] = kZ.s;
            }
            if (gs) gs[i] = kS.s;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Amplitude gradient for a grid with shared sigma through the sub-sample expansion
// (MomentTable): for a pair whose window starts at sample b with offset e,
//     sum_m delta[b + m] K(d0 - m Delta) = sum_p e^p Q_p[b] (+ the conditional last position),
//     Q_p[b] = sum_{m < L} delta[b + m] c[m][p],
// so one table of L-tap correlations per sensor replaces the per-sample evaluation.

// The table is split by term so that a warp's gathers of nearby window starts touch as few
// cache lines as possible: Qa[j][b + L] holds Q_0 .. Q_3 (16 bytes), Qb[j][b + L] the rest (Q_4,
// Q_5 as 8 bytes for P = 6; Q_4 .. Q_7 as 16 bytes for P = 7, 8), for window starts b in
// [-L, N_t); the residual is zero outside the record.  Qb starts N_d (N_t + L) float4 after Qa.
__host__ __device__ __forceinline__ size_t adj_qb_offset(int Nd, int Nt, int L) { return (size_t)Nd * (Nt + L); }

template <int P>
__global__ void __launch_bounds__(256)
adj_q_kernel(const float* __restrict__ delta, int Nt, const __grid_constant__ MomentTable T, float* __restrict__ Q) {
    extern __shared__ float sd[];   // residual samples b0 .. b0 + 256 + L
    const int j = blockIdx.y;
    const int L = T.L;
    const int b0 = -L + blockIdx.x * 256;
    const float* dj = delta + (size_t)j * Nt;
    for (int q = threadIdx.x; q < 256 + L; q += blockDim.x) {
        const int n = b0 + q;
        sd[q] = (n >= 0 && n < Nt) ? dj[n] : 0.f;
    }
    __syncthreads();
    const int b = b0 + (int)threadIdx.x;
    if (b >= Nt) return;
    float acc[MOM_P];
#pragma unroll
    for (int p = 0; p < MOM_P; ++p) acc[p] = 0.f;     // acc[p >= P] stays 0
    for (int m = 0; m < L; ++m) {
        const float dl = sd[threadIdx.x + m];
#pragma unroll
        for (int p = 0; p < P; ++p) acc[p] = fmaf(dl, T.c[m][p], acc[p]);
    }
    const size_t e = (size_t)j * (Nt + L) + (b + L);
    float4* Qa = reinterpret_cast<float4*>(Q);
    Qa[e] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    if constexpr (P == 6) reinterpret_cast<float2*>(Qa + adj_qb_offset(gridDim.y, Nt, L))[e] = make_float2(acc[4], acc[5]);
    else (Qa + adj_qb_offset(gridDim.y, Nt, L))[e] = make_float4(acc[4], acc[5], acc[6], acc[7]);
}

// One CTA per brick of 256 grid Gaussians, one thread per Gaussian, all sensors in chunks of 32.
template <int P>
__global__ void __launch_bounds__(ADJ_THREADS, 5)
adj_moment_kernel(GaussDev g, ArrDev a, const float* __restrict__ delta, const float* __restrict__ Q,
                  const __grid_constant__ MomentTable T, float* __restrict__ gA) {
    __shared__ PairRef refs2[2][ADJ_SC];
    const int64_t t = blockIdx.x;
    const int l = threadIdx.x, warp = l >> 5, lane = l & 31;
    const int tx = (int)(t % g.ntx), ty = (int)((t / g.ntx) % g.nty), tz = (int)(t / ((int64_t)g.ntx * g.nty));
    // warp w takes a 4 x 4 x 2 block of the 8 x 8 x 4 brick (w's bits: x half, y half, z pair), so
    // that the window starts of its 32 Gaussians for one sensor -- the table rows it gathers -- stay
    // close together for every direction of the cap
    static_assert(BX == 8 && BY == 8 && BZ == 4 && ADJ_THREADS == 256, "brick of 8 x 8 x 4, 8 warps");
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
    const float ks = a.k * g.sigma, Delta = a.Delta, invDelta = a.invDelta;
    const float c2 = -0.72134752044448170368f / (g.sigma * g.sigma);
    const int L = T.L, Nt = a.Nt;
    const float ED = (float)T.E * Delta;
    const float ksi = ks * invDelta;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));   // references below carry 2 (c0 - s)
    const float4* Qa = reinterpret_cast<const float4*>(Q);
    const size_t qb_off = adj_qb_offset(a.Nd, Nt, L);
    KahanF kA;
    // References are double-buffered: after each barrier the last warp forms the next chunk's
    // FP64 references while the others already work on the current chunk.
    if (warp == ADJ_THREADS / 32 - 1 && lane < min(ADJ_SC, a.Nd))
        refs2[0][lane] = ref_doubled(make_ref(c0x, c0y, c0z, a.xyz[3 * lane], a.xyz[3 * lane + 1], a.xyz[3 * lane + 2], a));
    int cur = 0;
    for (int j0 = 0; j0 < a.Nd; j0 += ADJ_SC, cur ^= 1) {
        const int nsc = min(ADJ_SC, a.Nd - j0);
        __syncthreads();
        if (warp == ADJ_THREADS / 32 - 1 && j0 + ADJ_SC + lane < a.Nd) {
            const int j = j0 + ADJ_SC + lane;
            refs2[cur ^ 1][lane] = ref_doubled(make_ref(c0x, c0y, c0z, a.xyz[3 * j], a.xyz[3 * j + 1], a.xyz[3 * j + 2], a));
        }
        const PairRef* refs = refs2[cur];
        if (valid) {
            float acc = 0.f;         // FP32 over the chunk's 32 sensors, Kahan across chunks
            constexpr int UNROLL = P <= 7 ? 4 : 2;   // 8 terms need the registers of the deeper unroll
#pragma unroll UNROLL
            for (int q = 0; q < nsc; ++q) {
                const PairRef r = refs[q];
                float invR, phi;
                pair_phase_pre(r, dx, dy, dz, d2, invR, phi);
                const float mf = ceilf(fmaf(phi, invDelta, -ksi));   // as the forward
                const int b = r.n0 + (int)mf;
                if (b < -L || b >= Nt) continue;
                const float d0 = fmaf(-mf, Delta, phi);
                const float e = (d0 - T.dstar) * T.inv_half;
                const size_t qe = (size_t)(j0 + q) * (Nt + L) + (b + L);
                const float4 q0 = __ldg(Qa + qe);
                float s;
                if constexpr (P == 6) {
                    const float2 q1 = __ldg(reinterpret_cast<const float2*>(Qa + qb_off) + qe);
                    s = fmaf(q1.y, e, q1.x);
                } else {
                    const float4 q1 = __ldg(Qa + qb_off + qe);
                    if constexpr (P == 8) s = fmaf(fmaf(fmaf(q1.w, e, q1.z), e, q1.y), e, q1.x);
                    else s = fmaf(fmaf(q1.z, e, q1.y), e, q1.x);
                }
                s = fmaf(s, e, q0.w);
                s = fmaf(s, e, q0.z);
                s = fmaf(s, e, q0.y);
                s = fmaf(s, e, q0.x);
                if (edge_corrected(T, e)) {            // edge position E: rare direct correction
                    const float dE = d0 - ED;
                    const int n = b + T.E;
                    if (n >= 0 && n < Nt)
                        s = fmaf(edge_factor(T) * delta[(size_t)(j0 + q) * Nt + n] * dE, ex2_approx(dE * dE * c2), s);
                }
                acc = fmaf(s, invR, acc);
            }
            kA.add(acc);
        }
    }
    if (valid) gA[i] = kA.s;                 // the table carries the 1/2 of A / 2R
}

size_t adj_moment_q_bytes(const ArrDev& a, int L) { return (size_t)a.Nd * (a.Nt + L) * MOM_P * sizeof(float); }

cudaError_t launch_adjoint_moment(const GaussDev& g, const ArrDev& a, const float* delta, float* gA,
                                  const MomentTable& T, float* Q, const cudaEvent_t* ev, cudaStream_t st) {
    dim3 qgrid((a.Nt + T.L + 255) / 256, a.Nd);
    if (T.P == 6) adj_q_kernel<6><<<qgrid, 256, (256 + T.L) * sizeof(float), st>>>(delta, a.Nt, T, Q);
    else if (T.P == 7) adj_q_kernel<7><<<qgrid, 256, (256 + T.L) * sizeof(float), st>>>(delta, a.Nt, T, Q);
    else adj_q_kernel<8><<<qgrid, 256, (256 + T.L) * sizeof(float), st>>>(delta, a.Nt, T, Q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    if (T.P == 6) adj_moment_kernel<6><<<(unsigned)g.ntiles, ADJ_THREADS, 0, st>>>(g, a, delta, Q, T, gA);
    else if (T.P == 7) adj_moment_kernel<7><<<(unsigned)g.ntiles, ADJ_THREADS, 0, st>>>(g, a, delta, Q, T, gA);
    else adj_moment_kernel<8><<<(unsigned)g.ntiles, ADJ_THREADS, 0, st>>>(g, a, delta, Q, T, gA);
    e = cudaGetLastError();
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
    return e;
}

int adj_band_len(float rad, float smax, float k, float invDelta) {
    int half = (int)ceilf((rad + k * smax) * invDelta) + 4;
    int lb = 2 * half + 8;
    return (lb + 3) & ~3;
}

cudaError_t launch_adjoint(const GaussDev& g, const ArrDev& a, const TileInfo* ti, const float* delta, float* gA,
                           float* gc, float* gs, int LBA, cudaStream_t st) {
    const bool full = gc != nullptr || gs != nullptr;
    size_t smem = (size_t)ADJ_SC * LBA * sizeof(float);
    unsigned blocks = (unsigned)g.ntiles;
    cudaError_t e = cudaSuccess;
#define GP_LAUNCH_ADJ(G, F)                                                                                   \
    do {                                                                                                      \
        e = cudaFuncSetAttribute(adj_kernel<G, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);   \
        if (e != cudaSuccess) return e;                                                                       \
        adj_kernel<G, F><<<blocks, ADJ_THREADS, smem, st>>>(g, a, ti, delta, gA, gc, gs, LBA);               \
    } while (0)
    if (g.grid) {
        if (full) GP_LAUNCH_ADJ(true, true); else GP_LAUNCH_ADJ(true, false);
    } else {
        if (full) GP_LAUNCH_ADJ(false, true); else GP_LAUNCH_ADJ(false, false);
    }
#undef GP_LAUNCH_ADJ
    return cudaGetLastError();
}

}  // namespace gp
