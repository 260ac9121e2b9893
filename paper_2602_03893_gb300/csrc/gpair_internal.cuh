// gpair_internal.cuh -- device-side types and helpers shared by the library's kernels.
//
// Geometry precision (Methods, Eq. single_forward): the phase d = R - v t_n of a pair cancels
// two numbers of ~10 cm to resolve ~10 nm, which FP32 alone cannot do.  Every tile of Gaussians
// therefore carries a reference point c0; for each (tile, sensor) the distance R0 = |c0 - s| and
// the phase phi0 = R0 - v t_{n0} at the nearest sample n0 are formed in FP64 once, and each
// Gaussian adds its small offset delta = c - c0 in FP32 through the cancellation-free form
//     R - R0 = (2 (c0 - s) . delta + |delta|^2) / (R + R0).
// The remaining per-sample phase d_m = phi0 + (R - R0) - m * (v / fs) is a sum of small FP32
// terms, accurate to ~1e-10 m.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gpair.h"

namespace gp {

// Tile of Gaussians processed together.  Grid mode: a BX x BY x BZ brick of lattice nodes
// (loaded by one 3-D TMA copy); SoA mode: TILE consecutive Gaussians.
constexpr int TILE = 256;
constexpr int BX = 8, BY = 8, BZ = 4;
static_assert(BX * BY * BZ == TILE, "brick must hold one tile");

// Device status word values (set by kernels, read by gpair_last_device_status).
constexpr int DEV_OK = 0;
constexpr int DEV_TIMEOUT = 1;
constexpr int DEV_CAPACITY = 2;

// Bounded wait: iterations of mbarrier.try_wait before a kernel gives up and flags TIMEOUT.
constexpr uint32_t WAIT_LIMIT = 1u << 24;

struct GaussDev {
    int grid;                // 1: grid-implicit centres and shared sigma
    int64_t M;
    const float *cx, *cy, *cz, *sg, *A;
    int nx, ny, nz;          // grid mode
    float h, sigma;
    double ox, oy, oz;
    int ntx, nty, ntz;       // bricks per axis (grid mode)
    int64_t ntiles;
};

struct ArrDev {
    int Nd;
    const float* xyz;
    float v, fs, t0;
    int Nt;
    float k;
    float Delta;             // v / fs: metres per sample
    float invDelta;          // fs / v
    double fs_v, t0fs;       // fs / v and t0 fs, for the reference sample n0
    double vt0, dlt;         // v t0 and v / fs, for the reference phase
};

// Per-tile summary: reference point (float, so that FP64 differences with it are exact), the
// radius of the tile about it, the widest sigma and the number of valid Gaussians.
struct TileInfo {
    float c0x, c0y, c0z;
    float rad;
    float smax;
    int count;
    int pad0, pad1;
};

// A slab is the set of tiles one forward CTA walks.  Grid mode: a block of bdx x bdy x bdz
// bricks starting at brick (bx0, by0, bz0) (compact, so its band of samples is short).  SoA mode:
// the contiguous tile range [t_begin, t_end).  lo/hi bound the Gaussian centres; smax is the
// widest sigma.
struct SlabInfo {
    float lo[3], hi[3];
    float smax;
    int t_begin, t_end;
    int bx0, by0, bz0;
    int bdx, bdy, bdz;
    int pad;
};

// Per-(tile, sensor) reference, formed in FP64 and rounded once.
struct PairRef {
    float v0x, v0y, v0z;     // c0 - s
    float R0;                // |c0 - s|
    float phi0;              // R0 - v t_{n0}
    int n0;                  // nearest sample to the time of flight of c0
};

// Sub-sample expansion of the windowed pulse for a shared sigma.  A pair's window starts at the
// first sample whose phase d0 satisfies d0 <= k sigma, so d0 lies in (k sigma - Delta, k sigma].
// Writing d0 = dstar + e * Delta / 2 with dstar = k sigma - Delta / 2 and e in (-1, 1], the
// pulse K(d) = d exp(-d^2 / 2 sigma^2) at window position m is a smooth function of e, replaced
// by a polynomial of degree P - 1,
//     K(d0 - m Delta) ~ sum_p c[m][p] e^p,
// the Chebyshev-point fit of the host (make_moment_table), whose largest error over every
// position and offset stays below 3e-7 of the pulse's peak (P = 6 at Delta = 0.375 sigma, the
// 0.1 mm / 40 MHz workloads; 7 or 8 up to Delta = sigma / 2).  Positions
// m < E = floor(2 k sigma / Delta) are always inside the window, position E is inside when
// d0 - E Delta >= -k sigma (for a fraction 2 k sigma / Delta - E of the pairs), later positions
// never.  The table covers positions m < L: L = E + 1 when position E is inside for most pairs
// (edge_in = 1; the pairs for which it is outside subtract its term, evaluated directly), else
// L = E (the pairs for which it is inside add its term).  The coefficients carry the factor 1/2 of
// the weight A / 2R, so that a pair's weight is A / R.
constexpr int MOM_P = 8;
constexpr int MOM_LMAX = 128;
struct MomentTable {
    int P;                       // terms used (6, 7 or 8; c[m][p] = 0 for p >= P)
    int L;                       // positions covered by the expansion
    int E;                       // edge position
    int edge_in;                 // 1: the table covers position E
    float dstar, inv_half;       // reference phase and 2 / Delta
    float e_thr;                 // position E is inside a pair's window iff e >= e_thr
    float c[MOM_LMAX][MOM_P];
};

// Edge position E is inside a pair's window when d0 >= E Delta - k sigma, i.e. e >= e_thr.  A pair
// needs the direct correction when that differs from edge_in; its factor is then -1/2 (subtract,
// edge_in = 1) or +1/2 (add), times (A / R) dE exp(-dE^2 / 2 sigma^2), dE = d0 - E Delta.  Forward
// and adjoint take the decision from the same e, so they stay exact transposes.
__device__ __forceinline__ bool edge_corrected(const MomentTable& T, float e) {
    return (e >= T.e_thr) != (T.edge_in != 0);
}
__device__ __forceinline__ float edge_factor(const MomentTable& T) { return T.edge_in ? -0.5f : 0.5f; }

// The paper's discretised operator (Methods, adaptive supersampling alignment): pulse centres
// snapped to a grid ALPHA times finer than fs, pulse sampled there over |k| <= K.
// hr[t] = h[K - t], t = 0..2K, with h[k] = (1/2) d exp(-d^2 / 2 sigma^2), d = -v k / (alpha fs).
constexpr int ASSA_KMAX = 256;
struct AssaTable {
    int alpha, K, n_half;
    float hr[2 * ASSA_KMAX + 1];
};

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Largest |n0| kept; the host limits n_samples to 2^27, so every window-bound expression of the
// kernels (w - n0, Nt - 1 - n0, ...) stays inside int32.
constexpr double N0_CLAMP = 268435456.0;   // 2^28

// Reference for tile centre c0 and sensor s, in FP64 (GB300 runs FP64 at a small fraction of the
// FP32 rate, so the reference avoids double division and square root).  R0 = |c0 - s| from one
// Newton-Raphson step y1 = y0 (3 - q y0^2) / 2 for 1 / sqrt(q), started from the FP32 rsqrt
// (relative error ~1e-7 -> ~1e-14); n0 is the nearest sample up to rounding (any nearby integer
// serves: phi0 is formed from the same n0); phi0 = R0 - v (t0 + n0 / fs) with v t0 and v / fs
// from the host (error ~1e-15 m).
__device__ __forceinline__ PairRef make_ref(double c0x, double c0y, double c0z, float sx, float sy,
                                            float sz, const ArrDev& a) {
    double vx = c0x - (double)sx, vy = c0y - (double)sy, vz = c0z - (double)sz;
    const double q = fma(vx, vx, fma(vy, vy, vz * vz));
    double R0;
    if (q > 1e-30) {
        const double y0 = (double)rsqrtf((float)q);
        const double y1 = y0 * fma(-0.5 * q, y0 * y0, 1.5);
        R0 = q * y1;
    } else {
        R0 = sqrt(q);
    }
    double n0 = rint(fma(R0, a.fs_v, -a.t0fs));
    n0 = fmin(fmax(n0, -N0_CLAMP), N0_CLAMP);
    double phi = fma(-n0, a.dlt, R0 - a.vt0);
    PairRef r;
    r.v0x = (float)vx; r.v0y = (float)vy; r.v0z = (float)vz;
    r.R0 = (float)R0;
    r.phi0 = (float)phi;
    r.n0 = (int)n0;
    return r;
}

// Radius of a grid brick about its centre (with a little slack for rounding).
__host__ __device__ __forceinline__ float brick_radius(float h) {
    const float hx = 0.5f * (BX - 1), hy = 0.5f * (BY - 1), hz = 0.5f * (BZ - 1);
    return sqrtf(hx * hx + hy * hy + hz * hz) * h * 1.0001f + 1e-9f;
}

// Offset of Gaussian l of a grid brick from the brick's reference point (the brick centre).
__device__ __forceinline__ void brick_offset(int l, float h, float& dx, float& dy, float& dz) {
    int lx = l & (BX - 1), ly = (l / BX) & (BY - 1), lz = l / (BX * BY);
    dx = ((float)lx - 0.5f * (BX - 1)) * h;
    dy = ((float)ly - 0.5f * (BY - 1)) * h;
    dz = ((float)lz - 0.5f * (BZ - 1)) * h;
}

// Phase of a pair at the reference sample n0 (d at m = 0) and R, from the reference and the
// Gaussian's offset (see the header comment).
__device__ __forceinline__ void pair_phase(const PairRef& r, float dx, float dy, float dz,
                                           float& R, float& phi) {
    float num = dx * (2.f * r.v0x + dx) + dy * (2.f * r.v0y + dy) + dz * (2.f * r.v0z + dz);
    R = sqrtf(fmaf(r.R0, r.R0, num));
    float dR = num / (r.R0 + R);
    phi = r.phi0 + dR;
}

// Same as pair_phase with hardware reciprocal square root and reciprocal (a few ulp): returns
// 1/R (for the weight A/2R) and the phase.  The relative error of 1/R is ~1e-7; the phase
// correction R - R0 (at most a few mm) keeps an absolute error of ~1e-10 m.
// Second half of pair_phase_fast, from num = R^2 - R0^2 = 2 (c0 - s) . delta + |delta|^2.
__device__ __forceinline__ void pair_phase_num(const PairRef& r, float num, float& invR, float& phi) {
    const float R2 = fmaf(r.R0, r.R0, num);
    invR = rsqrtf(R2);
    const float R = R2 * invR;
    float rc;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rc) : "f"(r.R0 + R));
    phi = fmaf(num, rc, r.phi0);
}

// Shared per-(tile, sensor) reference of the adjoints that give each thread one Gaussian: 2 (c0 - s)
// (doubled exactly), R0, phi0, the reference sample n0 plus a kernel-specific offset, and the
// sensor's first entry in the kernel's table; 32 bytes, read as two 16-byte loads.
struct __align__(16) AdjRef {
    float v2x, v2y, v2z, R0;
    float phi0;
    int n0;      // n0 + the kernel's offset
    int row;     // the sensor's row in the kernel's table
    int pad;
};

__device__ __forceinline__ AdjRef adj_ref(const PairRef& r, int n0, int row) {
    AdjRef a;
    a.v2x = 2.f * r.v0x; a.v2y = 2.f * r.v0y; a.v2z = 2.f * r.v0z;
    a.R0 = r.R0;
    a.phi0 = r.phi0;
    a.n0 = n0;
    a.row = row;
    a.pad = 0;
    return a;
}

// Phase and 1 / R of the pair of a thread's Gaussian (offset with |delta|^2 = d2) and a reference.
__device__ __forceinline__ void pair_phase_r(const AdjRef& r, float dx, float dy, float dz, float d2, float& invR,
                                             float& phi) {
    const float num = fmaf(dx, r.v2x, fmaf(dy, r.v2y, fmaf(dz, r.v2z, d2)));
    const float R2 = fmaf(r.R0, r.R0, num);
    invR = rsqrtf(R2);
    const float R = R2 * invR;
    float rc;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rc) : "f"(r.R0 + R));
    phi = fmaf(num, rc, r.phi0);
}

// Reference with v0 doubled (exact in FP32) for pair_phase_pre.
__device__ __forceinline__ PairRef ref_doubled(PairRef r) {
    r.v0x *= 2.f; r.v0y *= 2.f; r.v0z *= 2.f;
    return r;
}

// pair_phase_fast for a thread that owns one Gaussian: r from ref_doubled, d2 = |delta|^2 of the
// thread's offset, so that num = 2 (c0 - s) . delta + |delta|^2 takes three FMAs.
__device__ __forceinline__ void pair_phase_pre(const PairRef& r2, float dx, float dy, float dz, float d2,
                                               float& invR, float& phi) {
    pair_phase_num(r2, fmaf(dx, r2.v0x, fmaf(dy, r2.v0y, fmaf(dz, r2.v0z, d2))), invR, phi);
}

__device__ __forceinline__ void pair_phase_fast(const PairRef& r, float dx, float dy, float dz,
                                                float& invR, float& phi) {
    const float num = dx * (2.f * r.v0x + dx) + dy * (2.f * r.v0y + dy) + dz * (2.f * r.v0z + dz);
    const float R2 = fmaf(r.R0, r.R0, num);
    invR = rsqrtf(R2);
    const float R = R2 * invR;
    float rc;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rc) : "f"(r.R0 + R));
    phi = fmaf(num, rc, r.phi0);
}

// Nearest and farthest distance from a sensor to a slab's box of Gaussian centres (FP64).
__device__ __forceinline__ void box_distance(const SlabInfo& sl, float sx, float sy, float sz,
                                             double& dmin, double& dmax) {
    double s[3] = {sx, sy, sz}, mn = 0, mx = 0;
    for (int q = 0; q < 3; ++q) {
        double lo = sl.lo[q], hi = sl.hi[q];
        double a = lo - s[q], b = s[q] - hi;
        double out = a > 0 ? a : (b > 0 ? b : 0.0);
        mn += out * out;
        double far = fabs(s[q] - lo) > fabs(s[q] - hi) ? fabs(s[q] - lo) : fabs(s[q] - hi);
        mx += far * far;
    }
    dmin = sqrt(mn);
    dmax = sqrt(mx);
}

// Tile t (0-based within the slab) -> brick coordinates (grid mode).
__device__ __forceinline__ void slab_brick(const SlabInfo& sl, int t, int& tx, int& ty, int& tz) {
    tx = sl.bx0 + t % sl.bdx;
    ty = sl.by0 + (t / sl.bdx) % sl.bdy;
    tz = sl.bz0 + t / (sl.bdx * sl.bdy);
}

// Kahan-compensated FP32 sum.
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Number of SMs of the current device (cudaDevAttrMultiProcessorCount, queried once per device and
// cached); grid sizes and reduction partial counts are multiples of it.  Host only; returns 1 if the
// query fails, so launches stay valid.
int device_sms();

// Device scratch of the calling stream (one pool per device and stream, shared by every call on
// that stream, so stream order keeps its users apart), at least `bytes` long.  Host only.
gpair_status stream_scratch(cudaStream_t st, size_t bytes, void** buf);

__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicMax(status, code);
}

// ---- mbarrier / TMA helpers (sm_90+ PTX; used single-CTA, no multicast) -------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Plain arrive (release semantics at CTA scope): completes a phase of a count-1 barrier after
// the calling thread's (and, after a __syncwarp, its warp's) shared-memory stores.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// Returns true when the phase with the given parity has completed, false after `limit`
// unsuccessful polls.
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, uint32_t parity, uint32_t limit) {
    uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(addr), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) { return mbar_wait_n(bar, parity, WAIT_LIMIT); }

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(smem_u32(dst)), "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace gp
