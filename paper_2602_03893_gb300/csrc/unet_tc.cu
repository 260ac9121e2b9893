// unet_tc.cu -- the U-Net's 3-D convolution as an implicit GEMM on the 5th-generation tensor
// cores (tcgen05.mma kind::f16: BF16 operands, FP32 accumulators in tensor memory), fed by TMA.
//
// Rows of one MMA: 16 halo positions along x x 8 along y of one z-slice (128 voxels); K: 16 input
// channels; columns: for a 3 x 3 x 3 stencil the NT output channels of the three x-taps of one
// (dz, dy), N = 3 NT.  Row (x', y) then holds, in column block dx, the (dz, dy, dx) terms of input
// x' for all (dz, dy), and output x = x' - dx + 1 is the sum over dx of row x + dx, block dx: the
// epilogue adds the three blocks with lane shuffles, and 14 of the 16 positions are outputs.  So a
// tile is 14 x 8 x ZT output voxels and NT channels, and nine MMAs per slice and K step replace 27.
// The CTA stages the tile's input halo (16 x 10 x (ZT + 2) voxels, KC channels) with one TMA load
// in the layout [8-channel chunk][z][y][x][8 channels]: a core matrix (8 voxels consecutive in x,
// 16 bytes each) is contiguous, and the operand of (dz, dy) and slice zs is the same K-major layout
// ((zs + dz) 10 + dy) 16 rows further in.  Shifting the descriptor replaces the im2col copy; the
// zero padding is the TMA's out-of-range fill.  The weights of the stage (taps x NT x KC) arrive by
// a second TMA load as [8-channel chunk][tap][co][8], so the rows (dx, co) of one (dz, dy) are
// consecutive.  When one stage holds every input channel, the weights are loaded once per CTA and
// stay resident.  A 1 x 1 x 1 convolution uses the same tile without halo (16 x 8 outputs, N = NT).
// For channel tiles NT > 32 (where three column blocks leave room for one slice only) the kernel
// takes the other tiling (MODE 0): rows 8 along x x 16 along y, a 10 x 18 x (ZT + 2) halo, one MMA
// per tap with N = NT, the dx shift also a descriptor offset.
//
// Warp roles of the persistent CTA: warp 0 issues the TMA loads into a ring of stages, warp 1
// owns tensor memory and issues the MMAs (one thread), warps 2-5 drain the accumulators
// (tcgen05.ld; warp w reads TMEM lanes 32 (w mod 4) ...), add the bias, apply the ReLU and store
// BF16.  Two accumulator buffers in tensor memory let the epilogue of one tile overlap the MMAs of
// the next.  Every wait is bounded; after a wait gives up, its warp sets the status word and
// skips its remaining waits, so the CTA runs to its end.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gpair_internal.cuh"

namespace gp {

constexpr int TC_THREADS = 192;      // 6 warps: TMA, MMA, 4 x epilogue
constexpr int TC_TX = 8, TC_TY = 16; // weight-gradient tile in x and y
constexpr int FW_XR = 16, FW_TY = 8; // forward: MMA rows per slice, 16 along x x 8 along y
constexpr int TC_MAX_STAGES = 4;
constexpr size_t TC_SMEM_MAX = 227 * 1024;

__device__ int g_conv_tc_status;     // 1: a bounded wait gave up

// Shared-memory matrix descriptor, no swizzle: start address, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1 at bits 46-47, layout type 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at bits 17-22, M / 16 at bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int N, int M) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void* tmap, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const void* tmap, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
        ::"r"(dst), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint16_t f2bf_rn(float f) {
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    return *reinterpret_cast<const uint16_t*>(&h);
}

struct ConvTcArgs {
    int D, H, W, Cout;
    int NT, N, ZT, KC, nK;          // channel tile, MMA columns, z-slices per tile, channels per stage, stages
    int tiles_x, tiles_y, n_tiles;  // spatial tiles along x and y, channel tiles
    int64_t units;                  // spatial tiles x channel tiles
    int nstages;                    // ring depth
    uint32_t a_bytes, a_stride;     // halo box bytes, and its slot size (128-byte multiple)
    uint32_t b_bytes;               // weight box bytes
    uint32_t tmem_cols;
    int b_resident;                 // nK == 1: weights loaded once per CTA
    int relu;
    const float* bias;
    uint16_t* out;
};

// Shared memory: [ring of stages: halo (a_stride) + weights (b_bytes, unless resident)]
// [resident weights] [barriers: full, empty per stage; acc_full, acc_empty x 2; weights] [tmem slot]
template <int TAPS, int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
conv3d_fwd_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const ConvTcArgs p) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int R = TAPS == 27 ? 1 : 0;                         // halo width
    constexpr int NX = (TAPS == 27 && MODE == 1) ? 3 : 1;         // x-taps per MMA (column blocks)
    constexpr int RX = MODE == 1 ? FW_XR : TC_TX;                 // MMA rows along x (then along y)
    constexpr int RY = 128 / RX;
    constexpr int HX = MODE == 1 ? RX : RX + 2 * R, HY = RY + 2 * R;   // halo box in x and y
    constexpr int TXO = MODE == 1 ? RX - 2 * R : RX;              // outputs per tile along x
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = p.nstages;
    const uint32_t stage_bytes = p.a_stride + (p.b_resident ? 0u : p.b_bytes);
    unsigned char* bres = sm + (size_t)NS * stage_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(bres + (p.b_resident ? p.b_bytes : 0u));
    uint64_t* empty = full + TC_MAX_STAGES;
    uint64_t* acc_full = empty + TC_MAX_STAGES;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* wbar = acc_empty + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(wbar + 1);

    if (threadIdx.x == 0) {
        for (int q = 0; q < NS; ++q) { mbar_init(&full[q], 1); mbar_init(&empty[q], 1); }
        for (int q = 0; q < 2; ++q) { mbar_init(&acc_full[q], 1); mbar_init(&acc_empty[q], 4); }
        mbar_init(wbar, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(p.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;
    const int ntile_xy = p.tiles_x * p.tiles_y;

    if (warp == 0) {
        // ---- TMA producer
        if (lane == 0) {
            if (p.b_resident) {
                mbar_arrive_expect_tx(wbar, p.b_bytes);
                tma_load_4d(smem_u32(bres), &tmB, 0, 0, 0, 0, wbar);     // n_tiles == 1 when resident
            }
            int s = 0;
            uint32_t ph = 0;
            for (int64_t u = blockIdx.x; u < p.units; u += gridDim.x) {
                const int nt = (int)(u % p.n_tiles);
                const int64_t st = u / p.n_tiles;
                const int tx = (int)(st % p.tiles_x), ty = (int)((st / p.tiles_x) % p.tiles_y);
                const int tz = (int)(st / ntile_xy);
                for (int k = 0; k < p.nK; ++k) {
                    if (ok && !mbar_wait(&empty[s], ph ^ 1u)) ok = false;
                    const uint32_t dst = smem_u32(sm + (size_t)s * stage_bytes);
                    mbar_arrive_expect_tx(&full[s], p.a_bytes + (p.b_resident ? 0u : p.b_bytes));
                    tma_load_5d(dst, &tmA, 0, tx * TXO - R, ty * RY - R, tz * p.ZT - R, k * (p.KC / 8), &full[s]);
                    if (!p.b_resident) tma_load_4d(dst + p.a_stride, &tmB, 0, nt * p.NT, 0, k * (p.KC / 8), &full[s]);
                    if (++s == NS) { s = 0; ph ^= 1u; }
                }
            }
            // every load issued has landed before the CTA ends (the MMA warp waited on each; this
            // only matters after a wait gave up)
            for (int q = 0; q < NS; ++q) {
                int s2 = s - 1 - q;
                uint32_t ph2 = ph;
                if (s2 < 0) { s2 += NS; ph2 ^= 1u; }
                mbar_wait_n(&full[s2], ph2, WAIT_LIMIT / 16);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc_idesc(p.N, 128);
            const uint32_t lboA = p.a_bytes / (p.KC / 8);        // one 8-channel chunk of the halo
            const uint32_t lboB = (uint32_t)(TAPS * p.NT * 16);  // one 8-channel chunk of the weights
            if (p.b_resident && ok && !mbar_wait(wbar, 0)) ok = false;
            int s = 0, ab = 0;
            uint32_t ph = 0, aph = 0;
            for (int64_t u = blockIdx.x; u < p.units; u += gridDim.x) {
                if (ok && !mbar_wait(&acc_empty[ab], aph ^ 1u)) ok = false;
                tc_fence_after();
                const uint32_t dcol = tmem + (uint32_t)(ab * p.ZT * p.N);
                for (int k = 0; k < p.nK; ++k) {
                    if (ok && !mbar_wait(&full[s], ph)) ok = false;
                    tc_fence_after();
                    const uint32_t aaddr = smem_u32(sm + (size_t)s * stage_bytes);
                    const uint32_t baddr = p.b_resident ? smem_u32(bres) : aaddr + p.a_stride;
                    // 8-row groups: MODE 1 (x-octet, y) 128 bytes apart; MODE 0 one y-row apart
                    const uint64_t a0 = smem_desc(aaddr, lboA, MODE == 1 ? 128 : HX * 16);
                    const uint64_t b0 = smem_desc(baddr, lboB, 128);
                    for (int zs = 0; zs < p.ZT; ++zs) {
                        const uint64_t az = a0 + (uint64_t)(zs * HY * HX);      // 16-byte units
                        for (int kk = 0; kk < p.KC / 16; ++kk) {
                            const uint64_t ak = az + (uint64_t)(kk * 2 * (lboA >> 4));
                            const uint64_t bk = b0 + (uint64_t)(kk * 2 * (lboB >> 4));
#pragma unroll
                            for (int g = 0; g < TAPS / NX; ++g) {   // MODE 1: g = 3 dz + dy, taps 3g ... 3g + 2
                                int dz = 0, dy = 0, dx = 0;
                                if (TAPS == 27) {
                                    if (MODE == 1) { dz = g / 3; dy = g % 3; }
                                    else { dz = g / 9; dy = (g / 3) % 3; dx = g % 3; }
                                }
                                const uint64_t at = ak + (uint64_t)((dz * HY + dy) * HX + dx);
                                const uint64_t bt = bk + (uint64_t)(g * NX * p.NT);
                                tc_mma(dcol + (uint32_t)(zs * p.N), at, bt, idesc, (k | kk | g) != 0 ? 1u : 0u);
                            }
                        }
                    }
                    tc_commit(&empty[s]);         // the stage's slot is free once these MMAs are done
                    if (++s == NS) { s = 0; ph ^= 1u; }
                }
                tc_commit(&acc_full[ab]);
                if (++ab == 2) { ab = 0; aph ^= 1u; }
            }
        }
    } else {
        // ---- epilogue: TMEM lanes 32 q ... 32 q + 31, q = warp mod 4; lane m <-> row position
        // (m % RX, m / RX); in MODE 1 the 16 lanes of a y-row are consecutive, so rows x + 1, x + 2
        // are the lanes above
        const int q = warp & 3;
        const int m = 32 * q + lane;
        const int lx = m % RX, ly = m / RX;
        int ab = 0;
        uint32_t aph = 0;
        for (int64_t u = blockIdx.x; u < p.units; u += gridDim.x) {
            const int nt = (int)(u % p.n_tiles);
            const int64_t st = u / p.n_tiles;
            const int tx = (int)(st % p.tiles_x), ty = (int)((st / p.tiles_x) % p.tiles_y);
            const int tz = (int)(st / ntile_xy);
            if (ok && !mbar_wait(&acc_full[ab], aph)) ok = false;
            tc_fence_after();
            const int x = tx * TXO + lx, y = ty * RY + ly;
            const int n0 = nt * p.NT;
            for (int zs = 0; zs < p.ZT; ++zs) {
                const int z = tz * p.ZT + zs;
                const bool inb = lx < TXO && x < p.W && y < p.H && z < p.D;
                const int64_t o = inb ? (((int64_t)z * p.H + y) * p.W + x) * p.Cout + n0 : 0;
                for (int c0 = 0; c0 < p.NT; c0 += 16) {
                    const uint32_t col = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ab * p.ZT * p.N + zs * p.N + c0);
                    uint32_t r[16];
                    float v[16];
                    tc_ld16(col, r);
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
                    if (NX == 3) {
#pragma unroll
                        for (int dx = 1; dx < 3; ++dx) {
                            tc_ld16(col + (uint32_t)(dx * p.NT), r);
#pragma unroll
                            for (int i = 0; i < 16; ++i) v[i] += __shfl_down_sync(0xffffffffu, __uint_as_float(r[i]), dx);
                        }
                    }
                    if (inb) {
                        uint32_t pk[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            float o0 = v[2 * i], o1 = v[2 * i + 1];
                            if (p.bias) { o0 += p.bias[n0 + c0 + 2 * i]; o1 += p.bias[n0 + c0 + 2 * i + 1]; }
                            if (p.relu) { o0 = fmaxf(o0, 0.f); o1 = fmaxf(o1, 0.f); }
                            pk[i] = (uint32_t)f2bf_rn(o0) | ((uint32_t)f2bf_rn(o1) << 16);
                        }
                        uint4* d4 = reinterpret_cast<uint4*>(p.out + o + c0);
                        d4[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        d4[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ab]);
            if (++ab == 2) { ab = 0; aph ^= 1u; }
        }
    }
    if (!ok) atomicMax(&g_conv_tc_status, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols));
    }
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 conv_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

int channel_tile(int Cout) {
    if (Cout <= 64) return Cout;
    for (int nt : {64, 48, 32, 16})
        if (Cout % nt == 0) return nt;
    return 0;
}

uint32_t tmem_columns(int n) {
    uint32_t c = 32;
    while (c < (uint32_t)n) c <<= 1;
    return c;
}

}  // namespace

// Eligible shapes: Cin and Cout multiples of 16, 1 or 27 taps, 16-byte aligned tensors.  Returns
// cudaErrorNotSupported otherwise (the caller then uses the mma.sync kernel).
cudaError_t launch_conv3d_fwd_tc(const uint16_t* in, int D, int H, int W, int Cin, const uint16_t* w,
                                 const float* bias, int Cout, int taps, int relu, uint16_t* out, cudaStream_t st) {
    if (Cin % 16 != 0 || Cout % 16 != 0 || (taps != 27 && taps != 1)) return cudaErrorNotSupported;
    if (((uintptr_t)in | (uintptr_t)w | (uintptr_t)out) & 15) return cudaErrorNotSupported;
    const int NT = channel_tile(Cout);
    if (NT == 0) return cudaErrorNotSupported;
    auto enc = conv_encoder();
    if (!enc) return cudaErrorNotSupported;
    const int R = taps == 27 ? 1 : 0;
    const int MODE = (taps == 1 || NT <= 32) ? 1 : 0;
    const int NX = (taps == 27 && MODE == 1) ? 3 : 1;
    const int RX = MODE == 1 ? FW_XR : TC_TX, RY = 128 / RX;
    const int HX = MODE == 1 ? RX : RX + 2 * R, HY = RY + 2 * R, TXO = MODE == 1 ? RX - 2 * R : RX;
    const int N = NX * NT;
    const int sms = device_sms();
    const int tiles_x = (W + TXO - 1) / TXO, tiles_y = (H + RY - 1) / RY;
    const int n_tiles = Cout / NT;
    const size_t bar_bytes = 8 * (2 * TC_MAX_STAGES + 5) + 16;

    // z-slices per tile: the largest that keeps at least one unit per SM (two accumulator buffers
    // of ZT x N columns in the 512 of tensor memory); then the most channels per stage that let
    // two stages fit in shared memory.
    ConvTcArgs a{};
    int ZT = 8;
    while (ZT > 1 && (2 * ZT * N > 512 || (int64_t)((D + ZT - 1) / ZT) * tiles_x * tiles_y * n_tiles < sms)) ZT >>= 1;
    if (2 * ZT * N > 512) return cudaErrorNotSupported;
    int KC = 0;
    for (;;) {
        for (int kc = Cin; kc >= 16; kc -= 16) {
            if (Cin % kc != 0 || kc / 8 > 256) continue;
            const size_t abytes = (size_t)16 * HX * HY * (ZT + 2 * R) * (kc / 8);
            const size_t astr = (abytes + 1023) & ~(size_t)1023;
            const size_t bbytes = (size_t)taps * NT * kc * 2;
            const bool res = kc == Cin && n_tiles == 1;
            const size_t need = 2 * (astr + (res ? 0 : bbytes)) + (res ? bbytes : 0) + bar_bytes;
            if (need <= TC_SMEM_MAX) { KC = kc; break; }
        }
        if (KC || ZT == 1) break;
        ZT >>= 1;
    }
    if (KC == 0) return cudaErrorNotSupported;
    a.D = D; a.H = H; a.W = W; a.Cout = Cout;
    a.NT = NT; a.N = N; a.ZT = ZT; a.KC = KC; a.nK = Cin / KC;
    a.tiles_x = tiles_x; a.tiles_y = tiles_y; a.n_tiles = n_tiles;
    a.units = (int64_t)((D + ZT - 1) / ZT) * tiles_x * tiles_y * n_tiles;
    a.a_bytes = (uint32_t)(16 * HX * HY * (ZT + 2 * R) * (KC / 8));
    a.a_stride = (a.a_bytes + 1023u) & ~1023u;
    a.b_bytes = (uint32_t)(taps * NT * KC * 2);
    a.b_resident = (KC == Cin && n_tiles == 1) ? 1 : 0;
    a.tmem_cols = tmem_columns(2 * ZT * N);
    a.relu = relu;
    a.bias = bias;
    a.out = out;
    const size_t stage = a.a_stride + (a.b_resident ? 0 : a.b_bytes);
    int ns = (int)((TC_SMEM_MAX - bar_bytes - (a.b_resident ? a.b_bytes : 0)) / stage);
    a.nstages = ns < TC_MAX_STAGES ? ns : TC_MAX_STAGES;
    if (a.nstages < 2) return cudaErrorNotSupported;
    const size_t smem = (size_t)a.nstages * stage + (a.b_resident ? a.b_bytes : 0) + bar_bytes;

    // input halo: dims (8 channels, x, y, z, channel chunk), box (8, HX, HY, ZT + 2R, KC / 8);
    // out-of-range voxels read as zero
    CUtensorMap mA, mB;
    {
        cuuint64_t dims[5] = {8, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)(Cin / 8)};
        cuuint64_t strides[4] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2, 16};
        cuuint32_t box[5] = {8, (cuuint32_t)HX, (cuuint32_t)HY, (cuuint32_t)(ZT + 2 * R), (cuuint32_t)(KC / 8)};
        cuuint32_t es[5] = {1, 1, 1, 1, 1};
        if (enc(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<uint16_t*>(in), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
    }
    // weights w[co][tap][ci]: dims (8 channels, co, tap, channel chunk), box (8, NT, taps, KC / 8)
    {
        cuuint64_t dims[4] = {8, (cuuint64_t)Cout, (cuuint64_t)taps, (cuuint64_t)(Cin / 8)};
        cuuint64_t strides[3] = {(cuuint64_t)taps * Cin * 2, (cuuint64_t)Cin * 2, 16};
        cuuint32_t box[4] = {8, (cuuint32_t)NT, (cuuint32_t)taps, (cuuint32_t)(KC / 8)};
        cuuint32_t es[4] = {1, 1, 1, 1};
        if (enc(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t*>(w), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
    }
    auto kern = taps == 1 ? conv3d_fwd_tc_kernel<1, 1>
                          : (MODE == 1 ? conv3d_fwd_tc_kernel<27, 1> : conv3d_fwd_tc_kernel<27, 0>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = a.units < sms ? a.units : sms;
    kern<<<(unsigned)grid, TC_THREADS, smem, st>>>(mA, mB, a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Weight gradient: dW[co][t][ci] = sum_v dout[v][co] in[v + off(t)][ci], a GEMM whose rows are
// (tap, input channel), columns output channels and reduction the voxels.  Both operands are
// MN-major with the 32-byte swizzle: a voxel's 16 channels are one 32-byte row, 8 voxels
// consecutive in x one swizzle atom, which is how a TMA box [z][y][x][16 channels] with
// SWIZZLE_32B lands.  The rows of one MMA (M = 128) are 8 units of 16 input channels, each unit one
// TMA box of the input shifted by its tap; K = 16 is two x-rows of 8 voxels.  The columns are the
// output channels of NX = 3 dout boxes shifted by 1 - dx along x (or of one unshifted box, NX = 1,
// when 3 Cout > 256): with the reduction index u = v + dx - 1, the tap (dz, dy, dx) term is
// in[u + (0, dy - 1, dz - 1)] dout[u - dx + 1], so a unit is a (dz, dy) shift of the input and the
// three x-taps share it.  The terms left out at the volume's x faces multiply zero padding.
// CTA = (group of 128-row blocks held in tensor memory, range of voxel tiles): it accumulates
// over its tiles and writes its partial dW; wgrad_reduce_kernel sums the partials in fixed order.

constexpr int WG_THREADS = 128;        // warp 0: TMA, warp 1: MMA; all four drain tensor memory
constexpr int WG_UNITS = 8;            // (tap, 16-channel) units per 128-row block

struct WgradTcArgs {
    int Cin, Cout, taps, ZS;
    int tiles_x, tiles_y, n_tiles;     // voxel tiles of 8 x 16 x ZS
    int NX, N;                         // x-taps carried in the columns (3 or 1); columns = NX Cout
    int units, blocks;                 // (tap group, 16-channel) units = taps / NX Cin / 16; 128-row blocks
    int G, n_groups, n_splits;         // blocks per group (tensor memory), groups, voxel-tile splits
    int nstages;
    uint32_t unit_bytes, b_bytes, stage_bytes, tmem_cols;    // b_bytes: one dout box
    float* partial;                    // [split][taps * Cin][Cout]
};

// MN-major A and B (bits 15, 16), FP32 accumulator, BF16 operands.
// Shared-memory descriptor of an MN-major operand with the 32-byte swizzle (layout type 6 at bits
// 61-63): LBO = stride between 16-element (32-byte) atoms along M/N, SBO = stride between groups
// of 8 rows along K.
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    return smem_desc(saddr, lbo_bytes, sbo_bytes) | ((uint64_t)6 << 61);
}
__host__ __device__ constexpr uint32_t tc_idesc_mn(int N, int M) { return tc_idesc(N, M) | (1u << 15) | (1u << 16); }

template <int TAPS>
__global__ void __launch_bounds__(WG_THREADS, 1)
conv3d_wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmIn, const __grid_constant__ CUtensorMap tmOut,
                       const WgradTcArgs p) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int R = TAPS == 27 ? 1 : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = p.nstages;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + (size_t)NS * p.stage_bytes);
    uint64_t* empty = full + TC_MAX_STAGES;
    uint64_t* done = empty + TC_MAX_STAGES;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    const int grp = (int)(blockIdx.x % p.n_groups), split = (int)(blockIdx.x / p.n_groups);
    const int b0 = grp * p.G, b1 = min(p.blocks, b0 + p.G);
    const int t0 = (int)((int64_t)split * p.n_tiles / p.n_splits), t1 = (int)((int64_t)(split + 1) * p.n_tiles / p.n_splits);
    const int cp_per_tap = p.Cin / 16;

    if (threadIdx.x == 0) {
        for (int q = 0; q < NS; ++q) { mbar_init(&full[q], 1); mbar_init(&empty[q], 1); }
        mbar_init(done, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(p.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;

    if (warp == 0) {
        // lane 0 claims the slot and posts the byte count; lanes 0 ... 8 then issue one box each
        // (a box's issue has a fixed cost, so nine lanes keep nine in flight)
        int s = 0;
        uint32_t ph = 0;
        for (int tile = t0; tile < t1; ++tile) {
            const int tx = tile % p.tiles_x, ty = (tile / p.tiles_x) % p.tiles_y, tz = tile / (p.tiles_x * p.tiles_y);
            const int x0 = tx * TC_TX, y0 = ty * TC_TY, z0 = tz * p.ZS;
            for (int b = b0; b < b1; ++b) {
                const uint32_t dst = smem_u32(sm + (size_t)s * p.stage_bytes);
                const int nu = min(WG_UNITS, p.units - b * WG_UNITS);
                if (lane == 0) {
                    if (ok && !mbar_wait(&empty[s], ph ^ 1u)) ok = false;
                    mbar_arrive_expect_tx(&full[s], (uint32_t)nu * p.unit_bytes + (uint32_t)p.NX * p.b_bytes);
                }
                __syncwarp();
                if (lane < nu) {
                    const int U = b * WG_UNITS + lane;
                    const int g = U / cp_per_tap, cp = U - g * cp_per_tap;
                    int dz = 0, dy = 0, dx = R;        // NX = 3: unit g = 3 dz + dy, the x shift is dout's
                    if (TAPS == 27) {
                        if (p.NX == 3) { dz = g / 3; dy = g % 3; }
                        else { dz = g / 9; dy = (g / 3) % 3; dx = g % 3; }
                    }
                    tma_load_5d(dst + (uint32_t)lane * p.unit_bytes, &tmIn, 0, x0 + dx - R, y0 + dy - R, z0 + dz - R, cp,
                                &full[s]);
                } else if (lane >= WG_UNITS && lane < WG_UNITS + p.NX) {
                    const int j = lane - WG_UNITS;      // dout box of x-tap j: dout[u - j + 1]
                    tma_load_5d(dst + WG_UNITS * p.unit_bytes + (uint32_t)j * p.b_bytes, &tmOut, 0,
                                x0 + (p.NX == 3 ? 1 - j : 0), y0, z0, 0, &full[s]);
                }
                if (++s == NS) { s = 0; ph ^= 1u; }
            }
        }
        if (lane == 0)
            for (int q = 0; q < NS; ++q) {      // every load issued has landed before the CTA ends
                int s2 = s - 1 - q;
                uint32_t ph2 = ph;
                if (s2 < 0) { s2 += NS; ph2 ^= 1u; }
                mbar_wait_n(&full[s2], ph2, WAIT_LIMIT / 16);
            }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = tc_idesc_mn(p.N, 128);
        const int ksteps = TC_TX * TC_TY * p.ZS / 16;
        int s = 0;
        uint32_t ph = 0;
        for (int tile = t0; tile < t1; ++tile) {
            for (int b = b0; b < b1; ++b) {
                if (ok && !mbar_wait(&full[s], ph)) ok = false;
                tc_fence_after();
                const uint32_t aaddr = smem_u32(sm + (size_t)s * p.stage_bytes);
                // atoms of 16 channels one box (a unit, or 16 output channels) apart; 8-voxel row
                // groups 256 bytes apart; K = 16 voxels is 512 bytes, a whole number of swizzle repeats
                const uint64_t a0 = smem_desc_sw32(aaddr, p.unit_bytes, 256);
                const uint64_t bq = smem_desc_sw32(aaddr + WG_UNITS * p.unit_bytes, p.unit_bytes, 256);
                const uint32_t d = tmem + (uint32_t)((b - b0) * p.N);
                for (int kk = 0; kk < ksteps; ++kk)
                    tc_mma(d, a0 + (uint64_t)(kk * 32), bq + (uint64_t)(kk * 32), idesc,
                           (tile > t0 || kk > 0) ? 1u : 0u);
                tc_commit(&empty[s]);
                if (++s == NS) { s = 0; ph ^= 1u; }
            }
        }
        tc_commit(done);
    }
    __syncwarp();
    // drain: warp w holds TMEM lanes 32w ... 32w + 31, i.e. rows 32w + lane of each block
    if (t1 > t0) {
        if (ok && !mbar_wait(done, 0)) ok = false;
        tc_fence_after();
        const int rows = p.taps * p.Cin;
        for (int b = b0; b < b1; ++b) {
            // row 32 warp + lane of block b: unit U, input channel 16 cp + ci_in; column j Cout + co:
            // tap (dz, dy, j) (NX = 3) or the unit's own tap (NX = 1)
            const int mi = 32 * warp + lane;
            const int U = b * WG_UNITS + mi / 16;
            const bool valid = U < p.units;
            const int g = U / cp_per_tap, ci = (U - g * cp_per_tap) * 16 + (mi & 15);
            for (int j = 0; j < p.NX; ++j) {
                const int t = p.NX == 3 ? (g / 3) * 9 + (g % 3) * 3 + j : g;
                float* dst = p.partial + ((size_t)split * rows + (valid ? (size_t)t * p.Cin + ci : 0)) * p.Cout;
                for (int c0 = 0; c0 < p.Cout; c0 += 16) {
                    uint32_t r[16];
                    tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((b - b0) * p.N + j * p.Cout + c0), r);
                    if (valid) {
                        float4* d4 = reinterpret_cast<float4*>(dst + c0);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            d4[i] = make_float4(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1]),
                                                __uint_as_float(r[4 * i + 2]), __uint_as_float(r[4 * i + 3]));
                    }
                }
            }
        }
    }
    if (!ok) atomicMax(&g_conv_tc_status, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols));
    }
}

// dw[co][t][ci] += sum over splits (in order) of partial[split][t Cin + ci][co]
__global__ void wgrad_reduce_kernel(const float* __restrict__ partial, int n_splits, int rows, int Cout,
                                    float* __restrict__ dw) {
    const int64_t n = (int64_t)rows * Cout;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int co = (int)(i / rows), m = (int)(i - (int64_t)co * rows);   // dw index co * rows + m
        const float* src = partial + (size_t)m * Cout + co;
        const size_t step = (size_t)rows * Cout;
        float acc = 0.f;
        int s = 0;
        for (; s + 8 <= n_splits; s += 8) {      // eight loads in flight, added in split order
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = src[(size_t)(s + q) * step];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc += v[q];
        }
        for (; s < n_splits; ++s) acc += src[(size_t)s * step];
        dw[i] += acc;
    }
}

// Eligible: Cin and Cout multiples of 16, Cout <= 256, 1 or 27 taps, 16-byte aligned tensors.
// The partial sums live in the stream's scratch pool.
cudaError_t launch_conv3d_wgrad_tc(const uint16_t* in, const uint16_t* dout, int D, int H, int W, int Cin, int Cout,
                                   int taps, float* dw, cudaStream_t st) {
    if (Cin % 16 != 0 || Cout % 16 != 0 || Cout > 256 || (taps != 27 && taps != 1)) return cudaErrorNotSupported;
    if (((uintptr_t)in | (uintptr_t)dout) & 15) return cudaErrorNotSupported;
    auto enc = conv_encoder();
    if (!enc) return cudaErrorNotSupported;
    const int sms = device_sms();
    WgradTcArgs a{};
    const size_t bar_bytes = 8 * (2 * TC_MAX_STAGES + 1) + 16;
    a.Cin = Cin; a.Cout = Cout; a.taps = taps;
    a.NX = (taps == 27 && 3 * Cout <= 256) ? 3 : 1;
    a.N = a.NX * Cout;
    // the deepest tile (z-slices) for which two stages fit: fewer, larger boxes
    a.ZS = 2;
    while (a.ZS > 1 && 2 * ((size_t)WG_UNITS * 16 * 2 * TC_TX * TC_TY * a.ZS +
                            (size_t)a.NX * TC_TX * TC_TY * a.ZS * Cout * 2 + 1023) + bar_bytes > TC_SMEM_MAX)
        --a.ZS;
    a.tiles_x = (W + TC_TX - 1) / TC_TX; a.tiles_y = (H + TC_TY - 1) / TC_TY;
    a.n_tiles = a.tiles_x * a.tiles_y * ((D + a.ZS - 1) / a.ZS);
    a.units = taps / a.NX * Cin / 16;
    a.blocks = (a.units + WG_UNITS - 1) / WG_UNITS;
    a.G = 512 / a.N < a.blocks ? 512 / a.N : a.blocks;
    a.n_groups = (a.blocks + a.G - 1) / a.G;
    a.G = (a.blocks + a.n_groups - 1) / a.n_groups;        // even groups
    int ns = sms / a.n_groups;
    if (ns < 1) ns = 1;
    if (ns > a.n_tiles) ns = a.n_tiles;
    a.n_splits = ns;
    a.unit_bytes = (uint32_t)(16 * 2 * TC_TX * TC_TY * a.ZS);     // 16 channels x voxels x 2 B
    a.b_bytes = (uint32_t)(TC_TX * TC_TY * a.ZS * Cout * 2);
    a.stage_bytes = (WG_UNITS * a.unit_bytes + (uint32_t)a.NX * a.b_bytes + 1023u) & ~1023u;
    a.tmem_cols = tmem_columns(a.G * a.N);
    int nst = (int)((TC_SMEM_MAX - bar_bytes) / a.stage_bytes);
    a.nstages = nst < TC_MAX_STAGES ? nst : TC_MAX_STAGES;
    if (a.nstages < 2 || a.tmem_cols > 512) return cudaErrorNotSupported;
    const size_t smem = (size_t)a.nstages * a.stage_bytes + bar_bytes;
    const int rows = taps * Cin;
    void* scratch = nullptr;
    if (stream_scratch(st, (size_t)a.n_splits * rows * Cout * sizeof(float), &scratch) != GPAIR_OK)
        return cudaErrorMemoryAllocation;
    a.partial = static_cast<float*>(scratch);

    CUtensorMap mI, mO;
    const int R = taps == 27 ? 1 : 0;
    (void)R;
    // input and dout: dims (16 channels, x, y, z, 16-channel group), boxes of 16 channels x 8 x 16 x
    // ZS voxels (the input: one group per load; dout: all groups), 32-byte swizzle
    {
        cuuint64_t dims[5] = {16, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)(Cin / 16)};
        cuuint64_t strides[4] = {(cuuint64_t)Cin * 2, (cuuint64_t)W * Cin * 2, (cuuint64_t)H * W * Cin * 2, 32};
        cuuint32_t box[5] = {16, TC_TX, TC_TY, (cuuint32_t)a.ZS, 1};
        cuuint32_t es[5] = {1, 1, 1, 1, 1};
        if (enc(&mI, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<uint16_t*>(in), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
    }
    {
        cuuint64_t dims[5] = {16, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)(Cout / 16)};
        cuuint64_t strides[4] = {(cuuint64_t)Cout * 2, (cuuint64_t)W * Cout * 2, (cuuint64_t)H * W * Cout * 2, 32};
        cuuint32_t box[5] = {16, TC_TX, TC_TY, (cuuint32_t)a.ZS, (cuuint32_t)(Cout / 16)};
        cuuint32_t es[5] = {1, 1, 1, 1, 1};
        if (enc(&mO, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<uint16_t*>(dout), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
    }
    auto kern = taps == 27 ? conv3d_wgrad_tc_kernel<27> : conv3d_wgrad_tc_kernel<1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)(a.n_groups * a.n_splits), WG_THREADS, smem, st>>>(mI, mO, a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t n = (int64_t)rows * Cout;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    wgrad_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(a.partial, a.n_splits, rows, Cout, dw);
    return cudaGetLastError();
}

int conv_tc_status_and_clear() {
    int h = 0, z = 0;
    cudaMemcpyFromSymbol(&h, g_conv_tc_status, sizeof(int));
    cudaMemcpyToSymbol(g_conv_tc_status, &z, sizeof(int));
    return h;
}

}  // namespace gp
