// unet_tc.cu -- the U-Net's 3-D convolution as an implicit GEMM on the 5th-generation tensor
// cores (tcgen05, BF16 operands, FP32 accumulation in tensor memory).
//
// GEMM view: rows are output voxels, columns output channels, the reduction runs over
// (tap, input channel).  CTA = 128 consecutive output voxels (the 128 TMEM lanes of the
// accumulator) x NT output channels (NT columns of TMEM), four warps.  The reduction is cut into
// stages of one tap and Kc input channels; each stage's operand tiles are gathered into shared
// memory (A: the voxels' shifted input rows, zero where the tap falls outside the volume; B: the
// weights' rows) with cp.async, in the canonical K-major layout without swizzle (core matrices of
// 8 rows x 16 bytes; adjacent core matrices along K are 128 bytes apart, along M/N Kc * 16 bytes).
// One thread issues the stage's MMAs (K = 16 each) and commits them to the stage buffer's
// mbarrier; the gathers of the next stages, in a ring of shared buffers, overlap them.  Every wait
// is bounded.
// The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31),
// adds the bias, applies the ReLU and stores BF16.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gpair_internal.cuh"

namespace gp {

constexpr int TC_M = 128;          // voxels per CTA = accumulator lanes
constexpr int TC_THREADS = 128;

__device__ int g_conv_tc_status;   // 1: a bounded wait gave up

__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

// Shared-memory matrix descriptor, no swizzle: start address, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1 at bits 46-47, layout type 0.
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo_bytes, uint32_t sbo_bytes) {
    uint64_t d = (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu);
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

__device__ __forceinline__ uint16_t f2bf_rn(float f) {
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    return *reinterpret_cast<const uint16_t*>(&h);
}

// out[v][co0 + c] = act(bias + sum_{t, ci} in[v + off(t)][ci] w[co0 + c][t][ci]), c < NT.
// TC_STAGES shared buffers: the gathers of up to TC_STAGES - 1 stages are in flight (one cp.async
// group each) while the tensor cores work; a buffer is refilled once the commit of the MMAs that
// read it has arrived on its mbarrier.
constexpr int TC_STAGES = 4;

__global__ void __launch_bounds__(TC_THREADS)
conv3d_fwd_tc_kernel(const uint16_t* __restrict__ in, int D, int H, int W, int Cin, const uint16_t* __restrict__ w,
                     const float* __restrict__ bias, int Cout, int NT, int ncols, int taps, int relu, int Kc,
                     uint16_t* __restrict__ out) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t nv = (int64_t)D * H * W;
    const int64_t v = (int64_t)blockIdx.x * TC_M + tid;     // this thread's voxel row (A) and TMEM lane
    const int co0 = blockIdx.y * NT;
    const int K = taps * Cin;
    const uint32_t aBytes = (uint32_t)TC_M * Kc * 2, bBytes = (uint32_t)NT * Kc * 2;
    const uint32_t stBytes = aBytes + bBytes;               // stage buffer: A tile then B tile
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + TC_STAGES * stBytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + TC_STAGES);
    const uint32_t lbo = 128, sbo = (uint32_t)(Kc / 8) * 128;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int q = 0; q < TC_STAGES; ++q) mbar_init(&mbar[q], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    const bool vok = v < nv;
    const int64_t vv = vok ? v : 0;
    const int vx = (int)(vv % W), vy = (int)((vv / W) % H), vz = (int)(vv / ((int64_t)W * H));
    const int nchunk = Cin / Kc, S = taps * nchunk;
    const uint32_t idesc = tc_idesc(NT, TC_M);
    bool ok = true;

    // gather stage s into its buffer (one cp.async group; empty groups past the last stage keep
    // the group count uniform)
    auto gather = [&](int s) {
        if (s < S) {
            unsigned char* buf = sm + (s % TC_STAGES) * stBytes;
            const int t = s / nchunk, c0 = (s - t * nchunk) * Kc;
            int dz = 0, dy = 0, dx = 0;
            if (taps == 27) { dz = t / 9 - 1; dy = (t / 3) % 3 - 1; dx = t % 3 - 1; }
            const int x = vx + dx, y = vy + dy, z = vz + dz;
            const bool inb = vok && x >= 0 && x < W && y >= 0 && y < H && z >= 0 && z < D;
            const uint16_t* asrc = inb ? in + (((int64_t)z * H + y) * W + x) * Cin + c0 : in;
            unsigned char* arow = buf + (tid >> 3) * sbo + (tid & 7) * 16;
            for (int kc = 0; kc < Kc / 8; ++kc) cp_async16(arow + kc * 128, asrc + kc * 8, inb ? 16u : 0u);
            for (int r = tid; r < NT; r += TC_THREADS) {
                const uint16_t* bsrc = w + (int64_t)(co0 + r) * K + (int64_t)t * Cin + c0;
                unsigned char* brow = buf + aBytes + (r >> 3) * sbo + (r & 7) * 16;
                for (int kc = 0; kc < Kc / 8; ++kc) cp_async16(brow + kc * 128, bsrc + kc * 8, 16u);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int s = 0; s < TC_STAGES - 1; ++s) gather(s);
    for (int s = 0; s < S; ++s) {
        // stage s's group is complete once at most TC_STAGES - 2 newer groups are pending
        asm volatile("cp.async.wait_group %0;" ::"n"(TC_STAGES - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");     // generic writes -> tensor-core reads
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            unsigned char* buf = sm + (s % TC_STAGES) * stBytes;
            for (int ks = 0; ks < Kc / 16; ++ks)
                tc_mma(tmem, smem_desc(buf + ks * 2 * lbo, lbo, sbo), smem_desc(buf + aBytes + ks * 2 * lbo, lbo, sbo),
                       idesc, (s > 0 || ks > 0) ? 1u : 0u);
            tc_commit(&mbar[s % TC_STAGES]);
        }
        // refill the buffer of stage s - 1 with stage s + TC_STAGES - 1 once its MMAs are done
        const int sn = s + TC_STAGES - 1;
        if (sn < S && s >= 1) {
            const int sp = s - 1;
            if (!mbar_wait(&mbar[sp % TC_STAGES], (uint32_t)((sp / TC_STAGES) & 1))) ok = false;
        }
        gather(sn);
    }
    // the last commit covers every MMA issued before it
    if (!mbar_wait(&mbar[(S - 1) % TC_STAGES], (uint32_t)(((S - 1) / TC_STAGES) & 1))) ok = false;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    tc_fence_after();
    if (!ok) atomicMax(&g_conv_tc_status, 1);
    for (int cc = 0; cc < NT; cc += 16) {
        uint32_t r[16];
        tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc, r);
        if (vok) {
            uint32_t pk[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float o0 = __uint_as_float(r[2 * q]), o1 = __uint_as_float(r[2 * q + 1]);
                if (bias) { o0 += bias[co0 + cc + 2 * q]; o1 += bias[co0 + cc + 2 * q + 1]; }
                if (relu) { o0 = fmaxf(o0, 0.f); o1 = fmaxf(o1, 0.f); }
                pk[q] = (uint32_t)f2bf_rn(o0) | ((uint32_t)f2bf_rn(o1) << 16);
            }
            uint4* dst = reinterpret_cast<uint4*>(out + v * Cout + co0 + cc);
            dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// Eligible shapes: Cin and Cout multiples of 16, a channel tile NT = Cout (<= 128) or 128, 16-byte
// aligned tensors.  Returns cudaErrorNotSupported otherwise (the caller uses the mma.sync kernel).
cudaError_t launch_conv3d_fwd_tc(const uint16_t* in, int D, int H, int W, int Cin, const uint16_t* w,
                                 const float* bias, int Cout, int taps, int relu, uint16_t* out, cudaStream_t st) {
    if (Cin % 16 != 0 || Cout % 16 != 0) return cudaErrorNotSupported;
    const int NT = Cout <= 128 ? Cout : (Cout % 128 == 0 ? 128 : 0);
    if (NT == 0) return cudaErrorNotSupported;
    if (((uintptr_t)in | (uintptr_t)w | (uintptr_t)out) & 15) return cudaErrorNotSupported;
    const int Kc = Cin % 32 == 0 ? 32 : 16;
    const int ncols = NT <= 32 ? 32 : (NT <= 64 ? 64 : 128);
    const size_t smem = TC_STAGES * ((size_t)TC_M * Kc * 2 + (size_t)NT * Kc * 2) + 8 * TC_STAGES + 16;
    cudaError_t e = cudaFuncSetAttribute(conv3d_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t nv = (int64_t)D * H * W;
    dim3 grid((unsigned)((nv + TC_M - 1) / TC_M), (unsigned)(Cout / NT));
    conv3d_fwd_tc_kernel<<<grid, TC_THREADS, smem, st>>>(in, D, H, W, Cin, w, bias, Cout, NT, ncols, taps, relu, Kc,
                                                         out);
    return cudaGetLastError();
}

int conv_tc_status_and_clear() {
    int h = 0, z = 0;
    cudaMemcpyFromSymbol(&h, g_conv_tc_status, sizeof(int));
    cudaMemcpyToSymbol(g_conv_tc_status, &z, sizeof(int));
    return h;
}

}  // namespace gp
