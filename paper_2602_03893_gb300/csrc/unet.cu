// unet.cu -- BF16 tensor-core convolutions (FP32 accumulation) and the small elementwise kernels
// of the learned warm start (include/gpair_unet.h).
//
// A 3-D convolution over a channels-last volume is an implicit GEMM: rows are output voxels,
// columns output channels, and the reduction runs over (tap, input channel).  Each warp owns
// 32 output voxels (two 16-row tiles) and 8*NT output channels and issues
// mma.sync.m16n8k16 (bf16 x bf16 -> f32) with fragments gathered straight from the L1/L2-resident
// input and weights; zero padding is applied at fragment load.  The data gradient is the same
// kernel run on flipped, channel-transposed weights; the weight gradient is a GEMM over voxels
// (split-K across CTAs, FP32 atomics into the gradient).  These mma.sync kernels serve the shapes
// the tcgen05 kernels (unet_tc.cu) do not take, and tensor path 0.
#include <cuda_bf16.h>

#include <cstdint>

#include "../../include/gpair_unet.h"

namespace gp {
int device_sms();   // SMs of the current device (step.cu)
gpair_status stream_scratch(cudaStream_t st, size_t bytes, void** buf);   // the stream's scratch pool (gpair_abi.cu)
}

namespace {

typedef uint16_t bf16_t;

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float bf2f(bf16_t v) { return __uint_as_float((uint32_t)v << 16); }

__device__ __forceinline__ bf16_t f2bf(float f) {
    __nv_bfloat16 h = __float2bfloat16_rn(f);
    return *reinterpret_cast<bf16_t*>(&h);
}

__device__ __forceinline__ uint32_t pack2(bf16_t lo, bf16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

__device__ __forceinline__ uint32_t ld32(const bf16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// Tap t of a 3x3x3 stencil -> offsets (dz, dy, dx) in {-1, 0, 1}; a 1-tap stencil is the centre.
__device__ __forceinline__ void tap_offset(int t, int taps, int& dz, int& dy, int& dx) {
    if (taps == 1) { dz = dy = dx = 0; return; }
    dz = t / 9 - 1;
    dy = (t / 3) % 3 - 1;
    dx = t % 3 - 1;
}

constexpr int CONV_THREADS = 128;   // 4 warps
constexpr int CONV_MT = 2;          // 16-voxel tiles per warp

// out[v][co] = act(bias[co] + sum_{t, ci} in[v + off(t)][ci] w[co][t][ci]).  grid.y selects a
// group of 8*NT output channels.
template <int NT>
__global__ void __launch_bounds__(CONV_THREADS)
conv3d_fwd_kernel(const bf16_t* __restrict__ in, int D, int H, int W, int Cin, const bf16_t* __restrict__ w,
                  const float* __restrict__ bias, int Cout, int taps, int relu, bf16_t* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, c = lane & 3;
    const int64_t nv = (int64_t)D * H * W;
    const int64_t vbase = ((int64_t)blockIdx.x * (CONV_THREADS / 32) + warp) * (16 * CONV_MT);
    const int co_base = blockIdx.y * 8 * NT;
    const int K = taps * Cin;

    // the four voxels (rows g, g+8 of each 16-row tile) this lane loads and stores
    int vx[2 * CONV_MT], vy[2 * CONV_MT], vz[2 * CONV_MT];
    bool vok[2 * CONV_MT];
#pragma unroll
    for (int r = 0; r < 2 * CONV_MT; ++r) {
        const int64_t v = vbase + (r >> 1) * 16 + g + (r & 1) * 8;
        vok[r] = v < nv;
        const int64_t vv = vok[r] ? v : 0;
        vx[r] = (int)(vv % W);
        vy[r] = (int)((vv / W) % H);
        vz[r] = (int)(vv / ((int64_t)W * H));
    }
    float acc[CONV_MT][NT][4];
#pragma unroll
    for (int m = 0; m < CONV_MT; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[m][n][0] = acc[m][n][1] = acc[m][n][2] = acc[m][n][3] = 0.f;

    for (int t = 0; t < taps; ++t) {
        int dz, dy, dx;
        tap_offset(t, taps, dz, dy, dx);
        const bf16_t* rowp[2 * CONV_MT];
#pragma unroll
        for (int r = 0; r < 2 * CONV_MT; ++r) {
            const int x = vx[r] + dx, y = vy[r] + dy, z = vz[r] + dz;
            const bool ok = vok[r] && x >= 0 && x < W && y >= 0 && y < H && z >= 0 && z < D;
            rowp[r] = ok ? in + (((int64_t)z * H + y) * W + x) * Cin + 2 * c : nullptr;
        }
        const bf16_t* wt = w + ((int64_t)(co_base + g) * taps + t) * Cin + 2 * c;
        for (int kc = 0; kc < Cin; kc += 16) {
            uint32_t a[CONV_MT][4];
#pragma unroll
            for (int m = 0; m < CONV_MT; ++m) {
                const bf16_t* p0 = rowp[2 * m];
                const bf16_t* p1 = rowp[2 * m + 1];
                a[m][0] = p0 ? ld32(p0 + kc) : 0u;
                a[m][1] = p1 ? ld32(p1 + kc) : 0u;
                a[m][2] = p0 ? ld32(p0 + kc + 8) : 0u;
                a[m][3] = p1 ? ld32(p1 + kc + 8) : 0u;
            }
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const bf16_t* wp = wt + (int64_t)n * 8 * K + kc;
                uint32_t b[2] = {ld32(wp), ld32(wp + 8)};
#pragma unroll
                for (int m = 0; m < CONV_MT; ++m) mma16816(acc[m][n], a[m], b);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < CONV_MT; ++m) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int r = 2 * m + half;
            if (!vok[r]) continue;
            const int64_t v = vbase + m * 16 + g + half * 8;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int co = co_base + n * 8 + 2 * c;
                float o0 = acc[m][n][2 * half], o1 = acc[m][n][2 * half + 1];
                if (bias) { o0 += bias[co]; o1 += bias[co + 1]; }
                if (relu) { o0 = fmaxf(o0, 0.f); o1 = fmaxf(o1, 0.f); }
                *reinterpret_cast<uint32_t*>(out + v * Cout + co) = pack2(f2bf(o0), f2bf(o1));
            }
        }
    }
}

// wt[ci][t][co] = w[co][taps - 1 - t][ci]: the data gradient is a convolution with these.
__global__ void wtrans_kernel(const bf16_t* __restrict__ w, int Cout, int taps, int Cin, bf16_t* __restrict__ wt) {
    const int64_t n = (int64_t)Cout * taps * Cin;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(i % Cin);
        const int t = (int)((i / Cin) % taps);
        const int co = (int)(i / ((int64_t)Cin * taps));
        wt[((int64_t)ci * taps + (taps - 1 - t)) * Cout + co] = w[i];
    }
}

constexpr int WG_CHUNK = 4096;      // voxels per CTA (split-K)

// dw[co][t][ci] += sum_v dout[v][co] in[v + off(t)][ci]; grid = (voxel chunks, taps, Cout / 16).
// A = dout^T (16 output channels x 16 voxels), B = shifted input (16 voxels x 8 input channels).
template <int NTI>
__global__ void __launch_bounds__(128)
conv3d_wgrad_kernel(const bf16_t* __restrict__ in, const bf16_t* __restrict__ dout, int D, int H, int W, int Cin,
                    int Cout, int taps, float* __restrict__ dw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, c = lane & 3;
    const int64_t nv = (int64_t)D * H * W;
    const int t = blockIdx.y;
    const int co0 = blockIdx.z * 16;
    int dz, dy, dx;
    tap_offset(t, taps, dz, dy, dx);
    const int64_t off = ((int64_t)dz * H + dy) * W + dx;
    const int64_t v_begin = (int64_t)blockIdx.x * WG_CHUNK + warp * (WG_CHUNK / 4);
    const int64_t v_end = min(v_begin + WG_CHUNK / 4, nv);
    float acc[NTI][4];
#pragma unroll
    for (int n = 0; n < NTI; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    for (int64_t k0 = v_begin; k0 < v_end; k0 += 16) {
        // the four voxels (k0 + 2c + {0, 1, 8, 9}) this lane touches, and their shifted sources
        int64_t vk[4];
        bool okv[4], oks[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t v = k0 + 2 * c + (q & 1) + (q >> 1) * 8;
            vk[q] = v;
            okv[q] = v < v_end;
            const int64_t vv = okv[q] ? v : 0;
            const int x = (int)(vv % W) + dx, y = (int)((vv / W) % H) + dy, z = (int)(vv / ((int64_t)W * H)) + dz;
            oks[q] = okv[q] && x >= 0 && x < W && y >= 0 && y < H && z >= 0 && z < D;
        }
        uint32_t a[4];
        {
            const int r0 = co0 + g, r1 = co0 + g + 8;
            bf16_t e[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                e[2 * q] = okv[q] ? dout[vk[q] * Cout + r0] : (bf16_t)0;
                e[2 * q + 1] = okv[q] ? dout[vk[q] * Cout + r1] : (bf16_t)0;
            }
            // a0: (row g, cols 2c, 2c+1), a1: (row g+8, ...), a2: cols +8 (row g), a3: cols +8 (row g+8)
            a[0] = pack2(e[0], e[2]);
            a[1] = pack2(e[1], e[3]);
            a[2] = pack2(e[4], e[6]);
            a[3] = pack2(e[5], e[7]);
        }
#pragma unroll
        for (int n = 0; n < NTI; ++n) {
            const int ci = n * 8 + g;
            bf16_t s[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) s[q] = oks[q] ? in[(vk[q] + off) * Cin + ci] : (bf16_t)0;
            uint32_t b[2] = {pack2(s[0], s[1]), pack2(s[2], s[3])};
            mma16816(acc[n], a, b);
        }
    }
#pragma unroll
    for (int n = 0; n < NTI; ++n) {
        const int ci = n * 8 + 2 * c;
        float* d0 = dw + ((int64_t)(co0 + g) * taps + t) * Cin + ci;
        float* d1 = dw + ((int64_t)(co0 + g + 8) * taps + t) * Cin + ci;
        atomicAdd(d0, acc[n][0]);
        atomicAdd(d0 + 1, acc[n][1]);
        atomicAdd(d1, acc[n][2]);
        atomicAdd(d1 + 1, acc[n][3]);
    }
}

// db[co] += sum_v dout[v][co], in two deterministic passes.  Pass 1: block (Cout / 8) x rows
// threads; thread (c, r) sums channels 8c ... 8c + 7 of the voxels r, r + rows, ... of its block's
// range (16-byte loads, consecutive threads on consecutive chunks), then the block sums its rows
// in shared memory in fixed order and writes part[block][Cout].
__global__ void bias_grad_part_kernel(const bf16_t* __restrict__ dout, int64_t nv, int Cout, int64_t per_block,
                                      float* __restrict__ part) {
    extern __shared__ float sred[];                 // [rows][Cout]
    const int nc = Cout / 8, c = threadIdx.x, r = threadIdx.y, rows = blockDim.y;
    const int64_t v0 = blockIdx.x * per_block, v1 = min(nv, v0 + per_block);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t v = v0 + r; v < v1; v += rows) {
        const uint4 q = *reinterpret_cast<const uint4*>(dout + v * Cout + 8 * c);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            acc[2 * i] += __uint_as_float(w[i] << 16);
            acc[2 * i + 1] += __uint_as_float(w[i] & 0xFFFF0000u);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) sred[r * Cout + 8 * c + i] = acc[i];
    __syncthreads();
    for (int q = r * nc + c; q < Cout; q += rows * nc) {
        float s = 0.f;
        for (int k = 0; k < rows; ++k) s += sred[k * Cout + q];
        part[(int64_t)blockIdx.x * Cout + q] = s;
    }
}

// Pass 2: db[co] += sum over blocks of part[block][co]; one warp per channel, lane l sums blocks
// l, l + 32, ... and a fixed shuffle tree adds the lanes (the same order on every run).
__global__ void bias_grad_sum_kernel(const float* __restrict__ part, int nblocks, int Cout, float* __restrict__ db) {
    const int co = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (co >= Cout) return;
    float s = 0.f;
    for (int b = lane; b < nblocks; b += 32) s += part[(int64_t)b * Cout + co];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[co] += s;
}

__global__ void relu_bwd_kernel(const bf16_t* __restrict__ act, bf16_t* __restrict__ g, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(bf2f(act[i]) > 0.f)) g[i] = 0;
}

__global__ void pool2_fwd_kernel(const bf16_t* __restrict__ in, int D, int H, int W, int C, bf16_t* __restrict__ out) {
    const int d = D / 2, h = H / 2, w = W / 2;
    const int64_t n = (int64_t)d * h * w * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(i % C);
        const int64_t v = i / C;
        const int x = (int)(v % w), y = (int)((v / w) % h), z = (int)(v / ((int64_t)w * h));
        float s = 0.f;
        for (int q = 0; q < 8; ++q)
            s += bf2f(in[((((int64_t)(2 * z + (q >> 2)) * H) + 2 * y + ((q >> 1) & 1)) * W + 2 * x + (q & 1)) * C + ch]);
        out[i] = f2bf(0.125f * s);
    }
}

__global__ void pool2_bwd_kernel(const bf16_t* __restrict__ dout, int D, int H, int W, int C, bf16_t* __restrict__ din) {
    const int64_t n = (int64_t)D * H * W * C;
    const int h = H / 2, w = W / 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(i % C);
        const int64_t v = i / C;
        const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((int64_t)W * H));
        din[i] = f2bf(0.125f * bf2f(dout[((((int64_t)(z / 2) * h) + y / 2) * w + x / 2) * C + ch]));
    }
}

__global__ void up2_fwd_kernel(const bf16_t* __restrict__ in, int D, int H, int W, int C, bf16_t* __restrict__ out) {
    const int64_t n = (int64_t)8 * D * H * W * C;
    const int H2 = 2 * H, W2 = 2 * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(i % C);
        const int64_t v = i / C;
        const int x = (int)(v % W2), y = (int)((v / W2) % H2), z = (int)(v / ((int64_t)W2 * H2));
        out[i] = in[((((int64_t)(z / 2) * H) + y / 2) * W + x / 2) * C + ch];
    }
}

__global__ void up2_bwd_kernel(const bf16_t* __restrict__ dout, int D, int H, int W, int C, bf16_t* __restrict__ din) {
    const int64_t n = (int64_t)D * H * W * C;
    const int H2 = 2 * H, W2 = 2 * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(i % C);
        const int64_t v = i / C;
        const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((int64_t)W * H));
        float s = 0.f;
        for (int q = 0; q < 8; ++q)
            s += bf2f(dout[((((int64_t)(2 * z + (q >> 2)) * H2) + 2 * y + ((q >> 1) & 1)) * W2 + 2 * x + (q & 1)) * C + ch]);
        din[i] = f2bf(s);
    }
}

__global__ void concat_fwd_kernel(const bf16_t* __restrict__ a, int Ca, const bf16_t* __restrict__ b, int Cb,
                                  int64_t nv, bf16_t* __restrict__ out) {
    const int C = Ca + Cb;
    const int64_t n = nv * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(i % C);
        const int64_t v = i / C;
        out[i] = ch < Ca ? a[v * Ca + ch] : b[v * Cb + (ch - Ca)];
    }
}

__global__ void concat_bwd_kernel(const bf16_t* __restrict__ dout, int Ca, int Cb, int64_t nv, bf16_t* __restrict__ da,
                                  bf16_t* __restrict__ db) {
    const int C = Ca + Cb;
    const int64_t n = nv * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int ch = (int)(i % C);
        const int64_t v = i / C;
        if (ch < Ca) {
            if (da) da[v * Ca + ch] = dout[i];
        } else if (db) {
            db[v * Cb + (ch - Ca)] = dout[i];
        }
    }
}

__global__ void pack_input_kernel(const float* __restrict__ x, float scale, int64_t nv, int C, bf16_t* __restrict__ out) {
    const int64_t n = nv * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (i % C == 0) ? f2bf(scale * x[i / C]) : (bf16_t)0;
}

__global__ void unpack_output_kernel(const bf16_t* __restrict__ in, int64_t nv, int C, float scale, int relu,
                                     float* __restrict__ x) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        float f = scale * bf2f(in[v * C]);
        x[v] = relu ? fmaxf(f, 0.f) : f;
    }
}

__global__ void mse_kernel(const bf16_t* __restrict__ pred, const float* __restrict__ target, int64_t nv, int C,
                           bf16_t* __restrict__ dpred, double* __restrict__ loss) {
    __shared__ double red[8];
    double s = 0.0;
    const float k = 2.f / (float)nv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv * C; i += (int64_t)gridDim.x * blockDim.x) {
        if (i % C == 0) {
            const float e = bf2f(pred[i]) - target[i / C];
            s += (double)e * e;
            dpred[i] = f2bf(k * e);
        } else {
            dpred[i] = 0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        atomicAdd(loss, t);
    }
}

__global__ void adam_bf16_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                                 float* __restrict__ v, bf16_t* __restrict__ wb, int64_t n, float lr, float b1, float b2,
                                 float eps, float inv_c1, float inv_sqrt_c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi * inv_c1) / (sqrtf(vi) * inv_sqrt_c2 + eps);
        w[i] = wi;
        wb[i] = f2bf(wi);
    }
}

__global__ void add_bf16_kernel(const bf16_t* __restrict__ a, const bf16_t* __restrict__ b, bf16_t* __restrict__ out,
                                int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = f2bf(bf2f(a[i]) + bf2f(b[i]));
}

int blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > (int64_t)gp::device_sms() * 32) b = (int64_t)gp::device_sms() * 32;
    return (int)(b < 1 ? 1 : b);
}

gpair_status st(cudaError_t e) { return e == cudaSuccess ? GPAIR_OK : GPAIR_ERR_CUDA; }

bool dims_ok(int D, int H, int W, int C) { return D > 0 && H > 0 && W > 0 && C > 0; }

// 1: the tcgen05 kernel for every eligible shape, the mma.sync kernel for the others; 2: the
// tcgen05 kernel only (an ineligible shape is GPAIR_ERR_UNSUPPORTED); 0: the mma.sync kernel only.
int g_tensor_path = 1;

}  // namespace

namespace gp {
cudaError_t launch_conv3d_fwd_tc(const uint16_t* in, int D, int H, int W, int Cin, const uint16_t* w,
                                 const float* bias, int Cout, int taps, int relu, uint16_t* out, cudaStream_t st);
cudaError_t launch_conv3d_wgrad_tc(const uint16_t* in, const uint16_t* dout, int D, int H, int W, int Cin, int Cout,
                                   int taps, float* dw, cudaStream_t st);
int conv_tc_status_and_clear();
}  // namespace gp

extern "C" {

int gpair_unet_tensor_path(int mode) {
    if (mode >= 0 && mode <= 2) g_tensor_path = mode;
    return g_tensor_path;
}

int gpair_unet_tc_status(void) { return gp::conv_tc_status_and_clear(); }

gpair_status gpair_conv3d_fwd(const gpair_bf16* in, int D, int H, int W, int Cin, const gpair_bf16* w,
                              const float* bias, int Cout, int taps, int relu, gpair_bf16* out, void* stream) {
    if (!in || !w || !out || !dims_ok(D, H, W, Cin) || Cout <= 0 || (taps != 1 && taps != 27)) return GPAIR_ERR_INVALID_ARG;
    if (Cin % 16 != 0 || Cout % 8 != 0) return GPAIR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (g_tensor_path != 0) {
        const cudaError_t e = gp::launch_conv3d_fwd_tc(reinterpret_cast<const uint16_t*>(in), D, H, W, Cin,
                                                       reinterpret_cast<const uint16_t*>(w), bias, Cout, taps, relu,
                                                       reinterpret_cast<uint16_t*>(out), s);
        if (e != cudaErrorNotSupported) return st(e);
        cudaGetLastError();
        if (g_tensor_path == 2) return GPAIR_ERR_UNSUPPORTED;
        // not eligible: the mma.sync kernel below
    }
    const int64_t nv = (int64_t)D * H * W;
    const unsigned gx = (unsigned)((nv + 16 * CONV_MT * 4 - 1) / (16 * CONV_MT * 4));
    if (Cout % 64 == 0)
        conv3d_fwd_kernel<8><<<dim3(gx, Cout / 64), CONV_THREADS, 0, s>>>(in, D, H, W, Cin, w, bias, Cout, taps, relu, out);
    else if (Cout % 32 == 0)
        conv3d_fwd_kernel<4><<<dim3(gx, Cout / 32), CONV_THREADS, 0, s>>>(in, D, H, W, Cin, w, bias, Cout, taps, relu, out);
    else if (Cout % 16 == 0)
        conv3d_fwd_kernel<2><<<dim3(gx, Cout / 16), CONV_THREADS, 0, s>>>(in, D, H, W, Cin, w, bias, Cout, taps, relu, out);
    else
        conv3d_fwd_kernel<1><<<dim3(gx, Cout / 8), CONV_THREADS, 0, s>>>(in, D, H, W, Cin, w, bias, Cout, taps, relu, out);
    return st(cudaGetLastError());
}

gpair_status gpair_conv3d_dgrad(const gpair_bf16* dout, int D, int H, int W, int Cout, const gpair_bf16* w, int Cin,
                                int taps, gpair_bf16* wt_scratch, gpair_bf16* din, void* stream) {
    if (!dout || !w || !wt_scratch || !din || !dims_ok(D, H, W, Cout) || Cin <= 0 || (taps != 1 && taps != 27))
        return GPAIR_ERR_INVALID_ARG;
    if (Cout % 16 != 0 || Cin % 8 != 0) return GPAIR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    wtrans_kernel<<<blocks_for((int64_t)Cout * taps * Cin), 256, 0, s>>>(w, Cout, taps, Cin, wt_scratch);
    if (cudaGetLastError() != cudaSuccess) return GPAIR_ERR_CUDA;
    return gpair_conv3d_fwd(dout, D, H, W, Cout, wt_scratch, nullptr, Cin, taps, 0, din, stream);
}

gpair_status gpair_conv3d_wgrad(const gpair_bf16* in, const gpair_bf16* dout, int D, int H, int W, int Cin, int Cout,
                                int taps, float* dw, float* db, void* stream) {
    if (!in || !dout || !dw || !dims_ok(D, H, W, Cin) || Cout <= 0 || (taps != 1 && taps != 27)) return GPAIR_ERR_INVALID_ARG;
    if (Cin % 8 != 0 || Cout % 16 != 0 || Cin > 256) return GPAIR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nv = (int64_t)D * H * W;
    bool done = false;
    if (g_tensor_path != 0) {
        const cudaError_t e = gp::launch_conv3d_wgrad_tc(reinterpret_cast<const uint16_t*>(in),
                                                         reinterpret_cast<const uint16_t*>(dout), D, H, W, Cin, Cout,
                                                         taps, dw, s);
        if (e == cudaErrorMemoryAllocation) return GPAIR_ERR_NOMEM;
        if (e != cudaErrorNotSupported && e != cudaSuccess) return GPAIR_ERR_CUDA;
        if (e == cudaErrorNotSupported) {
            cudaGetLastError();
            if (g_tensor_path == 2) return GPAIR_ERR_UNSUPPORTED;
        }
        done = e == cudaSuccess;
    }
    dim3 grid((unsigned)((nv + WG_CHUNK - 1) / WG_CHUNK), taps, Cout / 16);
    if (!done) switch (Cin / 8) {
#define GP_WG(N) case N: conv3d_wgrad_kernel<N><<<grid, 128, 0, s>>>(in, dout, D, H, W, Cin, Cout, taps, dw); break;
        GP_WG(1) GP_WG(2) GP_WG(3) GP_WG(4) GP_WG(6) GP_WG(8) GP_WG(12) GP_WG(16) GP_WG(24) GP_WG(32)
#undef GP_WG
        default: return GPAIR_ERR_UNSUPPORTED;
    }
    if (cudaGetLastError() != cudaSuccess) return GPAIR_ERR_CUDA;
    if (db) {
        if (((uintptr_t)dout & 15) != 0 || Cout % 8 != 0 || Cout > 256) return GPAIR_ERR_UNSUPPORTED;
        const int nc = Cout / 8, rows = 256 / nc;
        int64_t nb = (int64_t)gp::device_sms() * 2;
        const int64_t per_block = (nv + nb - 1) / nb;
        nb = (nv + per_block - 1) / per_block;
        void* part = nullptr;
        if (gp::stream_scratch(s, (size_t)nb * Cout * sizeof(float), &part) != GPAIR_OK) return GPAIR_ERR_NOMEM;
        bias_grad_part_kernel<<<(unsigned)nb, dim3(nc, rows), (size_t)rows * Cout * sizeof(float), s>>>(
            dout, nv, Cout, per_block, static_cast<float*>(part));
        if (cudaGetLastError() != cudaSuccess) return GPAIR_ERR_CUDA;
        bias_grad_sum_kernel<<<(Cout + 7) / 8, 256, 0, s>>>(static_cast<const float*>(part), (int)nb, Cout, db);
    }
    return st(cudaGetLastError());
}

gpair_status gpair_relu_bwd(const gpair_bf16* act, gpair_bf16* g, int64_t n, void* stream) {
    if (!act || !g || n <= 0) return GPAIR_ERR_INVALID_ARG;
    relu_bwd_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(act, g, n);
    return st(cudaGetLastError());
}

gpair_status gpair_pool2_fwd(const gpair_bf16* in, int D, int H, int W, int C, gpair_bf16* out, void* stream) {
    if (!in || !out || !dims_ok(D, H, W, C) || (D | H | W) & 1) return GPAIR_ERR_INVALID_ARG;
    pool2_fwd_kernel<<<blocks_for((int64_t)D * H * W * C / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(in, D, H, W, C, out);
    return st(cudaGetLastError());
}

gpair_status gpair_pool2_bwd(const gpair_bf16* dout, int D, int H, int W, int C, gpair_bf16* din, void* stream) {
    if (!dout || !din || !dims_ok(D, H, W, C) || (D | H | W) & 1) return GPAIR_ERR_INVALID_ARG;
    pool2_bwd_kernel<<<blocks_for((int64_t)D * H * W * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(dout, D, H, W, C, din);
    return st(cudaGetLastError());
}

gpair_status gpair_up2_fwd(const gpair_bf16* in, int D, int H, int W, int C, gpair_bf16* out, void* stream) {
    if (!in || !out || !dims_ok(D, H, W, C)) return GPAIR_ERR_INVALID_ARG;
    up2_fwd_kernel<<<blocks_for((int64_t)8 * D * H * W * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(in, D, H, W, C, out);
    return st(cudaGetLastError());
}

gpair_status gpair_up2_bwd(const gpair_bf16* dout, int D, int H, int W, int C, gpair_bf16* din, void* stream) {
    if (!dout || !din || !dims_ok(D, H, W, C)) return GPAIR_ERR_INVALID_ARG;
    up2_bwd_kernel<<<blocks_for((int64_t)D * H * W * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(dout, D, H, W, C, din);
    return st(cudaGetLastError());
}

gpair_status gpair_concat_fwd(const gpair_bf16* a, int Ca, const gpair_bf16* b, int Cb, int64_t nv, gpair_bf16* out,
                              void* stream) {
    if (!a || !b || !out || Ca <= 0 || Cb <= 0 || nv <= 0) return GPAIR_ERR_INVALID_ARG;
    concat_fwd_kernel<<<blocks_for(nv * (Ca + Cb)), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, Ca, b, Cb, nv, out);
    return st(cudaGetLastError());
}

gpair_status gpair_concat_bwd(const gpair_bf16* dout, int Ca, int Cb, int64_t nv, gpair_bf16* da, gpair_bf16* db,
                              void* stream) {
    if (!dout || Ca <= 0 || Cb <= 0 || nv <= 0) return GPAIR_ERR_INVALID_ARG;
    concat_bwd_kernel<<<blocks_for(nv * (Ca + Cb)), 256, 0, static_cast<cudaStream_t>(stream)>>>(dout, Ca, Cb, nv, da, db);
    return st(cudaGetLastError());
}

gpair_status gpair_add_bf16(const gpair_bf16* a, const gpair_bf16* b, gpair_bf16* out, int64_t n, void* stream) {
    if (!a || !b || !out || n <= 0) return GPAIR_ERR_INVALID_ARG;
    add_bf16_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, b, out, n);
    return st(cudaGetLastError());
}

gpair_status gpair_pack_input(const float* x, float scale, int64_t nv, int C, gpair_bf16* out, void* stream) {
    if (!x || !out || nv <= 0 || C <= 0) return GPAIR_ERR_INVALID_ARG;
    pack_input_kernel<<<blocks_for(nv * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, scale, nv, C, out);
    return st(cudaGetLastError());
}

gpair_status gpair_unpack_output(const gpair_bf16* in, int64_t nv, int C, float scale, int relu, float* x, void* stream) {
    if (!in || !x || nv <= 0 || C <= 0) return GPAIR_ERR_INVALID_ARG;
    unpack_output_kernel<<<blocks_for(nv), 256, 0, static_cast<cudaStream_t>(stream)>>>(in, nv, C, scale, relu, x);
    return st(cudaGetLastError());
}

gpair_status gpair_mse_loss(const gpair_bf16* pred, const float* target, int64_t nv, int C, gpair_bf16* dpred,
                            double* loss_out, void* stream) {
    if (!pred || !target || !dpred || !loss_out || nv <= 0 || C <= 0) return GPAIR_ERR_INVALID_ARG;
    mse_kernel<<<blocks_for(nv * C), 256, 0, static_cast<cudaStream_t>(stream)>>>(pred, target, nv, C, dpred, loss_out);
    return st(cudaGetLastError());
}

gpair_status gpair_adam_bf16(float* w, const float* g, float* m, float* v, gpair_bf16* wb, int64_t n, float lr,
                             float b1, float b2, float eps, int t, void* stream) {
    if (!w || !g || !m || !v || !wb || n <= 0 || t < 1) return GPAIR_ERR_INVALID_ARG;
    const double c1 = 1.0 - pow((double)b1, t), c2 = 1.0 - pow((double)b2, t);
    adam_bf16_kernel<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        w, g, m, v, wb, n, lr, b1, b2, eps, (float)(1.0 / c1), (float)(1.0 / sqrt(c2)));
    return st(cudaGetLastError());
}

}  // extern "C"
