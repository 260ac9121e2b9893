// spatial_order.cu -- a spatially compact order of free-centre Gaussians for the forward: the
// Morton order of their centres in the set's bounding box, so that the 256 consecutive Gaussians
// of a tile lie close together and the sensor-lane kernel's sample bands stay short.  The
// forward is a sum over Gaussians, so the order changes its result only by FP32 summation order.
//
// The order is a stable LSD radix sort of 18-bit Morton keys (64 cells per axis, finer than a
// tile of 256 Gaussians needs) in two passes of 9 bits: per-block histograms, one exclusive scan
// in (digit, block) order, and a scatter whose ranks inside a block follow the index order
// through warp-level match masks.  Deterministic: equal keys keep their index order.  Then one
// gather writes the permuted centres, widths and amplitudes.
#include <cfloat>

#include "gpair_internal.cuh"

namespace gp {

constexpr int SO_THREADS = 256;
constexpr int SO_CHUNK = SO_THREADS * 16;   // keys per block of a radix pass
constexpr int SO_BB_BLOCKS = 256;           // blocks of the bounding-box reduction
constexpr int SO_AXIS_BITS = 6;             // Morton key: 6 bits per axis
constexpr int SO_DIGIT = 9, SO_RADIX = 1 << SO_DIGIT, SO_PASSES = 3 * SO_AXIS_BITS / SO_DIGIT;

__host__ __device__ __forceinline__ int so_blocks(int64_t M) { return (int)((M + SO_CHUNK - 1) / SO_CHUNK); }
inline size_t align256_sz(size_t x) { return (x + 255) & ~(size_t)255; }

// scratch: keys[2][M], vals[2][M], histogram [radix][blocks], box partials, permuted arrays [5][M]
size_t spatial_order_bytes(int64_t M) {
    const size_t a = align256_sz((size_t)M * 4);
    return 4 * a + align256_sz((size_t)SO_RADIX * so_blocks(M) * 4) + align256_sz((size_t)(SO_BB_BLOCKS + 1) * 6 * 4) +
           5 * a;
}

// Per-block minima and maxima of the centres (grid-stride), then their reduction by one block.
__global__ void so_box_partial_kernel(GaussDev g, float* __restrict__ part) {
    __shared__ float red[6][SO_THREADS];
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.M; i += (int64_t)gridDim.x * blockDim.x) {
        const float c[3] = {g.cx[i], g.cy[i], g.cz[i]};
#pragma unroll
        for (int q = 0; q < 3; ++q) { mn[q] = fminf(mn[q], c[q]); mx[q] = fmaxf(mx[q], c[q]); }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) { red[q][threadIdx.x] = mn[q]; red[3 + q][threadIdx.x] = mx[q]; }
    __syncthreads();
    for (int s = SO_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                red[q][threadIdx.x] = fminf(red[q][threadIdx.x], red[q][threadIdx.x + s]);
                red[3 + q][threadIdx.x] = fmaxf(red[3 + q][threadIdx.x], red[3 + q][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = red[threadIdx.x][0];
}

// One block of SO_BB_BLOCKS threads: thread b takes block b's partials, then a tree.
__global__ void so_box_final_kernel(const float* __restrict__ part, float* __restrict__ box) {
    __shared__ float red[6][SO_BB_BLOCKS];
#pragma unroll
    for (int q = 0; q < 6; ++q) red[q][threadIdx.x] = part[threadIdx.x * 6 + q];
    __syncthreads();
    for (int s = SO_BB_BLOCKS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                red[q][threadIdx.x] = fminf(red[q][threadIdx.x], red[q][threadIdx.x + s]);
                red[3 + q][threadIdx.x] = fmaxf(red[3 + q][threadIdx.x], red[3 + q][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) box[threadIdx.x] = red[threadIdx.x][0];
}

// the axis bits spread three apart (bit b to bit 3b), for interleaving x, y, z from the lowest bit
__device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
    uint32_t r = 0;
#pragma unroll
    for (int b = 0; b < SO_AXIS_BITS; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

__global__ void so_keys_kernel(GaussDev g, const float* __restrict__ box, uint32_t* __restrict__ keys,
                               int* __restrict__ vals) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.M) return;
    const float c[3] = {g.cx[i], g.cy[i], g.cz[i]};
    uint32_t k = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float lo = box[q], ext = box[3 + q] - lo;
        const float t = ext > 0.f ? (c[q] - lo) / ext : 0.f;
        const float top = (float)((1 << SO_AXIS_BITS) - 1);
        const uint32_t u = (uint32_t)fminf(fmaxf(t * top, 0.f), top);
        k |= spread_bits(u) << q;
    }
    keys[i] = k;
    vals[i] = (int)i;
}

// Radix pass, step 1: the block's digit counts, stored digit-major: hist[d * nblocks + block].
__global__ void so_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift, int* __restrict__ hist) {
    __shared__ int h[SO_RADIX];
    for (int d = threadIdx.x; d < SO_RADIX; d += SO_THREADS) h[d] = 0;
    __syncthreads();
    const int64_t b0 = (int64_t)blockIdx.x * SO_CHUNK;
    for (int q = threadIdx.x; q < SO_CHUNK; q += SO_THREADS) {
        const int64_t i = b0 + q;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (SO_RADIX - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < SO_RADIX; d += SO_THREADS) hist[(int64_t)d * gridDim.x + blockIdx.x] = h[d];
}

// Step 2: exclusive scan of the counts in (digit, block) order, i.e. of hist as one flat array.
// One block walks the array in tiles of SO_SCAN_THREADS x SO_SCAN_ITEMS entries: each thread loads
// its SO_SCAN_ITEMS consecutive entries (all loads of a tile in flight together), the block scans
// the thread sums with warp shuffles, and each thread writes its entries' running offsets; a
// carry takes the tile's total to the next tile.
constexpr int SO_SCAN_THREADS = 1024;
constexpr int SO_SCAN_ITEMS = 8;
__global__ void __launch_bounds__(SO_SCAN_THREADS) so_scan_kernel(int* __restrict__ hist, int nb) {
    __shared__ int wsum[SO_SCAN_THREADS / 32];
    __shared__ int carry_s;
    const int64_t N = (int64_t)SO_RADIX * nb;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    constexpr int64_t TILE_N = (int64_t)SO_SCAN_THREADS * SO_SCAN_ITEMS;
    int carry = 0;
    for (int64_t base = 0; base < N; base += TILE_N) {
        const int64_t a = base + (int64_t)t * SO_SCAN_ITEMS;
        int v[SO_SCAN_ITEMS];
        int s = 0;
#pragma unroll
        for (int k = 0; k < SO_SCAN_ITEMS; ++k) {
            v[k] = a + k < N ? hist[a + k] : 0;
            s += v[k];
        }
        int x = s;                                   // inclusive scan over the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {                                // inclusive scan of the warp totals
            int y = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += u;
            }
            wsum[lane] = y;
            if (lane == 31) carry_s = y;             // the tile's total
        }
        __syncthreads();
        int run = carry + x - s + (w ? wsum[w - 1] : 0);
#pragma unroll
        for (int k = 0; k < SO_SCAN_ITEMS; ++k) {
            if (a + k < N) hist[a + k] = run;
            run += v[k];
        }
        carry += carry_s;
        __syncthreads();                             // wsum and carry_s are reused by the next tile
    }
}

// Step 3: stable scatter.  The block takes its keys 256 at a time in index order; inside a warp
// the lanes of equal digit find each other with a match mask (rank = lower lanes of the same
// digit), the warps' counts per digit give each warp its start, and a running count per digit
// carries the offsets from one round to the next.
__global__ void so_scatter_kernel(const uint32_t* __restrict__ kin, const int* __restrict__ vin, int64_t n, int shift,
                                  const int* __restrict__ hist, uint32_t* __restrict__ kout, int* __restrict__ vout) {
    __shared__ int base[SO_RADIX], run[SO_RADIX];
    __shared__ int wcnt[SO_THREADS / 32][SO_RADIX];
    const int t = threadIdx.x, warp = t >> 5;
    for (int d = t; d < SO_RADIX; d += SO_THREADS) {
        base[d] = hist[(int64_t)d * gridDim.x + blockIdx.x];
        run[d] = 0;
        for (int w = 0; w < SO_THREADS / 32; ++w) wcnt[w][d] = 0;
    }
    __syncthreads();
    uint32_t lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const int64_t b0 = (int64_t)blockIdx.x * SO_CHUNK;
    for (int r = 0; r < SO_CHUNK / SO_THREADS; ++r) {
        const int64_t i = b0 + r * SO_THREADS + t;
        const bool ok = i < n;
        const uint32_t key = ok ? kin[i] : 0u;
        const int val = ok ? vin[i] : 0;
        const int d = ok ? (int)((key >> shift) & (SO_RADIX - 1)) : SO_RADIX;     // SO_RADIX: no key
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (ok && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        for (int dd = t; dd < SO_RADIX; dd += SO_THREADS) {   // each warp's start inside the block, then the running count
            int acc = run[dd];
            for (int w = 0; w < SO_THREADS / 32; ++w) {
                const int c = wcnt[w][dd];
                wcnt[w][dd] = acc;
                acc += c;
            }
            run[dd] = acc;
        }
        __syncthreads();
        if (ok) {
            const int pos = base[d] + wcnt[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        for (int dd = t; dd < SO_RADIX; dd += SO_THREADS)
            for (int w = 0; w < SO_THREADS / 32; ++w) wcnt[w][dd] = 0;
        __syncthreads();
    }
}

__global__ void so_gather_kernel(GaussDev g, const int* __restrict__ perm, float* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.M) return;
    const int64_t j = perm[i];
    const int64_t M = g.M;
    out[i] = g.cx[j];
    out[M + i] = g.cy[j];
    out[2 * M + i] = g.cz[j];
    out[3 * M + i] = g.sg[j];
    out[4 * M + i] = g.A[j];
}

// gp: g with its arrays replaced by the permuted copies in scratch (spatial_order_bytes(g.M)).
cudaError_t launch_spatial_order(const GaussDev& g, void* scratch, GaussDev& gp, cudaStream_t st) {
    const int64_t M = g.M;
    if (M > 0x7FFFFFFF) return cudaErrorNotSupported;
    const size_t a = align256_sz((size_t)M * 4);
    char* p = static_cast<char*>(scratch);
    uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(p), reinterpret_cast<uint32_t*>(p + a)};
    int* vals[2] = {reinterpret_cast<int*>(p + 2 * a), reinterpret_cast<int*>(p + 3 * a)};
    const int nb = so_blocks(M);
    int* hist = reinterpret_cast<int*>(p + 4 * a);
    float* boxp = reinterpret_cast<float*>(p + 4 * a + align256_sz((size_t)SO_RADIX * nb * 4));
    float* box = boxp + SO_BB_BLOCKS * 6;
    float* out = reinterpret_cast<float*>(p + 4 * a + align256_sz((size_t)SO_RADIX * nb * 4) +
                                          align256_sz((size_t)(SO_BB_BLOCKS + 1) * 6 * 4));
    so_box_partial_kernel<<<SO_BB_BLOCKS, SO_THREADS, 0, st>>>(g, boxp);
    so_box_final_kernel<<<1, SO_BB_BLOCKS, 0, st>>>(boxp, box);
    const unsigned eb = (unsigned)((M + 255) / 256);
    so_keys_kernel<<<eb, 256, 0, st>>>(g, box, keys[0], vals[0]);
    for (int pass = 0; pass < SO_PASSES; ++pass) {
        const int in = pass & 1;
        so_hist_kernel<<<nb, SO_THREADS, 0, st>>>(keys[in], M, SO_DIGIT * pass, hist);
        so_scan_kernel<<<1, SO_SCAN_THREADS, 0, st>>>(hist, nb);
        so_scatter_kernel<<<nb, SO_THREADS, 0, st>>>(keys[in], vals[in], M, SO_DIGIT * pass, hist, keys[in ^ 1],
                                                     vals[in ^ 1]);
    }
    static_assert(SO_PASSES % 2 == 0, "the order ends in buffer 0");
    so_gather_kernel<<<eb, 256, 0, st>>>(g, vals[0], out);
    gp = g;
    gp.cx = out;
    gp.cy = out + M;
    gp.cz = out + 2 * M;
    gp.sg = out + 3 * M;
    gp.A = out + 4 * M;
    return cudaGetLastError();
}

}  // namespace gp
