// gpair_abi.cu -- the C ABI declared in include/gpair.h: argument validation, the per-stream
// scratch pool, TMA descriptor set-up, launch configuration and the reconstruction solver.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "gpair_internal.cuh"
#include "step_sched.cuh"

namespace gp {
cudaError_t launch_tile_info(const GaussDev& g, TileInfo* ti, cudaStream_t st);
cudaError_t launch_slab_info_grid(const GaussDev& g, int sbx, int sby, int sbz, int S, SlabInfo* si, cudaStream_t st);
cudaError_t launch_slab_info_soa(const GaussDev& g, int64_t ntiles, int64_t tiles_per_slab, int S, SlabInfo* si,
                                 cudaStream_t st);
cudaError_t launch_forward(const GaussDev& g, const ArrDev& a, const TileInfo* ti, const SlabInfo* si, int S,
                           float* partial, int2* rows, int PL, int LB, int TB, bool binned, int* status,
                           const CUtensorMap* tmap, const MomentTable* mom, cudaStream_t st);
cudaError_t launch_slab_reduce(const GaussDev& g, const ArrDev& a, const float* partial, const int2* rows, int S,
                               int PL, float* y, cudaStream_t st);
size_t fwd_free_smem(int NW, int LB);
cudaError_t launch_slab_order(SlabInfo* si, int S, cudaStream_t st);
size_t spatial_order_bytes(int64_t M);
cudaError_t launch_spatial_order(const GaussDev& g, void* scratch, GaussDev& gp, cudaStream_t st);
cudaError_t launch_forward_free(const GaussDev& g, const ArrDev& a, const TileInfo* ti, const SlabInfo* si, int S,
                                float* partial, int2* rows, int PL, int LB, int NW, cudaStream_t st);
cudaError_t launch_slab_reduce_rows(const ArrDev& a, const float* partial, const int2* rows, int S, int PL, float* y,
                                    cudaStream_t st);
size_t fwd_lanes_smem(int NW, int NZ, int LB, int P, int L);
int fwd_lanes_nz(float h, float invDelta);
cudaError_t launch_slab_info_cubes(const GaussDev& g, int scx, int scy, int scz, int S, SlabInfo* si, cudaStream_t st);
cudaError_t launch_forward_lanes(const GaussDev& g, const ArrDev& a, const SlabInfo* si, int S, float* partial,
                                 int2* rows, int LB, int NZ, int NW, int* status, const CUtensorMap* tmap,
                                 const MomentTable& T, cudaStream_t st);
int adj_band_len(float rad, float smax, float k, float invDelta);
cudaError_t launch_adjoint(const GaussDev& g, const ArrDev& a, const TileInfo* ti, const float* delta, float* gA,
                           float* gc, float* gs, int LBA, cudaStream_t st);
size_t adj_moment_q_bytes(const ArrDev& a, int L);
cudaError_t launch_adjoint_moment(const GaussDev& g, const ArrDev& a, const float* delta, float* gA,
                                  const MomentTable& T, float* Q, const cudaEvent_t* ev, cudaStream_t st);
cudaError_t launch_npc(const float* z, float* x, int64_t M, int npc, float eps, cudaStream_t st);
cudaError_t launch_wait_selftest(uint32_t polls, int* status, cudaStream_t st);
cudaError_t launch_zmap(const float* vol, int nx, int ny, int nz, float* out, cudaStream_t st);
size_t ssim_scratch_bytes(int64_t M);
cudaError_t launch_ssim_sum(const float* x, const float* y, int nx, int ny, int nz, int win, float range, void* scratch,
                            double* out, cudaStream_t st);
cudaError_t launch_metrics_march(const float* x, const float* y, int nx, int ny, int nz, int win, float range,
                                 double* partial, double* res, cudaStream_t st);
size_t ssim_march_partial_doubles();
int metrics_march_pmax();
cudaError_t launch_vcr(const float* x, int nx, int ny, int nz, float beta, float eps, float lam, double* partial,
                       double* value_out, float* g, cudaStream_t st);
cudaError_t launch_assa_forward(const GaussDev& g, const ArrDev& a, const SlabInfo* si, int S, float* partial,
                                int2* rows, int LB, int* status, const CUtensorMap* tmap, const AssaTable& T,
                                unsigned* amax, const cudaEvent_t* ev, cudaStream_t st);
size_t assa_dconv_bytes(const ArrDev& a, const AssaTable& T);
cudaError_t launch_assa_adjoint(const GaussDev& g, const ArrDev& a, const float* delta, float* gA, const AssaTable& T,
                                float* dconv, const cudaEvent_t* ev, cudaStream_t st);
cudaError_t launch_resid(const float* y, const float* b, float* delta, float scale, int64_t n, double* partial,
                         double* out, cudaStream_t st);
cudaError_t launch_reduce2(const float* a, const float* b, const float* c, int64_t n, double* partial, double* out,
                           cudaStream_t st);
cudaError_t launch_ls(const float* r, const float* Fg, int64_t n, float* x, const float* g, int64_t M,
                      double* partial, double* nd, cudaStream_t st);
cudaError_t launch_adam(float* z, float* m, float* v, const float* gx, int64_t M, int npc, float eps, float b1,
                        float b2, float adam_eps, const StepSched* sd, cudaStream_t st);
cudaError_t launch_schedule(const SchedParams& p, StepSched* sd, cudaStream_t st);
cudaError_t launch_set_step(StepSched* sd, int t, const SchedParams& p, cudaStream_t st);
int red_blocks();
bool vox_is_lattice(const GaussDev& g, const gpair_grid& og);
cudaError_t launch_voxelize(const GaussDev& g, const gpair_grid& og, float k, float* vol, float* tmp, cudaStream_t st);
}  // namespace gp

using namespace gp;

namespace {

constexpr int SPC = 8;            // sensors per forward CTA (matches the kernel)

// ---- per-(device, stream) scratch pool -------------------------------------------------

struct Scratch {
    void* buf = nullptr;
    size_t cap = 0;
    int* status = nullptr;        // device status word
};

std::mutex g_pool_mu;
std::unordered_map<uint64_t, Scratch> g_pool;

uint64_t pool_key(int dev, cudaStream_t st) { return ((uint64_t)(uint32_t)dev << 48) ^ (uint64_t)(uintptr_t)st; }

gpair_status get_scratch(cudaStream_t st, size_t bytes, void** out_buf, int** out_status) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GPAIR_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    Scratch& s = g_pool[pool_key(dev, st)];
    if (!s.status) {
        if (cudaMalloc(&s.status, sizeof(int)) != cudaSuccess) { s.status = nullptr; return GPAIR_ERR_NOMEM; }
        if (cudaMemsetAsync(s.status, 0, sizeof(int), st) != cudaSuccess) return GPAIR_ERR_CUDA;
    }
    if (s.cap < bytes) {
        if (s.buf) {
            cudaStreamSynchronize(st);
            cudaFree(s.buf);
            s.buf = nullptr;
            s.cap = 0;
        }
        size_t want = bytes + bytes / 8 + 4096;
        if (cudaMalloc(&s.buf, want) != cudaSuccess) { s.buf = nullptr; cudaGetLastError(); return GPAIR_ERR_NOMEM; }
        s.cap = want;
    }
    if (out_buf) *out_buf = s.buf;
    if (out_status) *out_status = s.status;
    return GPAIR_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---- argument conversion ------------------------------------------------------------------

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

gpair_status make_gauss(const gpair_gaussians* gi, GaussDev& g) {
    if (!gi || gi->M <= 0 || !gi->A) return GPAIR_ERR_INVALID_ARG;
    memset(&g, 0, sizeof(g));
    g.M = gi->M;
    g.A = gi->A;
    if (!gi->cx) {
        const gpair_grid* gr = gi->grid;
        if (!gr || gr->nx <= 0 || gr->ny <= 0 || gr->nz <= 0) return GPAIR_ERR_INVALID_ARG;
        if ((int64_t)gr->nx * gr->ny * gr->nz != gi->M) return GPAIR_ERR_INVALID_ARG;
        if (!finite_pos(gr->dx) || !finite_pos(gr->sigma)) return GPAIR_ERR_INVALID_ARG;
        if (!std::isfinite(gr->ox) || !std::isfinite(gr->oy) || !std::isfinite(gr->oz)) return GPAIR_ERR_INVALID_ARG;
        g.grid = 1;
        g.nx = gr->nx; g.ny = gr->ny; g.nz = gr->nz;
        g.h = gr->dx; g.sigma = gr->sigma;
        g.ox = gr->ox; g.oy = gr->oy; g.oz = gr->oz;
        g.ntx = (gr->nx + BX - 1) / BX; g.nty = (gr->ny + BY - 1) / BY; g.ntz = (gr->nz + BZ - 1) / BZ;
        g.ntiles = (int64_t)g.ntx * g.nty * g.ntz;
    } else {
        if (!gi->cy || !gi->cz || !gi->sigma) return GPAIR_ERR_INVALID_ARG;
        g.grid = 0;
        g.cx = gi->cx; g.cy = gi->cy; g.cz = gi->cz; g.sg = gi->sigma;
        g.ntiles = (gi->M + TILE - 1) / TILE;
    }
    if (g.ntiles > (int64_t)INT32_MAX) return GPAIR_ERR_UNSUPPORTED;
    return GPAIR_OK;
}

gpair_status make_arr(const gpair_array* ai, ArrDev& a) {
    if (!ai || ai->n_sensors <= 0 || !ai->xyz || ai->n_samples <= 0) return GPAIR_ERR_INVALID_ARG;
    if (ai->n_samples > (1 << 27) || ai->n_sensors > 65535) return GPAIR_ERR_UNSUPPORTED;
    if (!finite_pos(ai->sound_speed) || !finite_pos(ai->fs) || !finite_pos(ai->window_k)) return GPAIR_ERR_INVALID_ARG;
    if (!std::isfinite(ai->t0)) return GPAIR_ERR_INVALID_ARG;
    a.Nd = ai->n_sensors;
    a.xyz = ai->xyz;
    a.v = ai->sound_speed;
    a.fs = ai->fs;
    a.t0 = ai->t0;
    a.Nt = ai->n_samples;
    a.k = ai->window_k;
    a.Delta = (float)((double)ai->sound_speed / (double)ai->fs);
    a.invDelta = (float)((double)ai->fs / (double)ai->sound_speed);
    a.fs_v = (double)ai->fs / (double)ai->sound_speed;
    a.t0fs = (double)ai->t0 * (double)ai->fs;
    a.vt0 = (double)ai->sound_speed * (double)ai->t0;
    a.dlt = (double)ai->sound_speed / (double)ai->fs;
    return GPAIR_OK;
}

// ---- TMA descriptor for the grid amplitude volume ------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3-D map over A[nz][ny][nx] float32 with a bx x by x bz box (default: one 8 x 8 x 4 brick);
// out-of-range elements read as 0.
bool make_tmap(const GaussDev& g, CUtensorMap* map, int bx = BX, int by = BY, int bz = BZ) {
    if (((uintptr_t)g.A & 15) != 0 || (g.nx % 4) != 0) return false;
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    cuuint64_t strides[2] = {(cuuint64_t)g.nx * 4, (cuuint64_t)g.nx * g.ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(g.A), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

gpair_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GPAIR_OK;
    if (e == cudaErrorMemoryAllocation) return GPAIR_ERR_NOMEM;
    if (e == cudaErrorInvalidValue) return GPAIR_ERR_UNSUPPORTED;
    return GPAIR_ERR_CUDA;
}

// ---- forward plan ---------------------------------------------------------------------------

struct FwdPlan {
    int S;                 // slabs
    int64_t tiles_per_slab;        // SoA mode
    int sbx, sby, sbz;     // grid mode: slab block size in bricks
    int LB;                // slab band entries per sensor (FP64 in shared memory)
    int TB;                // tile band entries per sensor (float, atomics)
    int PL;                // partial row length
    bool binned;           // grid mode: per-(tile, sensor) binned kernel
    bool lanes;            // grid mode: the sensor-lane moment kernel (slabs of 8^3-node cubes)
    bool free_lanes;       // SoA mode: the sensor-lane direct kernel (slabs of tile ranges)
    int NW, NZ;            // warps per CTA of the lanes kernels; moment-band bins (grid)
    size_t off_ti, off_si, off_rows, off_part, bytes;
    size_t off_sort;       // free-centre lanes plan: the spatial order's scratch (after the rest)
};

void plan_offsets(FwdPlan& p, const GaussDev& g, const ArrDev& a) {
    p.off_ti = 0;
    p.off_si = align256(sizeof(TileInfo) * (size_t)g.ntiles);
    p.off_rows = p.off_si + align256(sizeof(SlabInfo) * (size_t)p.S);
    p.off_part = p.off_rows + align256(sizeof(int2) * (size_t)p.S * a.Nd);
    p.bytes = p.off_part + align256((size_t)p.S * a.Nd * p.PL * 4);
}

// Grid mode: slabs are blocks of sb[0] x sb[1] x sb[2] bricks; the band of a block is bounded by
// its diagonal plus the window, the band of one brick by its radius plus the window.
void grid_plan_from_blocks(FwdPlan& p, const GaussDev& g, const ArrDev& a, const int sb[3]) {
    const int nt[3] = {g.ntx, g.nty, g.ntz};
    const double ext[3] = {BX * (double)g.h, BY * (double)g.h, BZ * (double)g.h};
    p.sbx = sb[0]; p.sby = sb[1]; p.sbz = sb[2];
    int64_t s = 1;
    for (int q = 0; q < 3; ++q) s *= (nt[q] + sb[q] - 1) / sb[q];
    p.S = (int)s;
    // span of the block's lattice centres (B sb - 1 spacings per axis)
    const double dx = sb[0] * ext[0] - g.h, dy = sb[1] * ext[1] - g.h, dz = sb[2] * ext[2] - g.h;
    const double diag = std::sqrt(dx * dx + dy * dy + dz * dz);
    // n_lo, n_hi of a (slab, sensor) are floor/ceil of the band edges -/+ 2 samples; with the inclusive
    // end and the 4-alignment of the band start the band spans at most (diag + 2 k sigma) / Delta + 10.
    p.LB = ((int)std::ceil((diag + 2.0 * a.k * g.sigma) * a.invDelta) + 10 + 3) & ~3;
    p.PL = p.LB;
    const double reach = brick_radius(g.h) + a.k * g.sigma;
    p.TB = ((int)std::ceil(2.0 * reach * a.invDelta) + 8 + 31) & ~31;
    // binned kernel: every tile band must fit in TB bins and windows in 4 chunks of 32 lanes
    const int Lmain = (int)std::floor(2.0 * a.k * g.sigma * a.invDelta) + 1;
    p.binned = p.TB <= 512 && Lmain <= 128;
    if (p.TB > 512) p.TB = 512;
    plan_offsets(p, g, a);
}

// SoA mode: S slabs of consecutive tiles, full-record partial rows.
void soa_plan_from_slabs(FwdPlan& p, const GaussDev& g, const ArrDev& a, int64_t S) {
    p.tiles_per_slab = (g.ntiles + S - 1) / S;
    p.S = (int)((g.ntiles + p.tiles_per_slab - 1) / p.tiles_per_slab);
    p.LB = std::min(512, ((a.Nt + 4) + 3) & ~3);
    p.PL = a.Nt;
    p.TB = 256;
    p.binned = false;
    plan_offsets(p, g, a);
}

FwdPlan plan_forward(const GaussDev& g, const ArrDev& a) {
    FwdPlan p;
    memset(&p, 0, sizeof(p));
    const int ngroups = (a.Nd + SPC - 1) / SPC;
    const int64_t target_S = ((int64_t)device_sms() * 4 * 4 + ngroups - 1) / ngroups;
    if (g.grid) {
        // Compact blocks of bricks: start from 4 x 4 x 8 bricks (a cube of 32 nodes a side) and
        // halve the longest side until there are enough CTAs; the band of a block is bounded by its
        // diagonal, and a short band keeps each warp's slab accumulators small.
        int sb[3] = {std::min(4, g.ntx), std::min(4, g.nty), std::min(8, g.ntz)};
        const int nt[3] = {g.ntx, g.nty, g.ntz};
        const double ext[3] = {BX * (double)g.h, BY * (double)g.h, BZ * (double)g.h};
        auto count = [&] {
            int64_t s = 1;
            for (int q = 0; q < 3; ++q) s *= (nt[q] + sb[q] - 1) / sb[q];
            return s;
        };
        while (count() < target_S) {
            int best = -1;
            double len = 0;
            for (int q = 0; q < 3; ++q)
                if (sb[q] > 1 && sb[q] * ext[q] > len) { len = sb[q] * ext[q]; best = q; }
            if (best < 0) break;
            sb[best] = (sb[best] + 1) / 2;
        }
        grid_plan_from_blocks(p, g, a, sb);
    } else {
        int64_t S = target_S;
        if (S > g.ntiles) S = g.ntiles;
        const int64_t row = (int64_t)a.Nd * a.Nt * 4;
        while (S > 1 && S * row > ((int64_t)2 << 30)) S = (S + 1) / 2;
        if (S < 1) S = 1;
        soa_plan_from_slabs(p, g, a, S);
    }
    return p;
}

// Plan for a fixed scratch capacity (used by the allocation-free entry point): the default plan,
// coarsened -- larger slab blocks, or fewer slabs -- until its scratch fits in `cap` bytes.
// Returns false when even the coarsest plan does not fit.
bool plan_forward_capped(const GaussDev& g, const ArrDev& a, size_t cap, FwdPlan& out) {
    FwdPlan p = plan_forward(g, a);
    if (g.grid) {
        int sb[3] = {p.sbx, p.sby, p.sbz};
        const int nt[3] = {g.ntx, g.nty, g.ntz};
        const double ext[3] = {BX * (double)g.h, BY * (double)g.h, BZ * (double)g.h};
        while (p.bytes > cap) {
            int best = -1;
            for (int q = 0; q < 3; ++q)
                if (sb[q] < nt[q] && (best < 0 || sb[q] * ext[q] < sb[best] * ext[best])) best = q;
            if (best < 0) return false;
            sb[best] = std::min(nt[best], 2 * sb[best]);
            grid_plan_from_blocks(p, g, a, sb);
        }
        if (p.LB > 2048) return false;    // slab band beyond the kernel's shared-memory budget
    } else {
        while (p.bytes > cap && p.S > 1) soa_plan_from_slabs(p, g, a, (p.S + 1) / 2);
        if (p.bytes > cap) return false;
    }
    out = p;
    return true;
}

bool make_moment_table(const GaussDev& g, const ArrDev& a, MomentTable& T);

// ---- forward plan of the sensor-lane moment kernel (grid Gaussians, shared sigma) ----------
constexpr int CUBE_SIDE = 8;                    // lattice nodes per cube side
constexpr size_t SMEM_PER_CTA = 227 * 1024;     // dynamic shared memory a CTA may use

// Slabs are blocks of sc[0] x sc[1] x sc[2] cubes; a sensor's sample band over a block is bounded
// by the block's diagonal plus the window.  Warps per CTA: as many (up to 4) as the shared
// memory holds.  Returns false when one warp's bands do not fit.
bool lanes_plan_from_blocks(FwdPlan& p, const GaussDev& g, const ArrDev& a, const MomentTable& T, const int sc[3]) {
    const int nc[3] = {(g.nx + CUBE_SIDE - 1) / CUBE_SIDE, (g.ny + CUBE_SIDE - 1) / CUBE_SIDE,
                       (g.nz + CUBE_SIDE - 1) / CUBE_SIDE};
    const int nn[3] = {g.nx, g.ny, g.nz};
    p.sbx = sc[0]; p.sby = sc[1]; p.sbz = sc[2];
    int64_t S = 1;
    double d2 = 0.0;
    for (int q = 0; q < 3; ++q) {
        S *= (nc[q] + sc[q] - 1) / sc[q];
        const double span = (std::min(sc[q] * CUBE_SIDE, nn[q]) - 1) * (double)g.h;   // centre to centre
        d2 += span * span;
    }
    if (S > 65535) return false;            // slabs are the grid's y dimension
    p.S = (int)S;
    p.LB = ((int)std::ceil((std::sqrt(d2) + 2.0 * a.k * g.sigma) * a.invDelta) + 10 + 3) & ~3;
    p.PL = p.LB;
    p.NZ = fwd_lanes_nz(g.h, a.invDelta);
    p.NW = 4;
    while (p.NW > 0 && fwd_lanes_smem(p.NW, p.NZ, p.LB, T.P, T.L) > SMEM_PER_CTA) --p.NW;
    if (p.NW == 0) return false;
    p.lanes = true;
    p.binned = true;
    p.TB = 0;
    plan_offsets(p, g, a);
    return true;
}

// Start from blocks of 4 x 4 x 2 cubes (32 x 32 x 16 nodes) and halve the longest side until the
// grid has about eight CTAs per SM (one CTA fills an SM's shared memory).
bool plan_forward_lanes(const GaussDev& g, const ArrDev& a, const MomentTable& T, FwdPlan& out) {
    const int nc[3] = {(g.nx + CUBE_SIDE - 1) / CUBE_SIDE, (g.ny + CUBE_SIDE - 1) / CUBE_SIDE,
                       (g.nz + CUBE_SIDE - 1) / CUBE_SIDE};
    int sc[3] = {std::min(4, nc[0]), std::min(4, nc[1]), std::min(2, nc[2])};
    FwdPlan p;
    memset(&p, 0, sizeof(p));
    if (!lanes_plan_from_blocks(p, g, a, T, sc)) return false;
    const int64_t target = (int64_t)device_sms() * 8;
    for (;;) {
        const int64_t ctas = (int64_t)p.S * ((a.Nd + 32 * p.NW - 1) / (32 * p.NW));
        if (ctas >= target) break;
        int best = -1;
        for (int q = 0; q < 3; ++q)
            if (sc[q] > 1 && (best < 0 || sc[q] > sc[best])) best = q;
        if (best < 0) break;
        sc[best] = (sc[best] + 1) / 2;
        FwdPlan t;
        memset(&t, 0, sizeof(t));
        if (!lanes_plan_from_blocks(t, g, a, T, sc)) break;
        p = t;
    }
    out = p;
    return true;
}

constexpr int FREE_LANES_WARPS = 8;    // warps (sensor groups of 32) per CTA of the free-centre kernel

// Free-centre Gaussians with the sensor-lane direct kernel: slabs of contiguous tile ranges,
// enough of them for about four CTAs per SM while the partial rows (capacity N_t, rounded up to
// 4, per slab and sensor) stay within 2 GB; the shared signal band per warp as long as 227 KB
// allow (a sensor whose slab band is longer takes several passes).
bool plan_forward_free(const GaussDev& g, const ArrDev& a, FwdPlan& p) {
    memset(&p, 0, sizeof(p));
    p.NW = std::min(FREE_LANES_WARPS, (a.Nd + 31) / 32);
    const int groups = (a.Nd + 32 * p.NW - 1) / (32 * p.NW);
    int64_t S = ((int64_t)device_sms() * 4 + groups - 1) / groups;
    if (S > g.ntiles) S = g.ntiles;
    p.PL = (a.Nt + 3) & ~3;
    const int64_t row = (int64_t)a.Nd * p.PL * 4;
    while (S > 1 && S * row > ((int64_t)2 << 30)) S = (S + 1) / 2;
    if (S < 1 || S > 65535) return false;
    p.tiles_per_slab = (g.ntiles + S - 1) / S;
    p.S = (int)((g.ntiles + p.tiles_per_slab - 1) / p.tiles_per_slab);
    const size_t per_warp = (SMEM_PER_CTA - fwd_free_smem(0, 0)) / p.NW;
    p.LB = std::min<int64_t>(p.PL, (int64_t)(per_warp / (32 * 4)) & ~(int64_t)3);
    if (p.LB < 64) return false;
    p.free_lanes = true;
    plan_offsets(p, g, a);
    p.off_sort = p.bytes;
    p.bytes += align256(spatial_order_bytes(g.M));
    return true;
}

// The operator's plan: the sensor-lane kernels where they apply (grid: the expansion and its
// bands fit; free centres: always), else the brick (grid) or tile-range (free centres) plan.
FwdPlan plan_forward_op(const GaussDev& g, const ArrDev& a) {
    MomentTable T;
    FwdPlan p;
    if (g.grid && make_moment_table(g, a, T) && plan_forward_lanes(g, a, T, p)) return p;
    if (!g.grid && plan_forward_free(g, a, p)) return p;
    return plan_forward(g, a);
}

// The same within `cap` bytes of scratch (the allocation-free entry point): the lanes plan
// coarsened -- its smallest block side doubled -- until its partial rows fit, else the brick or
// tile-range plan coarsened the same way.
bool plan_forward_op_capped(const GaussDev& g, const ArrDev& a, size_t cap, FwdPlan& out) {
    MomentTable T;
    FwdPlan p;
    if (g.grid && make_moment_table(g, a, T) && plan_forward_lanes(g, a, T, p)) {
        const int nc[3] = {(g.nx + CUBE_SIDE - 1) / CUBE_SIDE, (g.ny + CUBE_SIDE - 1) / CUBE_SIDE,
                           (g.nz + CUBE_SIDE - 1) / CUBE_SIDE};
        int sc[3] = {p.sbx, p.sby, p.sbz};
        bool ok = true;
        while (p.bytes > cap) {
            int best = -1;
            for (int q = 0; q < 3; ++q)
                if (sc[q] < nc[q] && (best < 0 || sc[q] < sc[best])) best = q;
            if (best < 0) { ok = false; break; }
            sc[best] = std::min(nc[best], 2 * sc[best]);
            if (!lanes_plan_from_blocks(p, g, a, T, sc)) { ok = false; break; }
        }
        if (ok) {
            out = p;
            return true;
        }
    }
    return plan_forward_capped(g, a, cap, out);
}

// ev (optional): two events recorded immediately before and after the slab kernel.
gpair_status run_forward(const GaussDev& g, const ArrDev& a, float* y, cudaStream_t st, void* scratch, int* status,
                         const FwdPlan& p, const cudaEvent_t* ev = nullptr) {
    char* base = static_cast<char*>(scratch);
    TileInfo* ti = reinterpret_cast<TileInfo*>(base + p.off_ti);
    SlabInfo* si = reinterpret_cast<SlabInfo*>(base + p.off_si);
    int2* rows = reinterpret_cast<int2*>(base + p.off_rows);
    float* part = reinterpret_cast<float*>(base + p.off_part);
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    cudaError_t e = cudaSuccess;
    if (p.free_lanes) {
        // the Gaussians in the Morton order of their centres: tiles of nearby Gaussians, short bands
        GaussDev gp;
        e = launch_spatial_order(g, base + p.off_sort, gp, st);
        if (e == cudaSuccess) e = launch_tile_info(gp, ti, st);
        if (e == cudaSuccess) e = launch_slab_info_soa(gp, gp.ntiles, p.tiles_per_slab, p.S, si, st);
        if (e == cudaSuccess) e = launch_slab_order(si, p.S, st);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], st);
        if (e == cudaSuccess) e = launch_forward_free(gp, a, ti, si, p.S, part, rows, p.PL, p.LB, p.NW, st);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
        if (e == cudaSuccess) e = launch_slab_reduce_rows(a, part, rows, p.S, p.PL, y, st);
        return cuda_status(e);
    }
    if (p.lanes) {
        MomentTable mom;
        if (!make_moment_table(g, a, mom)) return GPAIR_ERR_UNSUPPORTED;
        const bool tma = make_tmap(g, &map, CUBE_SIDE, CUBE_SIDE, CUBE_SIDE);   // ragged pitch: plain loads
        e = launch_slab_info_cubes(g, p.sbx, p.sby, p.sbz, p.S, si, st);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], st);
        if (e == cudaSuccess)
            e = launch_forward_lanes(g, a, si, p.S, part, rows, p.LB, p.NZ, p.NW, status, tma ? &map : nullptr, mom,
                                     st);
        if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
        if (e == cudaSuccess) e = launch_slab_reduce(g, a, part, rows, p.S, p.PL, y, st);
        return cuda_status(e);
    }
    const bool tma = g.grid && make_tmap(g, &map);   // ragged row pitch: plain brick loads instead
    if (g.grid) {
        e = launch_slab_info_grid(g, p.sbx, p.sby, p.sbz, p.S, si, st);
    } else {
        e = launch_tile_info(g, ti, st);
        if (e == cudaSuccess) e = launch_slab_info_soa(g, g.ntiles, p.tiles_per_slab, p.S, si, st);
    }
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], st);
    MomentTable mom;
    const bool use_mom = g.grid && make_moment_table(g, a, mom);
    if (e == cudaSuccess)
        e = launch_forward(g, a, ti, si, p.S, part, rows, p.PL, p.LB, p.TB, p.binned, status, tma ? &map : nullptr,
                           use_mom ? &mom : nullptr, st);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = launch_slab_reduce(g, a, part, rows, p.S, p.PL, y, st);
    return cuda_status(e);
}

// Coefficients of the sub-sample expansion (MomentTable, gpair_internal.cuh) for a shared sigma.
// For window position m the pulse, as a function of the offset e in [-1, 1],
//     K_m(e) = (1/2) d exp(-d^2 / 2 s^2),  d = dstar - m Delta + e Delta / 2
// (with the 1/2 of A / 2R), is replaced by the polynomial of degree P - 1 that interpolates it at
// the 64 Chebyshev points e_i = cos(pi (i + 1/2) / 64), truncated to its first P Chebyshev terms
// (the discrete least-squares fit in the Chebyshev basis, close to the best uniform fit), and
// written in monomials: K_m(e) ~ sum_p c[m][p] e^p.  P is the smallest of 6, 7, 8 whose
// largest error, evaluated against the pulse at 257 offsets per position, is below 3e-7 of the
// pulse's peak.  Returns false when the expansion does not apply (window longer than MOM_LMAX
// samples, or Delta > sigma / 2).
bool make_moment_table(const GaussDev& g, const ArrDev& a, MomentTable& T) {
    if (!g.grid) return false;
    const double s = g.sigma, Delta = (double)a.Delta, k = a.k;
    const double X = 2.0 * k * s / Delta;
    const int E = (int)std::floor(X);
    // position E is inside the window for a fraction X - E of the pairs: include it in the
    // expansion when that is the majority, so that the direct correction stays rare
    const int edge_in = (X - E > 0.5) ? 1 : 0;
    const int L = E + edge_in;
    if (E < 1 || L > MOM_LMAX || Delta > 0.5 * s) return false;
    const double dstar = k * s - 0.5 * Delta;
    T.L = L;
    T.E = E;
    T.edge_in = edge_in;
    T.dstar = (float)dstar;
    T.inv_half = (float)(2.0 / Delta);
    T.e_thr = (float)(((double)E * Delta - k * s - dstar) * (2.0 / Delta));
    for (int m = 0; m < MOM_LMAX; ++m)
        for (int p = 0; p < MOM_P; ++p) T.c[m][p] = 0.f;
    auto pulse = [&](int m, double e) {
        const double d = dstar - m * Delta + 0.5 * Delta * e;
        return 0.5 * d * std::exp(-0.5 * d * d / (s * s));
    };
    constexpr int NC = 64;                       // Chebyshev points
    // monomial coefficients of the Chebyshev polynomials T_0 .. T_{MOM_P-1}
    double Tm[MOM_P][MOM_P] = {};
    Tm[0][0] = 1.0;
    Tm[1][1] = 1.0;
    for (int n = 2; n < MOM_P; ++n)
        for (int q = 0; q < MOM_P; ++q) Tm[n][q] = (q > 0 ? 2.0 * Tm[n - 1][q - 1] : 0.0) - Tm[n - 2][q];
    const double peak = 0.5 * s * std::exp(-0.5);
    static thread_local double cd[MOM_LMAX][MOM_P];
    int P = MOM_P;
    for (int PP = 6; PP <= MOM_P; ++PP) {
        double err = 0.0;
        for (int m = 0; m < L; ++m) {
            double ch[MOM_P] = {};             // Chebyshev coefficients from the discrete orthogonality
            for (int i = 0; i < NC; ++i) {
                const double th = M_PI * (i + 0.5) / NC;
                const double f = pulse(m, std::cos(th));
                for (int n = 0; n < PP; ++n) ch[n] += f * std::cos(n * th);
            }
            for (int n = 0; n < PP; ++n) ch[n] *= (n == 0 ? 1.0 : 2.0) / NC;
            for (int q = 0; q < MOM_P; ++q) {
                double c = 0.0;
                for (int n = 0; n < PP; ++n) c += ch[n] * Tm[n][q];
                cd[m][q] = q < PP ? c : 0.0;
            }
            for (int q = 0; q <= 256; ++q) {
                const double e = -1.0 + q / 128.0;
                double ser = 0.0, ep = 1.0;
                for (int p = 0; p < PP; ++p, ep *= e) ser += cd[m][p] * ep;
                err = std::max(err, std::fabs(pulse(m, e) - ser) / peak);
            }
        }
        P = PP;
        if (err <= 3e-7) break;
    }
    T.P = P;
    for (int m = 0; m < L; ++m)
        for (int p = 0; p < P; ++p) T.c[m][p] = (float)cd[m][p];
    return true;
}

int adjoint_band(const GaussDev& g, const ArrDev& a) {
    if (g.grid) return adj_band_len(brick_radius(g.h), g.sigma, a.k, a.invDelta);
    return 256;
}

// Bytes of the expansion table Q an amplitude-only grid adjoint needs (0 when it does not apply).
size_t adjoint_q_bytes(const GaussDev& g, const ArrDev& a) {
    MomentTable T;
    if (!make_moment_table(g, a, T)) return 0;
    return align256(adj_moment_q_bytes(a, T.L));
}

// qbuf (optional): adjoint_q_bytes() of device memory for the expansion path.
gpair_status run_adjoint(const GaussDev& g, const ArrDev& a, const float* delta, float* gA, float* gc, float* gs,
                         cudaStream_t st, void* scratch, const cudaEvent_t* ev = nullptr, void* qbuf = nullptr) {
    if (qbuf && !gc && !gs) {
        MomentTable T;
        if (make_moment_table(g, a, T))
            return cuda_status(launch_adjoint_moment(g, a, delta, gA, T, static_cast<float*>(qbuf), ev, st));
    }
    TileInfo* ti = static_cast<TileInfo*>(scratch);
    cudaError_t e = launch_tile_info(g, ti, st);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = launch_adjoint(g, a, ti, delta, gA, gc, gs, adjoint_band(g, a), st);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
    return cuda_status(e);
}

}  // namespace

namespace gp {
// The calling stream's pooled device scratch, at least `bytes` long (grown on demand).
gpair_status stream_scratch(cudaStream_t st, size_t bytes, void** buf) { return get_scratch(st, bytes, buf, nullptr); }

// The forward operator run entirely inside caller-provided scratch (`cap` bytes of device memory
// at `scratch`, plus a device status word): validates, plans within the capacity and launches.
// Allocates nothing.  Used by the allocation-free entry point.
gpair_status forward_into_scratch(const gpair_gaussians* gi, const gpair_array* ai, float* y, cudaStream_t st,
                                  void* scratch, size_t cap, int* status) {
    GaussDev g;
    ArrDev a;
    gpair_status s = make_gauss(gi, g);
    if (s != GPAIR_OK) return s;
    if ((s = make_arr(ai, a)) != GPAIR_OK) return s;
    if (!y) return GPAIR_ERR_INVALID_ARG;
    FwdPlan p;
    if (!plan_forward_op_capped(g, a, cap, p)) return GPAIR_ERR_TOO_LARGE;
    return run_forward(g, a, y, st, scratch, status, p);
}
}  // namespace gp

// ============================================================================================
// Public entry points.

extern "C" {

const char* gpair_version(void) { return "gpair-gb300 0.1 (sm_103a)"; }

const char* gpair_status_string(gpair_status s) {
    switch (s) {
        case GPAIR_OK: return "ok";
        case GPAIR_ERR_INVALID_ARG: return "invalid argument";
        case GPAIR_ERR_CUDA: return "CUDA error";
        case GPAIR_ERR_NOMEM: return "out of device memory";
        case GPAIR_ERR_TIMEOUT: return "device-side wait timed out";
        case GPAIR_ERR_UNSUPPORTED: return "unsupported shape or layout";
        case GPAIR_ERR_NONFINITE: return "non-finite input";
        case GPAIR_ERR_TOO_LARGE: return "problem needs more scratch than the allocation-free entry point holds";
    }
    return "unknown status";
}

gpair_status gpair_forward(const gpair_gaussians* gi, const gpair_array* ai, float* y, void* stream) {
    GaussDev g;
    ArrDev a;
    gpair_status s = make_gauss(gi, g);
    if (s != GPAIR_OK) return s;
    if ((s = make_arr(ai, a)) != GPAIR_OK) return s;
    if (!y) return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FwdPlan p = plan_forward_op(g, a);
    void* scratch = nullptr;
    int* status = nullptr;
    if ((s = get_scratch(st, p.bytes, &scratch, &status)) != GPAIR_OK) return s;
    return run_forward(g, a, y, st, scratch, status, p);
}

gpair_status gpair_adjoint(const gpair_gaussians* gi, const gpair_array* ai, const float* delta, float* gA,
                           float* gc, float* gsigma, void* stream) {
    GaussDev g;
    ArrDev a;
    gpair_status s = make_gauss(gi, g);
    if (s != GPAIR_OK) return s;
    if ((s = make_arr(ai, a)) != GPAIR_OK) return s;
    if (!delta || !gA) return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    const size_t ti_bytes = align256(sizeof(TileInfo) * (size_t)g.ntiles);
    const size_t q_bytes = (gc || gsigma) ? 0 : adjoint_q_bytes(g, a);
    if ((s = get_scratch(st, ti_bytes + q_bytes, &scratch, nullptr)) != GPAIR_OK) return s;
    return run_adjoint(g, a, delta, gA, gc, gsigma, st, scratch, nullptr,
                       q_bytes ? static_cast<char*>(scratch) + ti_bytes : nullptr);
}

gpair_status gpair_shard_range(const gpair_grid* grid, int shard, int n_shards, int* z_begin, int* z_end) {
    if (!grid || !z_begin || !z_end || n_shards < 1 || shard < 0 || shard >= n_shards || grid->nz < 0)
        return GPAIR_ERR_INVALID_ARG;
    const int64_t nz = grid->nz, base = nz / n_shards, extra = nz % n_shards;
    const int64_t zb = shard * base + std::min<int64_t>(shard, extra);
    *z_begin = (int)zb;
    *z_end = (int)(zb + base + (shard < extra ? 1 : 0));
    return GPAIR_OK;
}

}  // extern "C"

namespace {
// The lattice rows [z0, z1) of a grid-implicit set as a set of its own: the same nodes (the
// origin moves by z0 spacings, exactly, in double) and amplitudes from row z0 on.
GaussDev zslab(const GaussDev& g, int z0, int z1, const float* A) {
    GaussDev s = g;
    s.nz = z1 - z0;
    s.oz = g.oz + (double)z0 * (double)g.h;
    s.A = A + (int64_t)z0 * g.nx * g.ny;
    s.M = (int64_t)g.nx * g.ny * s.nz;
    s.ntz = (s.nz + BZ - 1) / BZ;
    s.ntiles = (int64_t)s.ntx * s.nty * s.ntz;
    return s;
}

gpair_status shard_inputs(const gpair_gaussians* gi, const gpair_array* ai, int shard, int n_shards, GaussDev& g,
                          ArrDev& a, int& z0, int& z1) {
    gpair_status s = make_gauss(gi, g);
    if (s != GPAIR_OK) return s;
    if ((s = make_arr(ai, a)) != GPAIR_OK) return s;
    if (!g.grid) return GPAIR_ERR_UNSUPPORTED;
    return gpair_shard_range(gi->grid, shard, n_shards, &z0, &z1);
}
}  // namespace

extern "C" {

gpair_status gpair_forward_shard(const gpair_gaussians* gi, const gpair_array* ai, int shard, int n_shards, float* y,
                                 void* stream) {
    GaussDev g;
    ArrDev a;
    int z0 = 0, z1 = 0;
    gpair_status s = shard_inputs(gi, ai, shard, n_shards, g, a, z0, z1);
    if (s != GPAIR_OK) return s;
    if (!y) return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (z1 <= z0)
        return cuda_status(cudaMemsetAsync(y, 0, sizeof(float) * (size_t)a.Nd * a.Nt, st));
    const GaussDev gs = zslab(g, z0, z1, gi->A);
    FwdPlan p = plan_forward_op(gs, a);
    void* scratch = nullptr;
    int* status = nullptr;
    if ((s = get_scratch(st, p.bytes, &scratch, &status)) != GPAIR_OK) return s;
    return run_forward(gs, a, y, st, scratch, status, p);
}

gpair_status gpair_adjoint_shard(const gpair_gaussians* gi, const gpair_array* ai, int shard, int n_shards,
                                 const float* delta, float* gA, void* stream) {
    GaussDev g;
    ArrDev a;
    int z0 = 0, z1 = 0;
    gpair_status s = shard_inputs(gi, ai, shard, n_shards, g, a, z0, z1);
    if (s != GPAIR_OK) return s;
    if (!delta || !gA) return GPAIR_ERR_INVALID_ARG;
    if (z1 <= z0) return GPAIR_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const GaussDev gs = zslab(g, z0, z1, gi->A);
    void* scratch = nullptr;
    const size_t ti_bytes = align256(sizeof(TileInfo) * (size_t)gs.ntiles);
    const size_t q_bytes = adjoint_q_bytes(gs, a);
    if ((s = get_scratch(st, ti_bytes + q_bytes, &scratch, nullptr)) != GPAIR_OK) return s;
    return run_adjoint(gs, a, delta, gA + (int64_t)z0 * g.nx * g.ny, nullptr, nullptr, st, scratch, nullptr,
                       q_bytes ? static_cast<char*>(scratch) + ti_bytes : nullptr);
}

gpair_status gpair_voxelize(const gpair_gaussians* gi, const gpair_grid* og, float window_k, float* vol,
                            void* stream) {
    GaussDev g;
    gpair_status s = make_gauss(gi, g);
    if (s != GPAIR_OK) return s;
    if (!og || !vol || og->nx <= 0 || og->ny <= 0 || og->nz <= 0 || !finite_pos(og->dx) || !finite_pos(window_k))
        return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* tmp = nullptr;
    if (vox_is_lattice(g, *og)) {
        size_t bytes = (size_t)og->nx * og->ny * og->nz * 4;
        if ((s = get_scratch(st, bytes, &tmp, nullptr)) != GPAIR_OK) return s;
    }
    return cuda_status(launch_voxelize(g, *og, window_k, vol, static_cast<float*>(tmp), st));
}

gpair_status gpair_reduce_f64(const float* a, const float* b, const float* c, int64_t n, double* out, void* stream) {
    if (!a || !out || n <= 0) return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    gpair_status s = get_scratch(st, sizeof(double) * 2 * red_blocks(), &scratch, nullptr);
    if (s != GPAIR_OK) return s;
    return cuda_status(launch_reduce2(a, b, c, n, static_cast<double*>(scratch), out, st));
}

gpair_status gpair_last_device_status(void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* status = nullptr;
    gpair_status s = get_scratch(st, 0, nullptr, &status);
    if (s != GPAIR_OK) return s;
    int h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (h == DEV_TIMEOUT) return GPAIR_ERR_TIMEOUT;
    if (h == DEV_CAPACITY) return GPAIR_ERR_UNSUPPORTED;
    return GPAIR_OK;
}

}  // extern "C"

// ---- the paper's operator (Methods, adaptive supersampling alignment; Algorithm 1) -------------
// Helpers of the ASSA entry points and of the solver's ASSA path (file-local).
namespace {

// Grid parameters and the sampled pulse: N_half = ceil(3 sigma / (v / fs)),
// alpha = max(1, ceil(((N_min - 1) / 2) / N_half)), K = alpha N_half, all in double from the
// arguments as given; hr[t] = h[K - t], h[k] = (1/2) d exp(-d^2 / 2 sigma^2), d = -v k / (alpha fs).
bool make_assa_table(const GaussDev& g, const ArrDev& a, int n_min, AssaTable& T) {
    const double s = g.sigma, v = a.v, fs = a.fs;
    int nh = (int)std::ceil(3.0 * s / (v / fs));
    if (nh < 1) nh = 1;
    int alpha = (int)std::ceil(((double)(n_min - 1) / 2.0) / (double)nh);
    if (alpha < 1) alpha = 1;
    if ((int64_t)alpha * nh > ASSA_KMAX || (int64_t)alpha * a.Nt >= (1LL << 30)) return false;
    if ((int64_t)a.Nd * alpha * a.Nt >= (int64_t)INT32_MAX) return false;   // 32-bit row offsets in the adjoint
    T.alpha = alpha;
    T.n_half = nh;
    T.K = alpha * nh;
    const double fs_up = alpha * fs;
    for (int t = 0; t <= 2 * ASSA_KMAX; ++t) T.hr[t] = 0.f;
    for (int t = 0; t <= 2 * T.K; ++t) {
        const double d = -v * (double)(T.K - t) / fs_up;
        T.hr[t] = (float)(0.5 * d * std::exp(-d * d / (2.0 * s * s)));
    }
    return true;
}

gpair_status assa_inputs(const gpair_gaussians* gi, const gpair_array* ai, int n_min, GaussDev& g, ArrDev& a,
                         AssaTable& T) {
    gpair_status s = make_gauss(gi, g);
    if (s != GPAIR_OK) return s;
    if ((s = make_arr(ai, a)) != GPAIR_OK) return s;
    if (n_min < 1) return GPAIR_ERR_INVALID_ARG;
    if (!g.grid) return GPAIR_ERR_UNSUPPORTED;      // one pulse table: a shared width
    if (!make_assa_table(g, a, n_min, T)) return GPAIR_ERR_UNSUPPORTED;
    return GPAIR_OK;
}

// The slab bands of the ASSA forward hold the pulse half-width N_half v / fs plus half a fine step.
ArrDev assa_band_array(const GaussDev& g, const ArrDev& a, const AssaTable& T) {
    ArrDev aa = a;
    aa.k = (float)((T.n_half * (double)a.Delta + 0.5 * (double)a.Delta / T.alpha) / (double)g.sigma * 1.001 + 1e-3);
    return aa;
}

// Scratch of the ASSA forward beyond the plan: max |A| for the fixed-point bands.
constexpr size_t ASSA_EXTRA_BYTES = 256;

// ASSA forward into y with scratch of p.bytes + ASSA_EXTRA_BYTES (p = plan_forward(g, assa_band_array(...))).
gpair_status run_assa_forward(const GaussDev& g, const ArrDev& aa, const AssaTable& T, const FwdPlan& p, float* y,
                              void* scratch, int* status, const cudaEvent_t* ev, cudaStream_t st) {
    char* base = static_cast<char*>(scratch);
    SlabInfo* si = reinterpret_cast<SlabInfo*>(base + p.off_si);
    int2* rows = reinterpret_cast<int2*>(base + p.off_rows);
    float* part = reinterpret_cast<float*>(base + p.off_part);
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    const bool tma = make_tmap(g, &map);
    cudaError_t e = launch_slab_info_grid(g, p.sbx, p.sby, p.sbz, p.S, si, st);
    if (e == cudaSuccess)
        e = launch_assa_forward(g, aa, si, p.S, part, rows, p.LB, status, tma ? &map : nullptr, T,
                                reinterpret_cast<unsigned*>(base + p.bytes), ev, st);
    if (e == cudaSuccess) e = launch_slab_reduce(g, aa, part, rows, p.S, p.PL, y, st);
    return cuda_status(e);
}

}  // namespace

extern "C" {

gpair_status gpair_assa_forward(const gpair_gaussians* gi, const gpair_array* ai, int n_min, float* y, void* stream) {
    GaussDev g;
    ArrDev a;
    AssaTable T;
    gpair_status s = assa_inputs(gi, ai, n_min, g, a, T);
    if (s != GPAIR_OK) return s;
    if (!y) return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const ArrDev aa = assa_band_array(g, a, T);
    FwdPlan p = plan_forward(g, aa);
    void* scratch = nullptr;
    int* status = nullptr;
    if ((s = get_scratch(st, p.bytes + ASSA_EXTRA_BYTES, &scratch, &status)) != GPAIR_OK) return s;
    return run_assa_forward(g, aa, T, p, y, scratch, status, nullptr, st);
}

gpair_status gpair_assa_adjoint(const gpair_gaussians* gi, const gpair_array* ai, int n_min, const float* delta,
                                float* gA, void* stream) {
    GaussDev g;
    ArrDev a;
    AssaTable T;
    gpair_status s = assa_inputs(gi, ai, n_min, g, a, T);
    if (s != GPAIR_OK) return s;
    if (!delta || !gA) return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    if ((s = get_scratch(st, assa_dconv_bytes(a, T), &scratch, nullptr)) != GPAIR_OK) return s;
    return cuda_status(launch_assa_adjoint(g, a, delta, gA, T, static_cast<float*>(scratch), nullptr, st));
}

gpair_status gpair_vcr(const float* x, int nx, int ny, int nz, float beta, float eps, float lam, float* grad,
                       double* value_out, void* stream) {
    if (!x || nx <= 0 || ny <= 0 || nz <= 0 || !(eps >= 0.f) || !std::isfinite(beta) || !std::isfinite(lam))
        return GPAIR_ERR_INVALID_ARG;
    if ((int64_t)ny * nz > (int64_t)INT32_MAX) return GPAIR_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    gpair_status s = get_scratch(st, sizeof(double) * ((size_t)red_blocks() + 1), &scratch, nullptr);
    if (s != GPAIR_OK) return s;
    double* partial = static_cast<double*>(scratch);
    double* val = partial + red_blocks();
    cudaError_t e = launch_vcr(x, nx, ny, nz, beta, eps, lam, partial, value_out ? val : nullptr, grad, st);
    if (e != cudaSuccess) return cuda_status(e);
    if (value_out) {
        if (cudaMemcpyAsync(value_out, val, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return GPAIR_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return GPAIR_ERR_CUDA;
    }
    return GPAIR_OK;
}

gpair_status gpair_zmap(const float* vol, int nx, int ny, int nz, float* out, void* stream) {
    if (!vol || !out || nx <= 0 || ny <= 0 || nz <= 0) return GPAIR_ERR_INVALID_ARG;
    return cuda_status(launch_zmap(vol, nx, ny, nz, out, static_cast<cudaStream_t>(stream)));
}

gpair_status gpair_image_metrics(const float* x, const float* ref, int nx, int ny, int nz, int win, float data_range,
                                 double* out, void* stream) {
    if (!x || !ref || !out || nx <= 0 || ny <= 0 || nz <= 0 || win < 3 || (win & 1) == 0 || !(data_range > 0.f))
        return GPAIR_ERR_INVALID_ARG;
    if (nx < win || ny < win || (nz > 1 && nz < win) || (int64_t)ny * nz > (int64_t)INT32_MAX)
        return GPAIR_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t M = (int64_t)nx * ny * nz;
    const int p = (win - 1) / 2;
    // one fused pass for windows up to 15 (res[0] = sum (x - ref)^2, res[2] = sum of SSIM), else the
    // FP64 reduction and the per-axis box passes through 10 M floats of scratch volumes
    const bool fused = p <= metrics_march_pmax();
    const size_t sbytes = fused ? 0 : align256(ssim_scratch_bytes(M));
    const size_t npart = std::max(2 * (size_t)red_blocks(), ssim_march_partial_doubles());
    void* scratch = nullptr;
    gpair_status s = get_scratch(st, sbytes + sizeof(double) * (npart + 4), &scratch, nullptr);
    if (s != GPAIR_OK) return s;
    double* partial = reinterpret_cast<double*>(static_cast<char*>(scratch) + sbytes);
    double* res = partial + npart;
    cudaError_t e;
    if (fused) {
        e = launch_metrics_march(x, ref, nx, ny, nz, win, data_range, partial, res, st);
    } else {
        e = launch_reduce2(x, ref, nullptr, M, partial, res, st);
        if (e == cudaSuccess) e = launch_ssim_sum(x, ref, nx, ny, nz, win, data_range, scratch, res + 2, st);
    }
    if (e != cudaSuccess) return cuda_status(e);
    double h[3];
    if (cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GPAIR_ERR_CUDA;
    const double inner = (double)(nx - 2 * p) * (ny - 2 * p) * (nz > 1 ? nz - 2 * p : 1);
    out[0] = h[0] / (double)M;
    out[1] = 10.0 * std::log10((double)data_range * data_range / out[0]);
    out[2] = h[2] / inner;
    return GPAIR_OK;
}

gpair_status gpair_wait_selftest(int polls, void* stream) {
    if (polls < 1 || polls > (1 << 20)) return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* status = nullptr;
    gpair_status s = get_scratch(st, 0, nullptr, &status);
    if (s != GPAIR_OK) return s;
    return cuda_status(launch_wait_selftest((uint32_t)polls, status, st));
}

void gpair_release_scratch(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto it = g_pool.begin(); it != g_pool.end();) {
        if ((it->first >> 48) == (uint64_t)(uint32_t)dev) {
            cudaDeviceSynchronize();
            if (it->second.buf) cudaFree(it->second.buf);
            if (it->second.status) cudaFree(it->second.status);
            it = g_pool.erase(it);
        } else {
            ++it;
        }
    }
}

}  // extern "C"

// ============================================================================================
// Reconstruction solver (Algorithm 2).

struct gpair_solver {
    GaussDev g;              // A points at x (amplitudes of the current iterate)
    ArrDev a;
    gpair_step_params p;
    int t = 0;
    float *z = nullptr, *m = nullptr, *v = nullptr, *x = nullptr, *gx = nullptr;
    float *y = nullptr, *delta = nullptr, *Fg = nullptr;
    double* red = nullptr;   // reduction partials (2 * red_blocks) + results (4)
    void* fwd_scratch = nullptr;
    void* qbuf = nullptr;    // expansion table of the amplitude adjoint (grid Gaussians)
    bool vcr = false;        // vessel continuity regulariser in the step (vcr_lambda > 0)
    int* status = nullptr;
    FwdPlan plan;            // of a, or of aa with the ASSA operator
    // ASSA operator (op = 1): pulse table, band-widened array and the adjoint's kernel-response table.
    bool assa = false;
    AssaTable T;
    ArrDev aa;
    float* dconv = nullptr;
    // Per-step scalars on the device (CAWR step size, Adam bias corrections, the step count).
    StepSched* sd = nullptr;
    SchedParams sched{};
    // gpair_solver_steps: one step captured as a CUDA graph (on a private stream) for data b.
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const float* gb = nullptr;
    // Profiling (gpair_solver_profile): per recorded step six events on the step's stream --
    // step start, forward slab kernel start/end, adjoint kernel start/end, step end.
    bool prof = false;
    std::vector<cudaEvent_t> evs;
    int nrec = 0;
};

namespace {

// y = F(S->g with amplitudes S->g.A) on the solver's operator; ev (optional) brackets its main kernel.
gpair_status solver_forward(gpair_solver* S, float* y, const cudaEvent_t* ev, cudaStream_t st) {
    if (S->assa) return run_assa_forward(S->g, S->aa, S->T, S->plan, y, S->fwd_scratch, S->status, ev, st);
    return run_forward(S->g, S->a, y, st, S->fwd_scratch, S->status, S->plan, ev);
}

// gA = F^T delta on the solver's operator.
gpair_status solver_adjoint(gpair_solver* S, const float* delta, float* gA, const cudaEvent_t* ev, cudaStream_t st) {
    if (S->assa) return cuda_status(launch_assa_adjoint(S->g, S->a, delta, gA, S->T, S->dconv, ev, st));
    // the amplitude adjoint needs only the tile summaries of the forward scratch (same layout)
    return run_adjoint(S->g, S->a, delta, gA, nullptr, nullptr, st, S->fwd_scratch, ev, S->qbuf);
}
}  // namespace

extern "C" {

gpair_status gpair_solver_create(const gpair_gaussians* gi, const gpair_array* ai, const gpair_step_params* prm,
                                 gpair_solver** out) {
    if (!out || !prm) return GPAIR_ERR_INVALID_ARG;
    *out = nullptr;
    gpair_gaussians tmp = gi ? *gi : gpair_gaussians{};
    static const float one = 1.f;
    tmp.A = &one;   // amplitudes come from the solver; validate the rest
    GaussDev g;
    ArrDev a;
    gpair_status s = make_gauss(&tmp, g);
    if (s != GPAIR_OK) return s;
    if ((s = make_arr(ai, a)) != GPAIR_OK) return s;
    if (prm->rule != GPAIR_RULE_ADAM && prm->rule != GPAIR_RULE_GD_LINESEARCH) return GPAIR_ERR_INVALID_ARG;
    if (prm->rule == GPAIR_RULE_ADAM &&
        (!(prm->beta1 >= 0.f && prm->beta1 < 1.f) || !(prm->beta2 >= 0.f && prm->beta2 < 1.f) || !(prm->adam_eps >= 0.f)))
        return GPAIR_ERR_INVALID_ARG;
    const bool vcr = prm->vcr_lambda != 0.f;
    if (!std::isfinite(prm->vcr_lambda) || prm->vcr_lambda < 0.f || (vcr && (!(prm->vcr_eps >= 0.f) ||
                                                                          !std::isfinite(prm->vcr_beta))))
        return GPAIR_ERR_INVALID_ARG;
    if (vcr && (prm->rule != GPAIR_RULE_ADAM || !g.grid || (int64_t)g.ny * g.nz > (int64_t)INT32_MAX))
        return GPAIR_ERR_UNSUPPORTED;
    if (prm->op != 0 && prm->op != 1) return GPAIR_ERR_INVALID_ARG;
    const bool assa = prm->op == 1;
    if (assa && prm->n_min < 1) return GPAIR_ERR_INVALID_ARG;
    if (assa && !g.grid) return GPAIR_ERR_UNSUPPORTED;
    gpair_solver* S = new gpair_solver();
    S->g = g;
    S->a = a;
    S->p = *prm;
    S->assa = assa;
    S->vcr = vcr;
    if (assa && !make_assa_table(g, a, prm->n_min, S->T)) {
        delete S;
        return GPAIR_ERR_UNSUPPORTED;
    }
    const size_t M = (size_t)g.M, N = (size_t)a.Nd * a.Nt;
    if (assa) S->aa = assa_band_array(g, a, S->T);
    S->plan = assa ? plan_forward(g, S->aa) : plan_forward_op(g, a);
    const size_t qbytes = assa ? 0 : adjoint_q_bytes(g, a);
    bool ok = cudaMalloc(&S->z, M * 4) == cudaSuccess && cudaMalloc(&S->m, M * 4) == cudaSuccess &&
              cudaMalloc(&S->v, M * 4) == cudaSuccess && cudaMalloc(&S->x, M * 4) == cudaSuccess &&
              cudaMalloc(&S->gx, M * 4) == cudaSuccess && cudaMalloc(&S->y, N * 4) == cudaSuccess &&
              cudaMalloc(&S->delta, N * 4) == cudaSuccess &&
              (prm->rule != GPAIR_RULE_GD_LINESEARCH || cudaMalloc(&S->Fg, N * 4) == cudaSuccess) &&
              cudaMalloc(&S->red, sizeof(double) * (2 * red_blocks() + 8)) == cudaSuccess &&
              cudaMalloc(&S->fwd_scratch, S->plan.bytes + (assa ? ASSA_EXTRA_BYTES : 0)) == cudaSuccess &&
              (qbytes == 0 || cudaMalloc(&S->qbuf, qbytes) == cudaSuccess) &&
              (!assa || cudaMalloc(&S->dconv, assa_dconv_bytes(a, S->T)) == cudaSuccess) &&
              cudaMalloc(&S->status, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&S->sd, sizeof(StepSched)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        gpair_solver_destroy(S);
        return GPAIR_ERR_NOMEM;
    }
    cudaMemset(S->z, 0, M * 4);
    cudaMemset(S->m, 0, M * 4);
    cudaMemset(S->v, 0, M * 4);
    cudaMemset(S->status, 0, sizeof(int));
    S->sched = SchedParams{prm->eta_max, prm->eta_min, prm->T_mult, prm->beta1, prm->beta2, prm->T0};
    cudaMemset(S->sd, 0, sizeof(StepSched));
    launch_set_step(S->sd, 0, S->sched, 0);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        gpair_solver_destroy(S);
        return GPAIR_ERR_CUDA;
    }
    S->g.A = S->x;
    *out = S;
    return GPAIR_OK;
}

void gpair_solver_destroy(gpair_solver* S) {
    if (!S) return;
    cudaFree(S->z); cudaFree(S->m); cudaFree(S->v); cudaFree(S->x); cudaFree(S->gx);
    cudaFree(S->y); cudaFree(S->delta); cudaFree(S->Fg); cudaFree(S->red);
    cudaFree(S->fwd_scratch); cudaFree(S->qbuf); cudaFree(S->status); cudaFree(S->dconv); cudaFree(S->sd);
    if (S->gexec) cudaGraphExecDestroy(S->gexec);
    if (S->cap) cudaStreamDestroy(S->cap);
    for (cudaEvent_t ev : S->evs) cudaEventDestroy(ev);
    delete S;
}

gpair_status gpair_solver_profile(gpair_solver* S, int enable) {
    if (!S) return GPAIR_ERR_INVALID_ARG;
    S->prof = enable != 0;
    S->nrec = 0;
    return GPAIR_OK;
}

gpair_status gpair_solver_timings(gpair_solver* S, double* ms, int* nsteps) {
    if (!S || !ms) return GPAIR_ERR_INVALID_ARG;
    ms[0] = ms[1] = ms[2] = 0.0;
    if (S->nrec > 0 && cudaEventSynchronize(S->evs[6 * S->nrec - 1]) != cudaSuccess) return GPAIR_ERR_CUDA;
    for (int q = 0; q < S->nrec; ++q) {
        const cudaEvent_t* e = &S->evs[6 * q];
        float f = 0.f, a = 0.f, t = 0.f;
        if (cudaEventElapsedTime(&f, e[1], e[2]) != cudaSuccess || cudaEventElapsedTime(&a, e[3], e[4]) != cudaSuccess ||
            cudaEventElapsedTime(&t, e[0], e[5]) != cudaSuccess)
            return GPAIR_ERR_CUDA;
        ms[0] += f; ms[1] += a; ms[2] += t;
    }
    if (nsteps) *nsteps = S->nrec;
    S->nrec = 0;
    return GPAIR_OK;
}

}  // extern "C"

namespace {
// The launches of one reconstruction step on st: no host synchronisation, S->t unchanged, and the
// same launches with the same arguments at every step (so that they can be replayed as a graph).
gpair_status step_launches(gpair_solver* S, const float* b, const cudaEvent_t* ev, cudaStream_t st) {
    const int64_t M = S->g.M, N = (int64_t)S->a.Nd * S->a.Nt;
    double* partial = S->red;
    double* res = S->red + 2 * red_blocks();
    cudaError_t e;
    gpair_status s;
    if (S->p.rule == GPAIR_RULE_ADAM) {
        const int npc = S->p.npc != 0;
        if ((e = launch_npc(S->z, S->x, M, npc, S->p.npc_eps, st)) != cudaSuccess) return cuda_status(e);
        if ((s = solver_forward(S, S->y, ev ? ev + 1 : nullptr, st)) != GPAIR_OK) return s;
        if ((e = launch_resid(S->y, b, S->delta, (float)(2.0 / (double)N), N, partial, res, st)) != cudaSuccess)
            return cuda_status(e);
        if ((s = solver_adjoint(S, S->delta, S->gx, ev ? ev + 3 : nullptr, st)) != GPAIR_OK) return s;
        if (S->vcr &&    // grad_x += lambda grad R_VCR(x); R_VCR(x) into res[4]
            (e = launch_vcr(S->x, S->g.nx, S->g.ny, S->g.nz, S->p.vcr_beta, S->p.vcr_eps, S->p.vcr_lambda, partial,
                            res + 4, S->gx, st)) != cudaSuccess)
            return cuda_status(e);
        // CAWR step size and bias corrections of this step, from the device step count
        if ((e = launch_schedule(S->sched, S->sd, st)) != cudaSuccess) return cuda_status(e);
        if ((e = launch_adam(S->z, S->m, S->v, S->gx, M, npc, S->p.npc_eps, S->p.beta1, S->p.beta2, S->p.adam_eps,
                             S->sd, st)) != cudaSuccess)
            return cuda_status(e);
    } else {
        // steepest descent on x = z with the exact line search alpha = <r, F g> / |F g|^2
        S->g.A = S->z;
        s = solver_forward(S, S->y, ev ? ev + 1 : nullptr, st);
        if (s == GPAIR_OK && (e = launch_resid(S->y, b, S->delta, 1.0f, N, partial, res, st)) != cudaSuccess)
            s = cuda_status(e);
        if (s == GPAIR_OK) s = solver_adjoint(S, S->delta, S->gx, ev ? ev + 3 : nullptr, st);
        S->g.A = S->gx;
        if (s == GPAIR_OK) s = solver_forward(S, S->Fg, nullptr, st);
        if (s == GPAIR_OK && (e = launch_ls(S->delta, S->Fg, N, S->z, S->gx, M, partial, res + 2, st)) != cudaSuccess)
            s = cuda_status(e);
        S->g.A = S->x;
        if (s != GPAIR_OK) return s;
    }
    return GPAIR_OK;
}

// The FP64 loss and residual norm of the iterate that entered the last step (synchronises st).
gpair_status read_loss(gpair_solver* S, cudaStream_t st, double* loss_out, double* resid_out) {
    if (!loss_out && !resid_out) return GPAIR_OK;
    const double N = (double)S->a.Nd * S->a.Nt;
    const double* res = S->red + 2 * red_blocks();
    double h[5] = {0, 0, 0, 0, 0};
    if (cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GPAIR_ERR_CUDA;
    const double reg = S->vcr ? (double)S->p.vcr_lambda * h[4] : 0.0;
    if (loss_out) *loss_out = h[0] / N + reg;
    if (resid_out) *resid_out = std::sqrt(h[0]);
    return GPAIR_OK;
}
}  // namespace

extern "C" {

gpair_status gpair_step(gpair_solver* S, const float* b, double* loss_out, double* resid_out, void* stream) {
    if (!S || !b) return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaEvent_t* ev = nullptr;
    if (S->prof) {
        while ((int)S->evs.size() < 6 * (S->nrec + 1)) {
            cudaEvent_t x;
            if (cudaEventCreate(&x) != cudaSuccess) return GPAIR_ERR_CUDA;
            S->evs.push_back(x);
        }
        ev = &S->evs[6 * S->nrec];
        if (cudaEventRecord(ev[0], st) != cudaSuccess) return GPAIR_ERR_CUDA;
    }
    gpair_status s = step_launches(S, b, ev, st);
    if (s != GPAIR_OK) {
        // the schedule kernel may have advanced the device step count before a later launch failed:
        // put it back to the host count, so that a checkpoint taken now resumes with the right step
        if (S->p.rule == GPAIR_RULE_ADAM) launch_set_step(S->sd, S->t, S->sched, st);
        return s;
    }
    if (ev) {
        if (cudaEventRecord(ev[5], st) != cudaSuccess) return GPAIR_ERR_CUDA;
        S->nrec += 1;
    }
    S->t += 1;
    return read_loss(S, st, loss_out, resid_out);
}

gpair_status gpair_solver_steps(gpair_solver* S, const float* b, int n, double* loss_out, double* resid_out,
                                void* stream) {
    if (!S || !b || n < 0) return GPAIR_ERR_INVALID_ARG;
    if (n == 0) return GPAIR_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (S->prof) {   // profiling records events per step: step by step
        for (int k = 0; k < n; ++k) {
            const bool last = k == n - 1;
            const gpair_status s = gpair_step(S, b, last ? loss_out : nullptr, last ? resid_out : nullptr, stream);
            if (s != GPAIR_OK) return s;
        }
        return GPAIR_OK;
    }
    if (!S->gexec || S->gb != b) {
        if (S->gexec) {
            cudaGraphExecDestroy(S->gexec);
            S->gexec = nullptr;
        }
        if (!S->cap && cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking) != cudaSuccess) return GPAIR_ERR_CUDA;
        // the capture records the step's launches without running them
        if (cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return GPAIR_ERR_CUDA;
        const gpair_status s = step_launches(S, b, nullptr, S->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(S->cap, &graph);
        if (s != GPAIR_OK || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return s != GPAIR_OK ? s : GPAIR_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&S->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            S->gexec = nullptr;
            cudaGetLastError();
            return GPAIR_ERR_CUDA;
        }
        S->gb = b;
    }
    for (int k = 0; k < n; ++k)
        if (cudaGraphLaunch(S->gexec, st) != cudaSuccess) {
            S->t += k;      // the k replays already queued advance the device step count
            return GPAIR_ERR_CUDA;
        }
    S->t += n;
    return read_loss(S, st, loss_out, resid_out);
}

gpair_status gpair_solver_image(gpair_solver* S, float* x_out, void* stream) {
    if (!S || !x_out) return GPAIR_ERR_INVALID_ARG;
    const int npc = S->p.rule == GPAIR_RULE_ADAM && S->p.npc != 0;
    return cuda_status(launch_npc(S->z, x_out, S->g.M, npc, S->p.npc_eps, static_cast<cudaStream_t>(stream)));
}

gpair_status gpair_solver_get_state(gpair_solver* S, float* z, float* m, float* v, int* t, void* stream) {
    if (!S) return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)S->g.M * 4;
    if (z && cudaMemcpyAsync(z, S->z, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (m && cudaMemcpyAsync(m, S->m, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (v && cudaMemcpyAsync(v, S->v, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (t) *t = S->t;
    return GPAIR_OK;
}

gpair_status gpair_solver_set_state(gpair_solver* S, const float* z, const float* m, const float* v, int t,
                                    void* stream) {
    if (!S || t < 0) return GPAIR_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)S->g.M * 4;
    if (z && cudaMemcpyAsync(S->z, z, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (m && cudaMemcpyAsync(S->m, m, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (v && cudaMemcpyAsync(S->v, v, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return GPAIR_ERR_CUDA;
    if (launch_set_step(S->sd, t, S->sched, st) != cudaSuccess) return GPAIR_ERR_CUDA;
    S->t = t;
    return GPAIR_OK;
}

}  // extern "C"
