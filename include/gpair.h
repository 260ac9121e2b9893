/*
 * gpair.h -- C ABI of the GB300 GPAIR forward/adjoint library (libgpair.so).
 *
 * GPAIR (arXiv 2602.03893) models the photoacoustic initial pressure as a sum of isotropic
 * 3-D Gaussians (Methods, Eqs. 1-2) and derives the pressure one Gaussian produces at a point
 * detector in closed form (Eq. single_forward):
 *
 *     p(R, t) = A / (2R) * d * exp(-d^2 / (2 sigma^2)),   d = R - v t,
 *
 * kept where |d| <= k sigma (the paper's 3-sigma principle; k = window_k, inclusive).  This
 * library evaluates that window directly for every (Gaussian, sensor) pair -- the exact pair
 * enumeration the Methods section describes before introducing its approximate upsampled
 * alignment -- and its exact transpose.
 *
 * Units are SI throughout (metres, seconds, m/s, Hz).  Sample n of every sensor is taken at
 * t_n = t0 + n / fs.  Signals are float32, sensor-major: y[j * n_samples + n].
 *
 * Memory: every data pointer is caller-owned DEVICE memory on the current CUDA device unless a
 * field says otherwise; struct arguments themselves are host memory, read during the call
 * only.  The library owns a per-(device, stream) scratch pool (grown on demand with
 * cudaMalloc, released by gpair_release_scratch) and the workspace inside a gpair_solver.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 * are asynchronous on that stream; a call that returns a host scalar (gpair_step) synchronises
 * that stream only.
 *
 * Errors: every entry point returns a gpair_status and never aborts or prints.  Arguments are
 * validated before any launch (INVALID_ARG).  Device-side failures (a bounded wait that ran
 * out, an internal capacity exceeded) set a per-stream status word that
 * gpair_last_device_status() reads and clears.
 *
 * Thread safety: calls on distinct streams (or distinct solvers) may run concurrently from
 * different host threads.
 */
#ifndef GPAIR_H
#define GPAIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GPAIR_OK = 0,
    GPAIR_ERR_INVALID_ARG = 1,   /* a NULL pointer, a non-positive size, fs <= 0, k <= 0, ... */
    GPAIR_ERR_CUDA = 2,          /* a CUDA runtime call failed (launch, copy, ...) */
    GPAIR_ERR_NOMEM = 3,         /* scratch/workspace allocation failed */
    GPAIR_ERR_TIMEOUT = 4,       /* a device-side bounded wait ran out (reported on the stream) */
    GPAIR_ERR_UNSUPPORTED = 5,   /* shape outside the supported envelope (e.g. window too long) */
    GPAIR_ERR_NONFINITE = 6,     /* non-finite input detected (validation builds) */
    GPAIR_ERR_TOO_LARGE = 7      /* gpair_forward_noalloc: the problem does not fit its fixed scratch */
} gpair_status;

/* Regular grid of Gaussian centres (Methods, GKD: one Gaussian per voxel centre).
 * Centre of node (ix, iy, iz) is (ox, oy, oz) + ((ix, iy, iz) + 1/2) * dx, x fastest; index
 * i = (iz * ny + iy) * nx + ix.  sigma is shared by all Gaussians (the paper uses sigma = dx). */
typedef struct {
    int nx, ny, nz;
    float ox, oy, oz, dx;
    float sigma;
} gpair_grid;

/* A Gaussian set.  Two layouts:
 *  - grid-implicit: cx == NULL; `grid` (host pointer) gives centres and the shared sigma;
 *    M must equal nx*ny*nz; only A is read (device, [M]).
 *  - structure of arrays: cx, cy, cz, sigma, A are device float arrays of length M
 *    (free centres and per-Gaussian widths); `grid` is ignored. */
typedef struct {
    int64_t M;
    const float *cx, *cy, *cz, *sigma, *A;
    const gpair_grid* grid;
} gpair_gaussians;

/* Sensor array and acquisition (Methods: detector positions s_j, speed of sound v, sampling
 * rate f_s, N_t samples).  xyz is device memory [n_sensors][3]. */
typedef struct {
    int n_sensors;
    const float* xyz;
    float sound_speed;   /* v, m/s, > 0 */
    float fs;            /* Hz, > 0 */
    float t0;            /* time of sample 0, s (default 0) */
    int n_samples;       /* N_t >= 1 */
    float window_k;      /* k of the |d| <= k sigma window, > 0 (paper: 3) */
} gpair_array;

/* ----------------------------------------------------------------------------------------
 * gpair_forward -- the forward operator y = A(x) (Eq. single_forward summed over all
 * Gaussians; Methods, the direct pair enumeration):
 *     y[j][n] = sum_i A_i / (2 R_ij) * d * exp(-d^2 / 2 sigma_i^2),  d = R_ij - v t_n,
 * over |d| <= k sigma_i, R_ij = |c_i - s_j|, 0 <= n < N_t.
 * y: device [n_sensors][n_samples] float32, fully overwritten.
 * Returns INVALID_ARG for NULL/empty/inconsistent inputs; the call is asynchronous.
 * Accuracy: FP32 arithmetic with the phase R - v t_n referenced to an FP64 per-(tile, sensor)
 * origin; relative L2 error against the FP64 definition ~1e-6 (tested to 1e-5). */
gpair_status gpair_forward(const gpair_gaussians* g, const gpair_array* arr, float* y, void* stream);

/* ----------------------------------------------------------------------------------------
 * gpair_forward_noalloc -- gpair_forward for callers that cannot allocate device memory while
 * they run.  The paper has no counterpart; this is an interface convenience.
 * Some callers own all device memory through their own arena (a host framework that embeds the
 * reconstruction) or reserve their memory up front and must not stall or fail on a driver
 * allocation mid-run (a real-time acquisition loop).  gpair_forward grows a per-stream scratch
 * pool with cudaMalloc; this entry point instead uses one fixed 64 MiB device array that the
 * library declares at file scope, so it calls no cudaMalloc, cudaFree or allocating routine.
 * Every device that loads the library holds those 64 MiB until the process exits.
 * Same arguments, result and accuracy as gpair_forward (the slab partition may be coarser so
 * that the scratch fits).  Returns GPAIR_ERR_TOO_LARGE, launching nothing, when the problem
 * does not fit the array (the 256^3-class grid with 1024 sensors x 4096 samples fits).
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before capturing any stream.  All calls share the one array and it keeps
 * the last call's contents: calls that overlap on the GPU (different streams, or several host
 * threads) race and corrupt each other -- serialise them.  If a device-side bounded wait runs
 * out, y is filled with NaN. */
gpair_status gpair_forward_noalloc(const gpair_gaussians* g, const gpair_array* arr, float* y, void* stream);

/* ----------------------------------------------------------------------------------------
 * gpair_adjoint -- the exact transpose of gpair_forward (Methods, adjoint operator: the
 * back-projection of a detector residual delta), plus the closed-form parameter gradients of
 * L = sum_{j,n} delta[j][n] y[j][n]:
 *     gA[i]     = sum_{j,n} delta_j[n] * d e / (2R)
 *     gc[a][i]  = sum_{j,n} delta_j[n] * dp/dR * (c_i,a - s_j,a) / R,
 *                 dp/dR = -p/R + A/(2R) (1 - d^2/sigma^2) e
 *     gsigma[i] = sum_{j,n} delta_j[n] * A/(2R) * d^3/sigma^3 * e
 * with e = exp(-d^2/2sigma^2) and the window held fixed.  delta: device [n_sensors][n_samples].
 * gA: device [M] (required); gc: device [3][M] planar (x, y, z rows) or NULL; gsigma: device
 * [M] or NULL.  Outputs are overwritten.  Per-Gaussian sums over sensors use Kahan
 * compensation; no global atomics. */
gpair_status gpair_adjoint(const gpair_gaussians* g, const gpair_array* arr, const float* delta,
                           float* gA, float* gc, float* gsigma, void* stream);

/* ----------------------------------------------------------------------------------------
 * The operator partitioned over Gaussians (z-slabs of a grid-implicit set), for running it on
 * several GPUs.  Eq. single_forward is a sum over Gaussians, so the signals split into
 * per-slab partial signals that add up to y (one all-reduce per forward), and the adjoint of
 * each Gaussian depends only on the residual, so each slab's amplitude gradient is computed
 * without communication.  Shard s of n owns the lattice rows iz in [z_begin, z_end): the rows
 * are dealt out in order, the first nz % n shards taking one row more.
 *
 * gpair_shard_range: that row range (host arithmetic only; no device is touched).
 * INVALID_ARG for a NULL pointer, n_shards < 1 or shard outside [0, n_shards); a shard may own
 * no rows (z_begin == z_end) when n_shards > nz. */
gpair_status gpair_shard_range(const gpair_grid* grid, int shard, int n_shards, int* z_begin, int* z_end);

/* gpair_forward_shard: the forward operator of the shard's Gaussians only,
 *     y_s[j][n] = sum over i with iz(i) in [z_begin, z_end) of the terms of gpair_forward,
 * so that sum_s y_s = y.  g must be grid-implicit and describe the WHOLE lattice (A: device
 * [M], of which only the shard's rows are read).  y: device [n_sensors][n_samples], overwritten
 * (zeros when the shard owns no rows).  Same accuracy as gpair_forward; UNSUPPORTED for a
 * free-centre set. */
gpair_status gpair_forward_shard(const gpair_gaussians* g, const gpair_array* arr, int shard, int n_shards,
                                 float* y, void* stream);

/* gpair_adjoint_shard: the amplitude gradient (gpair_adjoint's gA) of the shard's Gaussians:
 * gA[i] for iz(i) in [z_begin, z_end) is overwritten, every other entry is left untouched.
 * gA: device [M].  delta: device [n_sensors][n_samples], the full residual. */
gpair_status gpair_adjoint_shard(const gpair_gaussians* g, const gpair_array* arr, int shard, int n_shards,
                                 const float* delta, float* gA, void* stream);

/* ----------------------------------------------------------------------------------------
 * gpair_voxelize -- Eq. (2) sampled on a voxel grid (Methods, the continuous source field):
 *     V[v] = sum_i A_i prod_a [|r_a - c_a| <= k sigma_i] exp(-(r_a - c_a)^2 / 2 sigma_i^2)
 * at voxel centres of out_grid (host pointer; its sigma field is ignored), box-truncated at
 * k sigma_i per axis with k = window_k.  vol: device [nz][ny][nx] float32, overwritten.
 * Grid-implicit Gaussians on the same lattice use three separable 1-D passes; any other set
 * uses a cell-binned gather. */
gpair_status gpair_voxelize(const gpair_gaussians* g, const gpair_grid* out_grid, float window_k,
                            float* vol, void* stream);

/* ----------------------------------------------------------------------------------------
 * Reconstruction step (Algorithm 2: NPC, forward, loss, adjoint, chain rule, CAWR, Adam). */
typedef enum { GPAIR_RULE_ADAM = 0, GPAIR_RULE_GD_LINESEARCH = 1 } gpair_rule;

typedef struct {
    int rule;            /* gpair_rule */
    int npc;             /* 1: x = (z + npc_eps)^2 (Methods, nonnegative parameterisation) */
    float npc_eps;       /* paper: 1e-8 */
    float eta_max, eta_min;  /* CAWR learning-rate range */
    int T0;              /* first restart period (iterations) */
    float T_mult;        /* period multiplier (>= 1) */
    float beta1, beta2, adam_eps;
    /* Vessel continuity regulariser (Methods: loss = data + lambda (R_H + beta R_TV), Algorithm 2);
     * vcr_lambda = 0 disables it.  Grid Gaussians and the Adam rule only; see gpair_vcr. */
    float vcr_lambda, vcr_beta, vcr_eps;
    /* Operator of every forward and adjoint in the step: 0 = the windowed closed form of
     * gpair_forward / gpair_adjoint (the default); 1 = the paper's discretised operator with
     * adaptive supersampling alignment (Algorithm 1, gpair_assa_forward / gpair_assa_adjoint;
     * grid Gaussians only) at the minimum pulse length n_min (the paper's is 25; ignored for 0). */
    int op, n_min;
} gpair_step_params;

typedef struct gpair_solver gpair_solver;

/* Create a solver for amplitudes only: centres/widths come from g (grid or SoA; the SoA arrays
 * must stay valid while the solver lives); g->A is ignored.  The solver owns z, Adam m and v
 * (zero-initialised, Algorithm 2 step 1), the iteration counter and workspace (y, residual,
 * gradient, FP64 reduction scratch).  Allocates device memory on the current device. */
gpair_status gpair_solver_create(const gpair_gaussians* g, const gpair_array* arr,
                                 const gpair_step_params* params, gpair_solver** out);
void gpair_solver_destroy(gpair_solver* s);

/* One iteration of Algorithm 2 with the exact data-term gradient 2 (y - b) / N, N = Nd Nt, plus
 * lambda grad R_VCR(x) when vcr_lambda > 0.  b: device [n_sensors][n_samples].  loss_out /
 * resid_out (host, may be NULL) receive the FP64 loss |y - b|^2 / N + lambda R_VCR(x) and
 * |y - b| of the iterate entering the step; when either is non-NULL the call synchronises
 * `stream`.  The reductions are done in FP64 on the GPU. */
gpair_status gpair_step(gpair_solver* s, const float* b, double* loss_out, double* resid_out,
                        void* stream);

/* n iterations of gpair_step on the same data b (device [n_sensors][n_samples]), replayed as one
 * CUDA graph: the step's launches are captured once per (solver, b) on a private stream and the
 * graph is launched n times on `stream`.  The per-step scalars (CAWR step size, Adam's bias
 * corrections) live on the device, so every step's launches are identical: the same kernels with
 * the same arguments as n gpair_step calls.  loss_out / resid_out (host, may be NULL) receive the values of the
 * iterate entering the last step (the call then synchronises `stream`).  With profiling enabled
 * the steps run one by one through gpair_step.  GPAIR_ERR_INVALID_ARG for NULL s or b, or n < 0. */
gpair_status gpair_solver_steps(gpair_solver* s, const float* b, int n, double* loss_out, double* resid_out,
                                void* stream);

/* Current image x = phi(z) (device [M] float32, written asynchronously). */
gpair_status gpair_solver_image(gpair_solver* s, float* x_out, void* stream);
/* Latent z, Adam moments m, v (device [M] each, any may be NULL) and the iteration count:
 * copies out (get) or in (set), for checkpoint / resume.  set with z != NULL also allows a
 * warm start. */
gpair_status gpair_solver_get_state(gpair_solver* s, float* z, float* m, float* v, int* t, void* stream);
gpair_status gpair_solver_set_state(gpair_solver* s, const float* z, const float* m, const float* v,
                                    int t, void* stream);

/* Device-side timing of gpair_step (tracing).  enable != 0: every following step records CUDA
 * events on its own stream around the forward slab kernel (ASSA: the band kernel), the adjoint
 * kernel (ASSA: the gather kernel) and the whole step.  gpair_solver_timings synchronises on the last recorded event, writes the summed
 * milliseconds ms[0] = forward slab kernel, ms[1] = adjoint kernel, ms[2] = whole step and the
 * number of recorded steps (may be NULL), and clears the record. */
gpair_status gpair_solver_profile(gpair_solver* s, int enable);
gpair_status gpair_solver_timings(gpair_solver* s, double* ms /*[3]*/, int* nsteps);

/* ----------------------------------------------------------------------------------------
 * FP64 reductions on the device (used by the step and exported for tests):
 * out[0] = sum (a - b)^2, out[1] = sum a*b'  where b' = c (dot with a third vector; c may be
 * NULL then out[1] = 0).  a, b, c: device float [n]; out: device double [2]. */
gpair_status gpair_reduce_f64(const float* a, const float* b, const float* c, int64_t n,
                              double* out, void* stream);

/* Misc. */
const char* gpair_status_string(gpair_status s);
/* Reads and clears the device status word of `stream` (synchronises that stream). */
gpair_status gpair_last_device_status(void* stream);
/* Frees the scratch pool of every stream on the current device. */
void gpair_release_scratch(void);

/* gpair_vcr -- the vessel continuity regulariser (Methods, vessel continuity regularisation):
 * R_VCR(x) = sum_i sqrt(sum_{p,q} (D_pq x)_i^2 + eps) + beta sum_i sqrt(sum_d (D_d x)_i^2 + eps) for a
 * lattice image x (device, [nz][ny][nx], x fastest).  The paper leaves the operators open; here
 * D_d is the central first difference (x[i+1] - x[i-1]) / 2, D_pp = x[i+1] - 2 x[i] + x[i-1], D_pq
 * (p != q) the four-point central mixed difference / 4 (counted for (p,q) and (q,p)), with Neumann
 * boundaries (neighbour indices clamped) and unit voxel spacing.  value_out (host, may be NULL):
 * R_VCR in FP64 (the call then synchronises `stream`); grad (device [M], may be NULL):
 * grad += lam * dR_VCR/dx.  One fused pass: the difference fields stay in shared memory, so only x
 * and grad cross device memory; scratch is a few KB of FP64 block partials from the library's
 * per-stream pool.  Errors:
 * GPAIR_ERR_INVALID_ARG for a NULL x, non-positive sizes or eps < 0; GPAIR_ERR_UNSUPPORTED when
 * ny nz >= 2^31. */
gpair_status gpair_vcr(const float* x, int nx, int ny, int nz, float beta, float eps, float lam, float* grad,
                       double* value_out, void* stream);

/* ---- The paper's own discretised operator (Methods, adaptive supersampling alignment;
 * Algorithm 1), for grid Gaussians sharing one width sigma.
 *
 * Grid: N_half = ceil(3 sigma / (v / fs)), alpha = max(1, ceil(((n_min - 1) / 2) / N_half)) (the
 * paper uses n_min = 25), K = alpha N_half; evaluated in double from the given float arguments.
 * Forward: each pair's time of flight is snapped to the fine sample
 * k_ij = floor((r_ij / v - t0) alpha fs + 1/2), its mass A_i / r_ij accumulates there when
 * 0 <= k_ij < alpha N_t, the impulse line is convolved with h[k] = (1/2) d exp(-d^2 / 2 sigma^2),
 * d = -v k / (alpha fs), |k| <= K, and decimated: y_j[n] = sum_i (A_i / r_ij) h[alpha n - k_ij].
 * arr->window_k is not used (the pulse support is the paper's 3-sigma rule, N_half samples).
 * Adjoint: gA_i = sum_j (1 / r_ij) sum_n h[alpha n - k_ij] delta_j[n], the exact transpose.
 * Layouts as gpair_forward / gpair_adjoint; gA has M entries.  Errors: GPAIR_ERR_UNSUPPORTED for
 * free-centre Gaussians, K > 256, alpha N_t >= 2^30 or N_d alpha N_t >= 2^31; GPAIR_ERR_INVALID_ARG for n_min < 1 or
 * NULL buffers.  Asynchronous on `stream`; scratch from the library's per-stream pool (the
 * adjoint's correlated residual: N_d alpha N_t floats). */
gpair_status gpair_assa_forward(const gpair_gaussians* g, const gpair_array* arr, int n_min, float* y, void* stream);
gpair_status gpair_assa_adjoint(const gpair_gaussians* g, const gpair_array* arr, int n_min, const float* delta,
                                float* gA, void* stream);

/* ---- Image metrics of reconstructions (Results, Table 1: PSNR, SSIM, MSE on the volume and on its
 * maximum amplitude projection along z).  The paper gives no formulas; these follow the common
 * definitions.
 *
 * gpair_zmap: out[y][x] = max_z vol[z][y][x] (device, vol [nz][ny][nx], out [ny][nx]).
 * gpair_image_metrics: x and ref (device, [nz][ny][nx], nz = 1 for an image) -> out (host, 3
 * doubles): MSE, PSNR = 10 log10(data_range^2 / MSE) and the mean SSIM (Wang et al., 2004) with a
 * uniform window of `win` samples per axis (odd, >= 3), sample (N / (N - 1)) variances and
 * covariance, C1 = (0.01 data_range)^2, C2 = (0.03 data_range)^2, over the positions whose window
 * lies inside; FP64 sums.  Synchronises `stream`; scratch 10 M floats from the per-stream pool.
 * Errors: GPAIR_ERR_INVALID_ARG for NULL pointers, even or < 3 win, data_range <= 0;
 * GPAIR_ERR_UNSUPPORTED when an axis (z only if nz > 1) is shorter than win. */
gpair_status gpair_zmap(const float* vol, int nx, int ny, int nz, float* out, void* stream);
gpair_status gpair_image_metrics(const float* x, const float* ref, int nx, int ny, int nz, int win, float data_range,
                                 double* out, void* stream);

/* gpair_wait_selftest -- exercises the failure-detection path of the bounded waits.  Launches one
 * warp that waits on a shared-memory barrier nothing completes, giving up after `polls` polls
 * (1 <= polls <= 2^20, else GPAIR_ERR_INVALID_ARG, nothing launched); the kernel records a timeout
 * in the stream's device status word and returns normally, leaving the context usable.  The next
 * gpair_last_device_status(stream) returns GPAIR_ERR_TIMEOUT.  The paper has no counterpart. */
gpair_status gpair_wait_selftest(int polls, void* stream);

/* gpair_pipe_peak -- measured throughput of a pipe that bounds the operators, for their roofline
 * (the operators are FP32/MUFU instruction work, not a contraction and not HBM traffic).
 * pipe GPAIR_PIPE_FP32: fused multiply-adds (fmaf), GPAIR_PIPE_MUFU: ex2.approx; each thread runs
 * 8 independent dependency chains, 8 CTAs of 256 threads per SM.  One warm-up launch, then `reps`
 * (1..1000) launches timed with CUDA events on `stream`; writes lane operations per second to
 * *lane_ops_per_s (host).  Synchronises `stream`; allocates and frees a small device buffer.
 * Errors: GPAIR_ERR_INVALID_ARG for an unknown pipe, reps outside 1..1000 or a NULL output. */
typedef enum { GPAIR_PIPE_FP32 = 0, GPAIR_PIPE_MUFU = 1 } gpair_pipe;
gpair_status gpair_pipe_peak(int pipe, int reps, double* lane_ops_per_s, void* stream);
/* Library version string. */
const char* gpair_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GPAIR_H */
