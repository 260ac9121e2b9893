/*
 * gpair_oracle.c -- plain FP64 CPU oracle for the GPAIR forward/adjoint hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that the
 * CUDA path is checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load it.  It shares no code, header, table or constant
 * with the CUDA library; every function restates the paper's mathematics directly.
 *
 * Paper: "GPAIR: Gaussian-Kernel-Based Ultrafast 3D Photoacoustic Iterative Reconstruction"
 * (arXiv 2602.03893), Methods section.
 *
 * Conventions (SI units throughout): a Gaussian i has centre c_i (m), width sigma_i (m) and
 * amplitude A_i; a sensor j sits at s_j (m); v is the speed of sound (m/s); sample n of every
 * sensor is taken at t_n = t0 + n / fs (s).  Signals are stored sensor-major, y[j*Nt + n].
 *
 * Pinning status (see tests/test_oracle_pins.py):
 *   ora_sphere_integral      pinned: 2-D quadrature of the surface integral I.
 *   ora_pressure_exact       pinned: spherical-means quadrature + d'Alembert invariants.
 *   ora_pressure_outgoing    pinned: equals ora_pressure_exact minus the incoming term; far field.
 *   ora_forward              pinned: brute-force spherical-means quadrature of the summed field,
 *                                    window-tail bound, single-Gaussian window count.
 *   ora_adjoint              pinned: adjoint identity <Fx,y>=<x,F^T y>; central FD for c, sigma.
 *   ora_voxelize             pinned: separable numpy convolution (grid case), brute force.
 *   ora_adam_cawr / ora_ir   pinned: torch.optim.Adam + CosineAnnealingWarmRestarts on a dense
 *                                    operator built column by column from ora_forward.
 *   ora_assa_forward/adjoint pinned: adjoint identity; the folded single-sum form; equality with
 *                                    the windowed forward where every time of flight lies on the
 *                                    upsampled grid; convergence to it as N_min grows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

void ora_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int ora_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. (sphere_int): closed form of the surface integral of one Gaussian
 * A exp(-|r - r'|^2 / 2 sigma^2) over the sphere of radius rp centred at the detector,
 * where r is the detector-to-centre distance:
 *   I = A * 2 pi sigma^2 * rp / r * (exp(-(r-rp)^2/2s^2) - exp(-(r+rp)^2/2s^2)). */
double ora_sphere_integral(double A, double sigma, double r, double rp) {
    double s2 = 2.0 * sigma * sigma;
    return A * 2.0 * ORA_PI * sigma * sigma * rp / r *
           (exp(-(r - rp) * (r - rp) / s2) - exp(-(r + rp) * (r + rp) / s2));
}

/* Methods, the two-term pressure obtained by substituting Eq. (sphere_int) into
 * Eq. (pa_wave): p = A/(2r) [ (r - vt) e^{-(r-vt)^2/2s^2} + (r + vt) e^{-(r+vt)^2/2s^2} ]. */
double ora_pressure_exact(double A, double sigma, double r, double t, double v) {
    double s2 = 2.0 * sigma * sigma;
    double dm = r - v * t, dp = r + v * t;
    return A / (2.0 * r) * (dm * exp(-dm * dm / s2) + dp * exp(-dp * dp / s2));
}

/* Eq. (single_forward): outgoing term only, p = A/(2r) d e^{-d^2/2 s^2}, d = r - v t. */
double ora_pressure_outgoing(double A, double sigma, double r, double t, double v) {
    double d = r - v * t;
    return A / (2.0 * r) * d * exp(-d * d / (2.0 * sigma * sigma));
}

/* Forward operator: y_j[n] = sum_i p_i(|c_i - s_j|, t_n).
 *  mode 0 ("windowed", the operator the reconstruction uses): Eq. (single_forward), kept only
 *         where |d| <= k sigma_i (Methods, the 3-sigma principle; inclusive bound, k a parameter).
 *  mode 1 ("exact"): both terms of the two-term pressure at every sample, no window.
 * amb (optional, mode 0): for every sample, the sum of |p| over the (i, j, n) terms whose
 * window decision is ambiguous at tolerance tau, i.e. ||d| - k sigma_i| < tau.  A
 * single-precision implementation may legitimately decide those terms either way. */
void ora_forward(int64_t M, const double* cx, const double* cy, const double* cz,
                 const double* sg, const double* A,
                 int Nd, const double* sxyz, double v, double fs, double t0, int Nt,
                 double k, int mode, double tau, double* y, double* amb) {
    memset(y, 0, sizeof(double) * (size_t)Nd * (size_t)Nt);
    if (amb) memset(amb, 0, sizeof(double) * (size_t)Nd * (size_t)Nt);
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < Nd; ++j) {
        double* yj = y + (size_t)j * Nt;
        double* aj = amb ? amb + (size_t)j * Nt : NULL;
        double sx = sxyz[3 * j], sy = sxyz[3 * j + 1], sz = sxyz[3 * j + 2];
        for (int64_t i = 0; i < M; ++i) {
            if (A[i] == 0.0) continue;
            double dx = cx[i] - sx, dy = cy[i] - sy, dz = cz[i] - sz;
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (mode == 1) {
                for (int n = 0; n < Nt; ++n)
                    yj[n] += ora_pressure_exact(A[i], sg[i], r, t0 + n / fs, v);
                continue;
            }
            /* Samples outside [n_a, n_b] have |d| > k sigma by a margin of two samples; every
             * candidate inside is still tested against the window definition itself. */
            double half = k * sg[i];
            long n_a = (long)floor(((r - half) / v - t0) * fs) - 2;
            long n_b = (long)ceil(((r + half) / v - t0) * fs) + 2;
            if (n_a < 0) n_a = 0;
            if (n_b > Nt - 1) n_b = Nt - 1;
            for (long n = n_a; n <= n_b; ++n) {
                double t = t0 + (double)n / fs;
                double d = r - v * t;
                double p = ora_pressure_outgoing(A[i], sg[i], r, t, v);
                if (fabs(d) <= half) yj[n] += p;
                if (aj && fabs(fabs(d) - half) < tau) aj[n] += fabs(p);
            }
        }
    }
}

/* Adjoint (exact transpose of mode 0 of ora_forward) and the closed-form parameter
 * derivatives of Eq. (single_forward):
 *   dp/dA     = d e / (2r)
 *   dp/dr     = -p / r + A/(2r) (1 - d^2/sigma^2) e        (d = r - v t, so dd/dr = 1)
 *   dr/dc     = (c - s) / r
 *   dp/dsigma = A/(2r) d (d^2 / sigma^3) e
 * with e = exp(-d^2 / 2 sigma^2).  The window |d| <= k sigma is held fixed (derivative almost
 * everywhere).  Outputs: gA[i] = sum_{j,n} delta_j[n] dp/dA; gc{x,y,z}[i] likewise for the
 * centre; gs[i] for sigma.  Any output pointer may be NULL.  ambA/ambC/ambS (optional) collect
 * |delta * dp/d.| over window-ambiguous terms (as in ora_forward); ambC sums the three axes. */
void ora_adjoint(int64_t M, const double* cx, const double* cy, const double* cz,
                 const double* sg, const double* A,
                 int Nd, const double* sxyz, double v, double fs, double t0, int Nt,
                 double k, const double* delta, double tau,
                 double* gA, double* gcx, double* gcy, double* gcz, double* gs,
                 double* ambA, double* ambC, double* ambS) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < M; ++i) {
        double aA = 0, ax = 0, ay = 0, az = 0, as = 0;
        double bA = 0, bC = 0, bS = 0;
        double s = sg[i], half = k * s;
        for (int j = 0; j < Nd; ++j) {
            const double* dj = delta + (size_t)j * Nt;
            double dx = cx[i] - sxyz[3 * j], dy = cy[i] - sxyz[3 * j + 1], dz = cz[i] - sxyz[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            long n_a = (long)floor(((r - half) / v - t0) * fs) - 2;
            long n_b = (long)ceil(((r + half) / v - t0) * fs) + 2;
            if (n_a < 0) n_a = 0;
            if (n_b > Nt - 1) n_b = Nt - 1;
            for (long n = n_a; n <= n_b; ++n) {
                double t = t0 + (double)n / fs;
                double d = r - v * t;
                int in = fabs(d) <= half;
                int ambig = fabs(fabs(d) - half) < tau;
                if (!in && !ambig) continue;
                double e = exp(-d * d / (2.0 * s * s));
                double dpdA = d * e / (2.0 * r);
                double p = A[i] * dpdA;
                double dpdr = -p / r + A[i] / (2.0 * r) * (1.0 - d * d / (s * s)) * e;
                double dpds = A[i] / (2.0 * r) * d * (d * d / (s * s * s)) * e;
                double w = dj[n];
                if (in) {
                    aA += w * dpdA;
                    ax += w * dpdr * dx / r;
                    ay += w * dpdr * dy / r;
                    az += w * dpdr * dz / r;
                    as += w * dpds;
                }
                if (ambig) {
                    bA += fabs(w * dpdA);
                    bC += fabs(w * dpdr * dx / r) + fabs(w * dpdr * dy / r) + fabs(w * dpdr * dz / r);
                    bS += fabs(w * dpds);
                }
            }
        }
        if (gA) gA[i] = aA;
        if (gcx) gcx[i] = ax;
        if (gcy) gcy[i] = ay;
        if (gcz) gcz[i] = az;
        if (gs) gs[i] = as;
        if (ambA) ambA[i] = bA;
        if (ambC) ambC[i] = bC;
        if (ambS) ambS[i] = bS;
    }
}

/* Voxelisation: Eq. (2) sampled at voxel centres o + (idx + 1/2) h of an (nx, ny, nz) grid,
 * x fastest, with every Gaussian truncated to the box |r_a - c_a| <= k sigma_i on each axis a:
 *   V[v] = sum_i A_i prod_a [|r_a - c_a| <= k s_i] exp(-(r_a - c_a)^2 / 2 s_i^2). */
void ora_voxelize(int64_t M, const double* cx, const double* cy, const double* cz,
                  const double* sg, const double* A, double k,
                  int nx, int ny, int nz, double ox, double oy, double oz, double h, double* vol) {
    size_t nvox = (size_t)nx * ny * nz;
    memset(vol, 0, sizeof(double) * nvox);
    /* One Gaussian at a time; each touches a small box of voxels.  Serial over i so the
     * accumulation order is fixed. */
    for (int64_t i = 0; i < M; ++i) {
        if (A[i] == 0.0) continue;
        /* The box edge is inclusive; a relative 1e-12 slack keeps lattice ties (|m h| == k s
         * exactly in real arithmetic) inside despite double rounding of the centre differences. */
        double half = k * sg[i] * (1.0 + 1e-12), s2 = 2.0 * sg[i] * sg[i];
        long xa = (long)floor((cx[i] - half - ox) / h - 0.5) - 1, xb = (long)ceil((cx[i] + half - ox) / h - 0.5) + 1;
        long ya = (long)floor((cy[i] - half - oy) / h - 0.5) - 1, yb = (long)ceil((cy[i] + half - oy) / h - 0.5) + 1;
        long za = (long)floor((cz[i] - half - oz) / h - 0.5) - 1, zb = (long)ceil((cz[i] + half - oz) / h - 0.5) + 1;
        if (xa < 0) xa = 0;
        if (ya < 0) ya = 0;
        if (za < 0) za = 0;
        if (xb > nx - 1) xb = nx - 1;
        if (yb > ny - 1) yb = ny - 1;
        if (zb > nz - 1) zb = nz - 1;
        for (long iz = za; iz <= zb; ++iz) {
            double rz = oz + (iz + 0.5) * h - cz[i];
            if (fabs(rz) > half) continue;
            for (long iy = ya; iy <= yb; ++iy) {
                double ry = oy + (iy + 0.5) * h - cy[i];
                if (fabs(ry) > half) continue;
                for (long ix = xa; ix <= xb; ++ix) {
                    double rx = ox + (ix + 0.5) * h - cx[i];
                    if (fabs(rx) > half) continue;
                    vol[((size_t)iz * ny + iy) * nx + ix] +=
                        A[i] * exp(-rx * rx / s2) * exp(-ry * ry / s2) * exp(-rz * rz / s2);
                }
            }
        }
    }
}

/* ---------------------------------------------------------------------------------------
 * ASSA: the paper's discretised operator (Methods, adaptive supersampling alignment;
 * Algorithm 1), for Gaussians sharing one width sigma.
 *
 * Grid parameters (Methods, adaptive grid parameters): the kernel half-width in original samples
 * N_half = ceil(3 sigma / (v dt)), dt = 1 / fs; the upsampling ratio
 * alpha = max(1, ceil(((N_min - 1) / 2) / N_half)); the upsampled kernel half-width K = alpha N_half.
 * Evaluated in double from the arguments as given. */
void ora_assa_params(double sigma, double v, double fs, int n_min, int* n_half, int* alpha, int* K) {
    int nh = (int)ceil(3.0 * sigma / (v / fs));
    if (nh < 1) nh = 1;
    int a = (int)ceil(((double)(n_min - 1) / 2.0) / (double)nh);
    if (a < 1) a = 1;
    *n_half = nh;
    *alpha = a;
    *K = a * nh;
}

/* The kernel h[k], k = -K..K, stored at h[k + K]: C d exp(-d^2 / 2 sigma^2) with
 * d = -v k dt_up and C = 1/2 (the 1/(2r) factor of Eq. single_forward, split as 1/r in the
 * projection times C in the kernel). */
static void assa_kernel(double sigma, double v, double fs_up, int K, double* h) {
    for (int k = -K; k <= K; ++k) {
        double d = -v * (double)k / fs_up;
        h[k + K] = 0.5 * d * exp(-d * d / (2.0 * sigma * sigma));
    }
}

/* Snapped index of a pair on the upsampled grid (sample 0 at t0):
 * k = floor((r / v - t0) fs_up + 1/2).  *tie is set when the rounding is within tau (in
 * upsampled samples) of the other choice; *k_alt is that other choice. */
static long assa_snap(double r, double v, double t0, double fs_up, double tau, int* tie, long* k_alt) {
    double u = (r / v - t0) * fs_up + 0.5;
    double f = floor(u);
    long k = (long)f;
    *tie = 0;
    *k_alt = k;
    if (u - f < tau) { *tie = 1; *k_alt = k - 1; }
    else if (f + 1.0 - u < tau) { *tie = 1; *k_alt = k + 1; }
    return k;
}

/* Forward, the paper's three stages per detector j:
 *   1. projection:   z_j[k] = sum_i (x_i / r_ij) [k == k_ij],  k = 0..alpha Nt - 1
 *   2. transposed convolution:  zt_j[k] = sum_m z_j[m] h[k - m]
 *   3. decimation:   y_j[n] = zt_j[alpha n].
 * Impulses snapped outside 0..alpha Nt - 1 are not in z (the sequence has that length).
 * amb (optional): for pairs whose snap is within tau of a tie, |x_i / r_ij| times the change of
 * their decimated contribution under the other choice, per sample. */
void ora_assa_forward(int64_t M, const double* cx, const double* cy, const double* cz, const double* A,
                      double sigma, int Nd, const double* sxyz, double v, double fs, double t0, int Nt,
                      int n_min, double tau, double* y, double* amb) {
    int nh, alpha, K;
    ora_assa_params(sigma, v, fs, n_min, &nh, &alpha, &K);
    const double fs_up = alpha * fs;
    const long Nup = (long)alpha * Nt;
    double* h = (double*)malloc(sizeof(double) * (size_t)(2 * K + 1));
    assa_kernel(sigma, v, fs_up, K, h);
    memset(y, 0, sizeof(double) * (size_t)Nd * (size_t)Nt);
    if (amb) memset(amb, 0, sizeof(double) * (size_t)Nd * (size_t)Nt);
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < Nd; ++j) {
        double* z = (double*)calloc((size_t)Nup, sizeof(double));
        double* zt = (double*)calloc((size_t)Nup, sizeof(double));
        double sx = sxyz[3 * j], sy = sxyz[3 * j + 1], sz = sxyz[3 * j + 2];
        double* yj = y + (size_t)j * Nt;
        double* aj = amb ? amb + (size_t)j * Nt : NULL;
        for (int64_t i = 0; i < M; ++i) {
            if (A[i] == 0.0) continue;
            double dx = cx[i] - sx, dy = cy[i] - sy, dz = cz[i] - sz;
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            int tie;
            long k_alt;
            long k = assa_snap(r, v, t0, fs_up, tau, &tie, &k_alt);
            if (k >= 0 && k < Nup) z[k] += A[i] / r;
            if (aj && tie) {
                /* the pair's decimated contribution under either choice (zero when outside) */
                for (long n = 0; n < Nt; ++n) {
                    long q1 = alpha * n - k, q2 = alpha * n - k_alt;
                    double c1 = (k >= 0 && k < Nup && q1 >= -K && q1 <= K) ? h[q1 + K] : 0.0;
                    double c2 = (k_alt >= 0 && k_alt < Nup && q2 >= -K && q2 <= K) ? h[q2 + K] : 0.0;
                    aj[n] += fabs(A[i] / r) * fabs(c1 - c2);
                }
            }
        }
        for (long k = 0; k < Nup; ++k) {
            double acc = 0.0;
            for (long m = k - K; m <= k + K; ++m)
                if (m >= 0 && m < Nup) acc += z[m] * h[k - m + K];
            zt[k] = acc;
        }
        for (int n = 0; n < Nt; ++n) yj[n] = zt[(long)alpha * n];
        free(z);
        free(zt);
    }
    free(h);
}

/* Adjoint, the transpose of each stage:
 *   1. zero filling: dup_j[k] = delta_j[k / alpha] when alpha divides k, else 0
 *   2. correlation with the flipped kernel: dconv_j[k] = sum_m h[m - k] dup_j[m]
 *   3. back-projection: g_i = sum_j dconv_j[k_ij] / r_ij  (pairs snapped inside the sequence).
 * amb (optional): per Gaussian, |dconv_j[k] - dconv_j[k_alt]| / r over pairs within tau of a tie. */
void ora_assa_adjoint(int64_t M, const double* cx, const double* cy, const double* cz, double sigma,
                      int Nd, const double* sxyz, double v, double fs, double t0, int Nt, int n_min,
                      const double* delta, double tau, double* g, double* amb) {
    int nh, alpha, K;
    ora_assa_params(sigma, v, fs, n_min, &nh, &alpha, &K);
    const double fs_up = alpha * fs;
    const long Nup = (long)alpha * Nt;
    double* h = (double*)malloc(sizeof(double) * (size_t)(2 * K + 1));
    assa_kernel(sigma, v, fs_up, K, h);
    double* dconv = (double*)malloc(sizeof(double) * (size_t)Nd * (size_t)Nup);
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < Nd; ++j) {
        double* dup = (double*)calloc((size_t)Nup, sizeof(double));
        for (int n = 0; n < Nt; ++n) dup[(long)alpha * n] = delta[(size_t)j * Nt + n];
        double* dc = dconv + (size_t)j * Nup;
        for (long k = 0; k < Nup; ++k) {
            double acc = 0.0;
            for (long m = k - K; m <= k + K; ++m)
                if (m >= 0 && m < Nup) acc += h[m - k + K] * dup[m];
            dc[k] = acc;
        }
        free(dup);
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < M; ++i) {
        double acc = 0.0, ab = 0.0;
        for (int j = 0; j < Nd; ++j) {
            double dx = cx[i] - sxyz[3 * j], dy = cy[i] - sxyz[3 * j + 1], dz = cz[i] - sxyz[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            int tie;
            long k_alt;
            long k = assa_snap(r, v, t0, fs_up, tau, &tie, &k_alt);
            const double* dc = dconv + (size_t)j * Nup;
            double c1 = (k >= 0 && k < Nup) ? dc[k] : 0.0;
            acc += c1 / r;
            if (tie) {
                double c2 = (k_alt >= 0 && k_alt < Nup) ? dc[k_alt] : 0.0;
                ab += fabs(c1 - c2) / r;
            }
        }
        g[i] = acc;
        if (amb) amb[i] = ab;
    }
    free(dconv);
    free(h);
}

/* Cosine annealing with warm restarts (Methods, learning-rate schedule; SGDR semantics):
 * periods T_0, T_0 T_mult, T_0 T_mult^2, ...; T_cur counts iterations since the last restart. */
double ora_cawr(int t, double eta_max, double eta_min, int T0, double Tmult) {
    double Tcur = t, Ti = T0;
    while (Tcur >= Ti) {
        Tcur -= Ti;
        Ti *= Tmult;
        if (Tmult == 1.0) { Tcur = fmod(Tcur, Ti); break; }
    }
    return eta_min + 0.5 * (eta_max - eta_min) * (1.0 + cos(ORA_PI * Tcur / Ti));
}

/* One Adam update (Kingma & Ba) of z with gradient g, step count t >= 1:
 *   m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
 *   z <- z - eta * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void ora_adam(int64_t M, double* z, double* m, double* vv, const double* g, int t,
              double eta, double b1, double b2, double eps) {
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t i = 0; i < M; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        vv[i] = b2 * vv[i] + (1.0 - b2) * g[i] * g[i];
        z[i] -= eta * (m[i] / c1) / (sqrt(vv[i] / c2) + eps);
    }
}

/* Algorithm 2 (GPAIR loop), amplitudes only, with the forward/adjoint of mode 0 above.
 *   rule 0 (Adam): z0 = 0; per iteration t = 0..iters-1:
 *       x = (z + eps)^2 if npc else z;  y = F x;  L = |y - b|^2 / N  (N = Nd Nt);
 *       grad_y = 2 (y - b) / N  (the exact gradient of L);  grad_x = F^T grad_y;
 *       grad_z = grad_x * 2 (z + eps) if npc else grad_x;  eta_t = CAWR(t);  Adam(z).
 *       Returns x* = (z + eps)^2 (or z).
 *   rule 1 (steepest descent with exact line search on x, no NPC): g = F^T (y - b),
 *       alpha = <y - b, F g> / |F g|^2,  x <- x - alpha g  (one extra forward per iteration).
 * loss[t] and resid[t] = |y - b| are recorded for the iterate entering iteration t. */
void ora_ir(int64_t M, const double* cx, const double* cy, const double* cz, const double* sg,
            int Nd, const double* sxyz, double v, double fs, double t0, int Nt, double k,
            const double* b, int iters, int rule, int npc, double npc_eps,
            double eta_max, double eta_min, int T0, double Tmult,
            double b1, double b2, double adam_eps,
            double* x_out, double* loss, double* resid) {
    size_t Ny = (size_t)Nd * Nt;
    double N = (double)Ny;
    double* z = calloc((size_t)M, sizeof(double));
    double* m = calloc((size_t)M, sizeof(double));
    double* vv = calloc((size_t)M, sizeof(double));
    double* x = calloc((size_t)M, sizeof(double));
    double* g = calloc((size_t)M, sizeof(double));
    double* y = calloc(Ny, sizeof(double));
    double* r = calloc(Ny, sizeof(double));
    double* Fg = rule == 1 ? calloc(Ny, sizeof(double)) : NULL;
    for (int t = 0; t < iters; ++t) {
        for (int64_t i = 0; i < M; ++i) x[i] = npc ? (z[i] + npc_eps) * (z[i] + npc_eps) : z[i];
        ora_forward(M, cx, cy, cz, sg, x, Nd, sxyz, v, fs, t0, Nt, k, 0, 0.0, y, NULL);
        double ss = 0.0;
        for (size_t q = 0; q < Ny; ++q) { double e = y[q] - b[q]; ss += e * e; }
        if (loss) loss[t] = ss / N;
        if (resid) resid[t] = sqrt(ss);
        if (rule == 0) {
            for (size_t q = 0; q < Ny; ++q) r[q] = 2.0 * (y[q] - b[q]) / N;
            ora_adjoint(M, cx, cy, cz, sg, x, Nd, sxyz, v, fs, t0, Nt, k, r, 0.0,
                        g, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
            if (npc) for (int64_t i = 0; i < M; ++i) g[i] *= 2.0 * (z[i] + npc_eps);
            double eta = ora_cawr(t, eta_max, eta_min, T0, Tmult);
            ora_adam(M, z, m, vv, g, t + 1, eta, b1, b2, adam_eps);
        } else {
            for (size_t q = 0; q < Ny; ++q) r[q] = y[q] - b[q];
            ora_adjoint(M, cx, cy, cz, sg, x, Nd, sxyz, v, fs, t0, Nt, k, r, 0.0,
                        g, NULL, NULL, NULL, NULL, NULL, NULL, NULL);
            ora_forward(M, cx, cy, cz, sg, g, Nd, sxyz, v, fs, t0, Nt, k, 0, 0.0, Fg, NULL);
            double num = 0.0, den = 0.0;
            for (size_t q = 0; q < Ny; ++q) { num += r[q] * Fg[q]; den += Fg[q] * Fg[q]; }
            double alpha = den > 0.0 ? num / den : 0.0;
            for (int64_t i = 0; i < M; ++i) z[i] -= alpha * g[i];
        }
    }
    for (int64_t i = 0; i < M; ++i)
        x_out[i] = (npc && rule == 0) ? (z[i] + npc_eps) * (z[i] + npc_eps) : z[i];
    free(z); free(m); free(vv); free(x); free(g); free(y); free(r); free(Fg);
}
