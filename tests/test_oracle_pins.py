"""Pins for the FP64 oracle (CPU only).

Each test checks the oracle against something other than itself: numerical quadrature of the
spherical-means solution (Methods, Eq. pa_wave / the surface integral I), the initial-value
problem the two-term pressure solves, brute force over every sample on tiny inputs, the
adjoint identity, central finite differences, numpy's convolution, and torch's Adam and
CosineAnnealingWarmRestarts.  A plausible slip in the oracle (a dropped term, a sign, an index,
a transposed operand) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_03893_gb300 import synth


# ---------------------------------------------------------------- quadrature helpers (test-only)

def _frame(axis):
    e3 = np.asarray(axis, float) / np.linalg.norm(axis)
    tmp = np.array([1.0, 0.0, 0.0]) if abs(e3[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(e3, tmp)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(e3, e1)
    return e1, e2, e3


def sphere_quadrature(f, centre, radius, axis=(0, 0, 1), theta_max=math.pi, n_theta=300, n_phi=300):
    """Integral of f over the sphere |x - centre| = radius: Gauss-Legendre in the polar angle on
    [0, theta_max] about `axis`, trapezoid rule in the azimuth (both generic, no symmetry)."""
    e1, e2, e3 = _frame(axis)
    xg, wg = np.polynomial.legendre.leggauss(n_theta)
    th = 0.5 * theta_max * (xg + 1.0)
    wth = 0.5 * theta_max * wg
    ph = np.arange(n_phi) * (2 * math.pi / n_phi)
    wph = 2 * math.pi / n_phi
    T, P = np.meshgrid(th, ph, indexing="ij")
    dirs = (np.sin(T)[..., None] * (np.cos(P)[..., None] * e1 + np.sin(P)[..., None] * e2)
            + np.cos(T)[..., None] * e3)
    X = np.asarray(centre, float) + radius * dirs
    W = (wth[:, None] * wph) * radius ** 2 * np.sin(T)
    return float(np.sum(W * f(X)))


def gaussian_field(centres, sigmas, amps):
    centres = np.atleast_2d(centres)

    def f(X):
        out = np.zeros(X.shape[:-1])
        for c, s, a in zip(centres, np.broadcast_to(sigmas, len(centres)), amps):
            out += a * np.exp(-np.sum((X - c) ** 2, -1) / (2 * s * s))
        return out
    return f


def d4(fun, t, h):
    """Fourth-order central difference of fun at t."""
    return (-fun(t + 2 * h) + 8 * fun(t + h) - 8 * fun(t - h) + fun(t - 2 * h)) / (12 * h)


# ---------------------------------------------------------------- Eq. (sphere_int)

@pytest.mark.parametrize("r,rp", [(1.0, 0.9), (1.0, 1.5), (1.0, 0.2), (2.0, 2.1)])
def test_sphere_integral_matches_quadrature(r, rp):
    A, sigma = 1.3, 0.3
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    det = np.array([0.1, 0.2, -0.3])
    c = det + r * u
    quad = sphere_quadrature(gaussian_field(c, sigma, [A]), det, rp, axis=(0, 0, 1),
                             n_theta=400, n_phi=400)
    closed = oracle.sphere_integral(A, sigma, r, rp)
    assert abs(closed - quad) <= 1e-10 * abs(quad)


# ---------------------------------------------------------------- two-term pressure (Methods)

@pytest.mark.parametrize("vt", [0.5, 0.9, 1.0, 1.2, 1.6])
def test_pressure_exact_matches_spherical_means(vt):
    """p = (1/4 pi v) d/dt[(1/vt) I], with I from quadrature (not from the closed form)."""
    A, sigma, r, v = 1.3, 0.3, 1.0, 1.5
    det = np.zeros(3)
    c = np.array([0.0, 0.6, 0.8]) * r
    field = gaussian_field(c, sigma, [A])

    def mean_term(t):
        return sphere_quadrature(field, det, v * t, axis=c, n_theta=300, n_phi=64) / (v * t)
    t = vt / v
    p_quad = d4(mean_term, t, 1e-3) / (4 * math.pi * v)
    p = oracle.pressure_exact(A, sigma, r, t, v)
    assert abs(p - p_quad) <= 1e-8 * A


def test_pressure_exact_initial_value_problem():
    """The two-term pressure solves the 3-D wave equation with p(.,0) the Gaussian and
    dp/dt(.,0) = 0 (the photoacoustic initial-value problem): check p(r,0), p_t(r,0) and
    that u = r p satisfies u_tt = v^2 u_rr (radial d'Alembert form)."""
    A, sigma, v = 0.7, 0.2, 1.5
    for r in [0.05, 0.3, 0.8, 2.0]:
        assert abs(oracle.pressure_exact(A, sigma, r, 0.0, v) - A * math.exp(-r * r / (2 * sigma ** 2))) < 1e-15
        pt = d4(lambda t: oracle.pressure_exact(A, sigma, r, t, v), 0.0, 1e-3)
        assert abs(pt) < 1e-10
    u = lambda r, t: r * oracle.pressure_exact(A, sigma, r, t, v)
    for r, t in [(0.5, 0.2), (1.0, 0.5), (0.7, 0.45), (1.3, 0.9)]:
        h = 1e-3
        utt = (-u(r, t + 2 * h) + 16 * u(r, t + h) - 30 * u(r, t) + 16 * u(r, t - h) - u(r, t - 2 * h)) / (12 * h * h)
        urr = (-u(r + 2 * h, t) + 16 * u(r + h, t) - 30 * u(r, t) + 16 * u(r - h, t) - u(r - 2 * h, t)) / (12 * h * h)
        assert abs(utt - v * v * urr) < 1e-6 * (abs(utt) + 1.0)


def test_outgoing_is_exact_minus_incoming_and_dominates_far_field():
    A, sigma, v = 1.0, 0.1e-3, 1500.0
    r = 20e-3
    for d in np.linspace(-0.3e-3, 0.3e-3, 7):
        t = (r - d) / v
        p_ex = oracle.pressure_exact(A, sigma, r, t, v)
        p_out = oracle.pressure_outgoing(A, sigma, r, t, v)
        assert abs(p_ex - p_out) <= 1e-300 + 1e-15 * abs(p_ex)
    # near field: the incoming term is visible and has the sign of (r + vt) > 0
    r, t = 0.1e-3, 0.05e-3 / v
    assert oracle.pressure_exact(A, sigma, r, t, v) > oracle.pressure_outgoing(A, sigma, r, t, v)


# ---------------------------------------------------------------- forward operator

def _cluster():
    g = synth.centred_grid(2, 2, 2, 0.3e-3, sigma=0.25e-3)
    rng = np.random.default_rng(11)
    A = rng.uniform(0.5, 1.5, g.M).astype(np.float32)
    return g, A


def test_forward_exact_matches_spherical_means_of_summed_field():
    """Linearity (Methods: the detected wave is the superposition): the oracle forward in
    exact mode equals quadrature of Eq. (pa_wave) applied to the summed initial field."""
    g, A = _cluster()
    G = oracle.gaussians_from_grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma, A)
    sensors = np.array([[0.4e-3, -0.2e-3, -3.0e-3], [2.5e-3, 1.0e-3, 1.2e-3]], np.float32)
    v, fs, t0, Nt = 1500.0, 40e6, 0.0, 128
    y = oracle.forward(G, sensors, v, fs, t0, Nt, mode="exact")
    field = gaussian_field(G.c, G.sigma, G.A)
    worst = 0.0
    for j, s in enumerate(sensors.astype(np.float64)):
        axis = -s
        for n in [60, 70, 78, 85, 95, 104]:
            t = t0 + n / fs

            def mean_term(tt):
                return sphere_quadrature(field, s, v * tt, axis=axis, theta_max=math.pi / 2,
                                         n_theta=240, n_phi=240) / (v * tt)
            p = d4(mean_term, t, 2e-10) / (4 * math.pi * v)
            worst = max(worst, abs(p - y[j, n]))
    assert worst <= 1e-7 * np.max(np.abs(y))


def test_forward_windowed_wide_window_equals_exact_far_field():
    w = synth.tiny(1)
    rng = np.random.default_rng(5)
    idx = rng.choice(w.M, 64, replace=False)
    G = oracle.gaussians_from_grid(w.grid.nx, w.grid.ny, w.grid.nz, w.grid.ox, w.grid.oy, w.grid.oz,
                                   w.grid.h, w.grid.sigma, np.zeros(w.M, np.float32))
    G = oracle.Gaussians(G.c[idx], G.sigma[idx], rng.uniform(0.2, 1.0, 64))
    sens = w.sensors[:8]
    y_ex = oracle.forward(G, sens, w.v, w.fs, w.t0, w.Nt, mode="exact")
    y_w = oracle.forward(G, sens, w.v, w.fs, w.t0, w.Nt, k=40.0)
    assert np.linalg.norm(y_w - y_ex) <= 1e-12 * np.linalg.norm(y_ex)
    # the 3-sigma window drops only the Gaussian tails: small but non-zero change
    y3 = oracle.forward(G, sens, w.v, w.fs, w.t0, w.Nt, k=3.0)
    rel = np.linalg.norm(y3 - y_ex) / np.linalg.norm(y_ex)
    assert 1e-4 < rel < 0.1


@pytest.mark.parametrize("t0", [0.0, 0.37e-6])
def test_forward_window_membership_brute_force(t0):
    """Single Gaussians: the non-zero samples are exactly {n : |R - v t_n| <= k sigma},
    checked against every sample index (brute force), including R near the array ends."""
    v, fs, Nt, k, sigma = 1500.0, 40e6, 600, 3.0, 0.1e-3
    rng = np.random.default_rng(3)
    n_all = np.arange(Nt)
    for R in list(rng.uniform(1e-3, 23e-3, 25)) + [v * (t0 + 3 / fs), v * (t0 + (Nt - 2) / fs)]:
        G = oracle.Gaussians(np.array([[0.0, 0.0, R]]), np.array([sigma]), np.array([1.0]))
        y = oracle.forward(G, np.zeros((1, 3), np.float32), v, fs, t0, Nt, k=k)[0]
        d = R - v * (t0 + n_all / fs)
        inside = np.abs(d) <= k * sigma
        nz = (y != 0.0) | (np.abs(d) < 1e-15)   # d == 0 exactly gives a zero sample
        assert np.array_equal(nz, inside)


def test_forward_ambiguity_bound_flags_boundary_samples():
    v, fs, t0, Nt, k, sigma = 1500.0, 40e6, 0.0, 800, 3.0, 0.1e-3
    n0 = 500
    R = v * (t0 + n0 / fs) + k * sigma           # sample n0 sits exactly on the window edge
    G = oracle.Gaussians(np.array([[R, 0.0, 0.0]]), np.array([sigma]), np.array([2.0]))
    y, amb = oracle.forward(G, np.zeros((1, 3), np.float32), v, fs, t0, Nt, k=k, tau=1e-9, want_amb=True)
    assert amb[0, n0] > 0 and np.count_nonzero(amb) <= 2
    assert amb[0, n0] == pytest.approx(abs(oracle.pressure_outgoing(2.0, sigma, R, n0 / fs, v)), rel=1e-6)


# ---------------------------------------------------------------- adjoint

def _small_free(seed, M=96, Nd=12, Nt=1024):
    g = synth.centred_grid(8, 4, 3, 0.15e-3)
    cx, cy, cz, sg, A = synth.free_gaussians(g, seed, jitter=0.05e-3)
    A = np.random.default_rng(seed).uniform(0.1, 1.0, g.M).astype(np.float32)
    G = oracle.gaussians_from_soa(cx, cy, cz, sg, A)
    sens = synth.cap_sensors(Nd, 20e-3, 160.0)
    return G, sens, 1500.0, 40e6, 0.0, Nt


@pytest.mark.parametrize("k", [3.0, 6.0])
def test_adjoint_identity(k):
    G, sens, v, fs, t0, Nt = _small_free(7)
    rng = np.random.default_rng(9)
    x = rng.normal(size=G.M)
    dl = rng.normal(size=(len(sens), Nt))
    Fx = oracle.forward(G, sens, v, fs, t0, Nt, k=k, A=x)
    FTd = oracle.adjoint(G, sens, v, fs, t0, Nt, dl, k=k)["A"]
    lhs, rhs = float(np.sum(Fx * dl)), float(x @ FTd)
    assert abs(lhs - rhs) <= 1e-12 * (np.linalg.norm(Fx) * np.linalg.norm(dl))


def test_adjoint_centre_and_sigma_gradients_match_central_fd():
    """Gradients of L = <delta, F(c, sigma) A> against central differences of the oracle
    forward, at k = 10 where the moving window edge carries no weight."""
    G, sens, v, fs, t0, Nt = _small_free(13, Nt=1024)
    k = 10.0
    rng = np.random.default_rng(17)
    dl = rng.normal(size=(len(sens), Nt))
    grads = oracle.adjoint(G, sens, v, fs, t0, Nt, dl, k=k, want=("A", "c", "sigma"))

    def L(Gx):
        return float(np.sum(oracle.forward(Gx, sens, v, fs, t0, Nt, k=k) * dl))
    for i in rng.choice(G.M, 6, replace=False):
        for ax in range(3):
            hstep = 1e-6 * 1e-3
            Gp = oracle.Gaussians(G.c.copy(), G.sigma.copy(), G.A.copy())
            Gm = oracle.Gaussians(G.c.copy(), G.sigma.copy(), G.A.copy())
            Gp.c[i, ax] += hstep
            Gm.c[i, ax] -= hstep
            fd = (L(Gp) - L(Gm)) / (2 * hstep)
            assert abs(fd - grads["c"][ax, i]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grads["c"]).max())
        hs = 1e-6 * G.sigma[i]
        Gp = oracle.Gaussians(G.c.copy(), G.sigma.copy(), G.A.copy())
        Gm = oracle.Gaussians(G.c.copy(), G.sigma.copy(), G.A.copy())
        Gp.sigma[i] += hs
        Gm.sigma[i] -= hs
        fd = (L(Gp) - L(Gm)) / (2 * hs)
        assert abs(fd - grads["sigma"][i]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grads["sigma"]).max())


# ---------------------------------------------------------------- voxelize

@pytest.mark.parametrize("k,ntap", [(3.0, 3), (2.5, 2)])
def test_voxelize_grid_case_is_separable_convolution(k, ntap):
    g = synth.centred_grid(10, 7, 6, 0.1e-3)
    A = np.random.default_rng(2).uniform(0, 1, g.M).astype(np.float32)
    G = oracle.gaussians_from_grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma, A)
    vol = oracle.voxelize(G, k, g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h)
    taps = np.exp(-np.arange(-ntap, ntap + 1) ** 2 / 2.0)
    ref = A.astype(np.float64).reshape(g.nz, g.ny, g.nx)
    for axis in range(3):
        ref = np.apply_along_axis(lambda r: np.convolve(r, taps, mode="full")[ntap:ntap + r.size], axis, ref)
    assert np.max(np.abs(vol - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_voxelize_free_centres_brute_force():
    rng = np.random.default_rng(4)
    M = 5
    c = rng.uniform(-0.2e-3, 0.2e-3, (M, 3))
    sg = rng.uniform(0.05e-3, 0.15e-3, M)
    A = rng.uniform(0.5, 1.0, M)
    G = oracle.Gaussians(c, sg, A)
    n, h, o = 6, 0.08e-3, -0.24e-3
    vol = oracle.voxelize(G, 3.0, n, n, n, o, o, o, h)
    f = lambda q: float(np.float32(q))
    ref = np.zeros((n, n, n))
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                p = np.array([f(o) + (ix + 0.5) * f(h), f(o) + (iy + 0.5) * f(h), f(o) + (iz + 0.5) * f(h)])
                for i in range(M):
                    dd = p - c[i]
                    if np.all(np.abs(dd) <= 3.0 * sg[i]):
                        ref[iz, iy, ix] += A[i] * math.exp(-float(dd @ dd) / (2 * sg[i] ** 2))
    assert np.max(np.abs(vol - ref)) <= 1e-13


# ---------------------------------------------------------------- Adam, CAWR, Algorithm 2

def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    z = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    zt = torch.tensor(z.copy(), requires_grad=True)
    opt = torch.optim.Adam([zt], lr=0.03, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 12):
        g = rng.normal(size=50)
        oracle.adam(z, m, v, g, t, 0.03)
        zt.grad = torch.tensor(g)
        opt.step()
    assert np.max(np.abs(z - zt.detach().numpy())) <= 1e-12


@pytest.mark.parametrize("T0,Tmult", [(10, 1.0), (4, 2.0), (3, 3.0)])
def test_cawr_matches_torch(T0, Tmult):
    torch = pytest.importorskip("torch")
    p = torch.zeros(1, requires_grad=True)
    opt = torch.optim.SGD([p], lr=0.5)
    sch = torch.optim.lr_scheduler.CosineAnnealingWarmRestarts(opt, T_0=T0, T_mult=int(Tmult), eta_min=0.01)
    for t in range(40):
        assert oracle.cawr(t, 0.5, 0.01, T0, Tmult) == pytest.approx(opt.param_groups[0]["lr"], abs=1e-12)
        opt.step()
        sch.step()


def _dense_problem():
    g = synth.centred_grid(4, 4, 4, 0.2e-3)
    G = oracle.gaussians_from_grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma, np.zeros(g.M, np.float32))
    sens = synth.cap_sensors(6, 5e-3, 180.0)
    v, fs, t0, Nt = 1500.0, 40e6, 0.0, 256
    F = np.stack([oracle.forward(G, sens, v, fs, t0, Nt, A=np.eye(g.M)[i]).ravel() for i in range(g.M)], 1)
    x_true = np.random.default_rng(21).uniform(0, 1, g.M)
    b = F @ x_true
    return G, sens, v, fs, t0, Nt, F, b


def test_ir_adam_npc_cawr_matches_torch_autograd():
    """Algorithm 2 (NPC, data loss |F x - b|^2 / N, Adam, CAWR) against torch autograd +
    torch.optim on the dense matrix of the same operator."""
    torch = pytest.importorskip("torch")
    G, sens, v, fs, t0, Nt, F, b = _dense_problem()
    iters, eta, T0 = 15, 0.05, 6
    x, loss, resid = oracle.ir(G, sens, v, fs, t0, Nt, b, iters, rule="adam", npc=True,
                               eta_max=eta, eta_min=0.001, T0=T0, Tmult=1.0)
    Ft = torch.tensor(F)
    bt = torch.tensor(b)
    z = torch.zeros(G.M, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([z], lr=eta, betas=(0.9, 0.999), eps=1e-8)
    sch = torch.optim.lr_scheduler.CosineAnnealingWarmRestarts(opt, T_0=T0, T_mult=1, eta_min=0.001)
    tl = []
    for t in range(iters):
        opt.zero_grad()
        L = torch.mean((Ft @ (z + 1e-8) ** 2 - bt) ** 2)
        tl.append(float(L))
        L.backward()
        opt.step()
        sch.step()
    xt = ((z + 1e-8) ** 2).detach().numpy()
    assert np.allclose(loss, tl, rtol=1e-9, atol=0)
    assert np.max(np.abs(x - xt)) <= 1e-9 * np.max(np.abs(xt))
    assert resid[0] == pytest.approx(np.linalg.norm(b), rel=1e-12)


def test_ir_line_search_is_exact_minimiser():
    G, sens, v, fs, t0, Nt, F, b = _dense_problem()
    x, loss, resid = oracle.ir(G, sens, v, fs, t0, Nt, b, 4, rule="linesearch", npc=False)
    assert np.all(np.diff(loss) < 0)
    x1, _, _ = oracle.ir(G, sens, v, fs, t0, Nt, b, 1, rule="linesearch", npc=False)
    g = F.T @ (F @ np.zeros(G.M) - b)
    f = lambda a: float(np.sum((F @ (-a * g) - b) ** 2))
    alpha = -x1[0] / g[0] if g[0] != 0 else -x1[1] / g[1]
    assert np.allclose(x1, -alpha * g, rtol=1e-10)
    assert f(alpha) <= f(alpha * 1.01) and f(alpha) <= f(alpha * 0.99)


# ---------------------------------------------------------------- ASSA (Algorithm 1)

def _assa_case(seed=21):
    g = synth.centred_grid(6, 5, 4, 0.1e-3)
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.2, 1.0, g.M)
    G = oracle.gaussians_from_grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma, A)
    sens = synth.cap_sensors(7, 6e-3, 150.0)
    return g, G, sens, 1500.0, 40e6, 0.0, 512


def test_assa_adjoint_identity():
    g, G, sens, v, fs, t0, Nt = _assa_case()
    rng = np.random.default_rng(5)
    x = rng.uniform(0.0, 1.0, G.M)
    delta = rng.normal(size=(len(sens), Nt))
    Gx = oracle.Gaussians(G.c, G.sigma, x)
    Fx = oracle.assa_forward(Gx, g.sigma, sens, v, fs, t0, Nt)
    FTd = oracle.assa_adjoint(Gx, g.sigma, sens, v, fs, t0, Nt, delta)
    lhs, rhs = float(np.sum(Fx * delta)), float(x @ FTd)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Fx) * np.linalg.norm(delta)


def _assa_dense_problem():
    g = synth.centred_grid(4, 4, 4, 0.2e-3)
    G = oracle.gaussians_from_grid(g.nx, g.ny, g.nz, g.ox, g.oy, g.oz, g.h, g.sigma, np.zeros(g.M))
    sens = synth.cap_sensors(6, 5e-3, 180.0)
    v, fs, t0, Nt = 1500.0, 40e6, 0.0, 256
    F = np.stack([oracle.assa_forward(oracle.Gaussians(G.c, G.sigma, np.eye(g.M)[i]), g.sigma, sens, v, fs, t0,
                                      Nt).ravel() for i in range(g.M)], 1)
    b = F @ np.random.default_rng(22).uniform(0, 1, g.M)
    return g, G, sens, v, fs, t0, Nt, F, b


def test_ir_on_assa_matches_torch_autograd():
    """Algorithm 2 with the discretised operator (NPC, Adam, CAWR) against torch autograd and
    torch.optim on the dense matrix of Algorithm 1's forward."""
    torch = pytest.importorskip("torch")
    g, G, sens, v, fs, t0, Nt, F, b = _assa_dense_problem()
    iters, eta, T0 = 12, 0.05, 5
    x, loss, resid = oracle.ir_assa(G, g.sigma, sens, v, fs, t0, Nt, b, iters, eta_max=eta, eta_min=0.001, T0=T0)
    Ft, bt = torch.tensor(F), torch.tensor(b)
    z = torch.zeros(G.M, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([z], lr=eta, betas=(0.9, 0.999), eps=1e-8)
    sch = torch.optim.lr_scheduler.CosineAnnealingWarmRestarts(opt, T_0=T0, T_mult=1, eta_min=0.001)
    tl = []
    for _ in range(iters):
        opt.zero_grad()
        L = torch.mean((Ft @ (z + 1e-8) ** 2 - bt) ** 2)
        tl.append(float(L))
        L.backward()
        opt.step()
        sch.step()
    xt = ((z + 1e-8) ** 2).detach().numpy()
    assert np.allclose(loss, tl, rtol=1e-9, atol=0)
    assert np.max(np.abs(x - xt)) <= 1e-9 * np.max(np.abs(xt))
    assert loss[-1] < loss[0]


def test_ir_on_assa_line_search_is_exact_minimiser():
    g, G, sens, v, fs, t0, Nt, F, b = _assa_dense_problem()
    x1, loss, _ = oracle.ir_assa(G, g.sigma, sens, v, fs, t0, Nt, b, 1, rule="linesearch", npc=False)
    gr = F.T @ -b
    alpha = -float(b @ (F @ gr)) / float(np.sum((F @ gr) ** 2))   # argmin_a |F(-a g) - b|^2, g = F^T (0 - b)
    assert np.allclose(x1, -alpha * gr, rtol=1e-10, atol=0)
    _, loss2, _ = oracle.ir_assa(G, g.sigma, sens, v, fs, t0, Nt, b, 3, rule="linesearch", npc=False)
    assert np.all(np.diff(loss2) < 0)


def test_assa_stages_equal_the_folded_single_sum():
    """Projection, transposed convolution and decimation collapse to
    y_j[n] = sum_i (x_i / r_ij) h[alpha n - k_ij] over |alpha n - k_ij| <= K; evaluated here pair by
    pair, which checks the staging's index conventions (kernel orientation, decimation phase)."""
    g, G, sens, v, fs, t0, Nt = _assa_case()
    nh, alpha, K = oracle.assa_params(g.sigma, v, fs)
    fs_up = alpha * fs
    y = oracle.assa_forward(G, g.sigma, sens, v, fs, t0, Nt)
    yd = np.zeros_like(y)
    n = np.arange(Nt)
    for j, s in enumerate(sens):
        r = np.linalg.norm(G.c - s, axis=1)
        k = np.floor((r / v - t0) * fs_up + 0.5).astype(np.int64)
        for i in range(G.M):
            q = alpha * n - k[i]
            m = np.abs(q) <= K
            d = -v * q[m] / fs_up
            yd[j, m] += G.A[i] / r[i] * 0.5 * d * np.exp(-d * d / (2 * g.sigma ** 2))
    assert np.abs(y).max() > 0
    assert np.linalg.norm(y - yd) <= 1e-12 * np.linalg.norm(yd)


def test_assa_equals_windowed_forward_when_times_of_flight_are_on_the_grid():
    """Gaussians on the axes through one sensor at distances v k / fs_up: snapping is exact, and
    ASSA then equals the outgoing term of Eq. (single_forward) over the window
    |d| <= N_half v / fs (K upsampled samples), as evaluated by the windowed forward."""
    v, fs, t0, Nt, sigma = 1500.0, 40e6, 0.0, 2048, 0.1e-3
    nh, alpha, K = oracle.assa_params(sigma, v, fs)
    fs_up = alpha * fs
    ks = [1500, 1623, 1777, 2101, 2400, 2999]
    dirs = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [-1, 0, 0], [0, -1, 0], [0, 0, -1]], float)
    c = np.array([v * k / fs_up * d for k, d in zip(ks, dirs)])
    A = np.random.default_rng(2).uniform(0.5, 1.5, len(ks))
    G = oracle.Gaussians(c, np.full(len(ks), sigma), A)
    sens = np.zeros((1, 3))
    y = oracle.assa_forward(G, sigma, sens, v, fs, t0, Nt)
    # window just wider than N_half v dt by less than one upsampled step: the same sample set
    kw = (nh + 0.4 / alpha) * (v / fs) / sigma
    yw = oracle.forward(G, sens, v, fs, t0, Nt, k=kw)
    assert np.abs(yw).max() > 0
    assert np.linalg.norm(y - yw) <= 1e-12 * np.linalg.norm(yw)


def test_assa_converges_to_the_windowed_forward_as_n_min_grows():
    """The snapping error is at most half an upsampled step, so the difference to the exact
    windowed operator falls roughly as 1 / alpha."""
    g, G, sens, v, fs, t0, Nt = _assa_case(seed=4)
    nh, _, _ = oracle.assa_params(g.sigma, v, fs)
    kw = nh * (v / fs) / g.sigma             # ASSA's window, |d| <= N_half v dt, for every alpha
    yw = oracle.forward(G, sens, v, fs, t0, Nt, k=kw)
    errs = []
    for n_min in (25, 101, 401):
        _, alpha, _ = oracle.assa_params(g.sigma, v, fs, n_min)
        y = oracle.assa_forward(G, g.sigma, sens, v, fs, t0, Nt, n_min=n_min)
        errs.append((alpha, np.linalg.norm(y - yw) / np.linalg.norm(yw)))
    (a1, e1), (a2, e2), (a3, e3) = errs
    assert e2 < e1 * 2.0 * a1 / a2 and e3 < e2 * 2.0 * a2 / a3, errs
    assert all(0.005 < e * a < 0.05 for a, e in errs), errs     # error x alpha roughly constant


# ---------------------------------------------------------------- VCR regulariser

def test_vcr_gradient_matches_central_differences():
    from oracle import vcr

    rng = np.random.default_rng(7)
    x = rng.uniform(0.0, 1.0, (4, 5, 6))
    beta = 0.7
    _, g = vcr.value_and_grad(x, beta)
    h = 1e-6
    for idx in [(0, 0, 0), (3, 4, 5), (1, 2, 3), (2, 0, 5), (0, 4, 2), (3, 1, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (vcr.value_and_grad(xp, beta)[0] - vcr.value_and_grad(xm, beta)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, g[idx])


def test_vcr_constant_image():
    from oracle import vcr

    x = np.full((3, 4, 5), 2.5)
    val, g = vcr.value_and_grad(x, 0.3, eps=1e-8)
    assert abs(val - x.size * 1e-4 * 1.3) <= 1e-12 * val
    assert np.abs(g).max() == 0.0


def test_vcr_linear_ramp_closed_form():
    """x = a * ix: central differences give a inside and a / 2 on the two x faces (clamped
    neighbour); second differences vanish inside and are +a / -a on the faces; no mixed terms."""
    from oracle import vcr

    nz, ny, nx, a, eps, beta = 3, 4, 6, 0.8, 1e-8, 0.5
    x = a * np.broadcast_to(np.arange(nx, dtype=np.float64), (nz, ny, nx))
    val, _ = vcr.value_and_grad(x, beta, eps)
    rows = ny * nz
    R_TV = rows * ((nx - 2) * np.sqrt(a * a + eps) + 2 * np.sqrt(a * a / 4 + eps))
    R_H = rows * ((nx - 2) * np.sqrt(eps) + 2 * np.sqrt(a * a + eps))
    assert abs(val - (R_H + beta * R_TV)) <= 1e-12 * val


def test_vcr_mixed_derivative_of_a_bilinear_image():
    from oracle import vcr

    nz, ny, nx = 3, 5, 6
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x = (ix * iy).astype(np.float64)
    first, hess = vcr.operators(x.shape)
    Dxy = hess[3][0] @ x.ravel()
    inner = ((ix > 0) & (ix < nx - 1) & (iy > 0) & (iy < ny - 1)).ravel()
    assert np.allclose(Dxy[inner], 1.0)
    assert hess[3][1] == 2.0
    Dxx = (hess[0][0] @ x.ravel())[((ix > 0) & (ix < nx - 1)).ravel()]
    assert np.allclose(Dxx, 0.0)


# ---------------------------------------------------------------- image metrics (Table 1)

def test_metrics_closed_forms():
    from oracle import metrics

    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (9, 10, 11))
    assert abs(metrics.ssim(x, x) - 1.0) < 1e-12
    assert abs(metrics.psnr(x + 0.1, x) - 20.0) < 1e-9          # MSE 0.01, range 1
    # constant image against a shifted one: only the luminance term remains
    a, c, C1 = 0.4, 0.25, (0.01) ** 2
    ones = np.ones((9, 9, 9))
    expect = (2 * a * (a + c) + C1) / (a * a + (a + c) ** 2 + C1)
    assert abs(metrics.ssim(a * ones, (a + c) * ones) - expect) < 1e-12
    # the projection, brute force
    m = metrics.zmap(x)
    for iy, ix in [(0, 0), (3, 7), (9, 10)]:
        assert m[iy, ix] == max(x[z, iy, ix] for z in range(x.shape[0]))


def test_ssim_window_by_brute_force():
    """One interior position of a 2-D SSIM map, from its window's samples directly."""
    from oracle import metrics

    rng = np.random.default_rng(6)
    x, y = rng.uniform(0, 1, (12, 13)), rng.uniform(0, 1, (12, 13))
    win, C1, C2 = 7, 1e-4, 9e-4
    # SSIM over a 7 x 7 image is the single value of its one interior position
    xs, ys = x[:7, :7], y[:7, :7]
    mx, my = xs.mean(), ys.mean()
    sx, sy = xs.var(ddof=1), ys.var(ddof=1)
    sxy = ((xs - mx) * (ys - my)).sum() / (xs.size - 1)
    expect = (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sx + sy + C2))
    assert abs(metrics.ssim(xs, ys, win=win) - expect) < 1e-12


# ---------------------------------------------------------------- U-Net reference (warm start)

def _unet_weights(rng, scale=1.0):
    from oracle import unet_ref

    W, B = {}, {}
    for n, ci, co, taps, relu in unet_ref.architecture():
        W[n] = rng.normal(size=(co, taps, ci)) * scale * math.sqrt(2.0 / (taps * ci))
        B[n] = rng.normal(size=co) * 0.1
    return W, B


def test_unet_architecture_is_the_configured_one():
    """Four levels with 16, 32, 64 and 128 channels, one channel in and one out (the input padded
    to 16 stored channels, the prediction channel 0 of 16 computed); two 3x3x3 convolutions per
    level; the decoder concatenates the upsampled level with the skip.  The product network
    (paper_2602_03893_gb300.unet) declares the same layers."""
    from oracle import unet_ref
    from paper_2602_03893_gb300 import unet

    assert unet_ref.LEVEL_CHANNELS == (16, 32, 64, 128)
    assert unet_ref.IN_CHANNELS == 1 and unet_ref.OUT_CHANNELS == 1
    arch = {n: (ci, co, taps, relu) for n, ci, co, taps, relu in unet_ref.architecture()}
    assert tuple(arch) == unet_ref.ORDER and len(arch) == 15
    for lvl, c in enumerate(unet_ref.LEVEL_CHANNELS):
        enc = ["e1", "e2", "e3", "b4"][lvl]
        assert arch[enc + "a"][1] == c and arch[enc + "b"][:2] == (c, c)
    assert arch["d3a"][0] == 128 + 64 and arch["d2a"][0] == 64 + 32 and arch["d1a"][0] == 32 + 16
    assert arch["out"] == (16, 16, 1, False) and all(v[2] == 27 and v[3] for k, v in arch.items() if k != "out")
    prod = unet.layer_specs(unet.UNet3D.CH)
    assert {k: (c.cin, c.cout, c.taps, c.relu) for k, c in prod.items()} == arch
    assert unet.CIN_PAD == unet_ref.IN_STORED and unet.COUT_PAD == unet_ref.OUT_STORED


def test_unet_layers_against_plain_loops():
    """3x3x3 and 1x1x1 convolutions with zero padding (with and without ReLU), 2x2x2 average
    pooling and nearest x2 upsampling of the torch reference, against the sums written out."""
    import torch

    from oracle import unet_ref

    rng = np.random.default_rng(21)
    x = rng.normal(size=(3, 3, 4, 5))
    for taps, relu in ((27, True), (27, False), (1, False)):
        w = rng.normal(size=(4, taps, 3))
        b = rng.normal(size=4)
        ref = unet_ref.conv(torch.tensor(x)[None], torch.tensor(w), torch.tensor(b), taps, relu)[0].numpy()
        np.testing.assert_allclose(ref, unet_ref.conv_loops(x, w, b, taps, relu), rtol=0, atol=1e-12)
    x = rng.normal(size=(3, 4, 6, 2))
    np.testing.assert_allclose(unet_ref.pool(torch.tensor(x)[None])[0].numpy(), unet_ref.pool_loops(x),
                               rtol=0, atol=1e-15)
    np.testing.assert_array_equal(unet_ref.up(torch.tensor(x)[None])[0].numpy(), unet_ref.up_loops(x))
    # a one-hot input places each tap where the definition says: output (z, y, x) sees tap
    # (dz, dy, dx) from input (z + dz, y + dy, x + dx)
    xo = np.zeros((1, 3, 3, 3))
    xo[0, 2, 1, 0] = 1.0
    wt = np.arange(27, dtype=float).reshape(1, 27, 1)
    yo = unet_ref.conv(torch.tensor(xo)[None], torch.tensor(wt), torch.zeros(1, dtype=torch.float64), 27,
                       False)[0, 0].numpy()
    assert yo[1, 1, 1] == (1 + 1) * 9 + (0 + 1) * 3 + (-1 + 1)      # dz = 1, dy = 0, dx = -1


def test_bf16_rounding_against_bit_pattern():
    """torch's BF16 conversion (used by the reference's storage rounding) against round to
    nearest even on the float32 pattern, including exact ties, subnormals and large values."""
    import torch

    from oracle import unet_ref

    rng = np.random.default_rng(22)
    base = rng.normal(size=4000).astype(np.float32) * np.float32(10.0) ** rng.integers(-30, 30, 4000).astype(np.float32)
    # ties: a bf16 value plus exactly half of its last place, both parities of the kept bit
    expo = rng.integers(100, 150, 2000, dtype=np.uint32) << np.uint32(23)
    kept = rng.integers(0, 128, 2000, dtype=np.uint32) << np.uint32(16)
    ties = (expo | kept | np.uint32(0x8000)).view(np.float32)
    sub = (rng.integers(1, 2 ** 23, 500, dtype=np.uint32)).view(np.float32)
    x = np.concatenate([base, ties, -ties, sub, np.float32([0.0, -0.0, 3.0e38, -3.0e38])])
    got = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(got, unet_ref.bf16_round_loops(x))
    g = torch.tensor(x.astype(np.float64), requires_grad=True)
    (gr,) = torch.autograd.grad(unet_ref.RoundBF16.apply(g), g, torch.tensor(x.astype(np.float64)))
    np.testing.assert_array_equal(gr.numpy(), unet_ref.bf16_round_loops(x))


@pytest.mark.parametrize("bf16", [False, True])
def test_unet_forward_against_plain_loops(bf16):
    """The whole network (8 x 8 x 8 volume, all four levels) against the composition of the
    written-out layers; with BF16 storage both sides round the same stored activations."""
    import torch

    from oracle import unet_ref

    rng = np.random.default_rng(23)
    W, B = _unet_weights(rng)
    x0 = np.zeros((16, 8, 8, 8))
    x0[0] = rng.normal(size=(8, 8, 8))
    ref = unet_ref.unet_forward(torch.tensor(x0)[None], {k: torch.tensor(v) for k, v in W.items()},
                                {k: torch.tensor(v) for k, v in B.items()}, bf16_storage=bf16)[0].numpy()
    loops = unet_ref.unet_forward_loops(x0, W, B, bf16_storage=bf16)
    assert np.abs(ref).max() > 0.1
    err = np.linalg.norm(ref - loops) / np.linalg.norm(loops)
    assert err <= (1e-3 if bf16 else 1e-12), err


def test_unet_gradients_against_central_differences():
    """torch autograd through the FP64 reference against central differences of the loop network
    on sampled weights of five layers, a bias and an input voxel (loss = sum of c * output)."""
    import torch

    from oracle import unet_ref

    rng = np.random.default_rng(24)
    W, B = _unet_weights(rng)
    x0 = np.zeros((16, 8, 8, 8))
    x0[0] = rng.normal(size=(8, 8, 8))
    cvec = rng.normal(size=(16, 8, 8, 8))
    Wt = {k: torch.tensor(v, requires_grad=True) for k, v in W.items()}
    Bt = {k: torch.tensor(v, requires_grad=True) for k, v in B.items()}
    xt = torch.tensor(x0, requires_grad=True)
    out = unet_ref.unet_forward(xt[None], Wt, Bt)[0]
    (out * torch.tensor(cvec)).sum().backward()
    loss = lambda W_, B_, x_: float(np.sum(cvec * unet_ref.unet_forward_loops(x_, W_, B_)))
    probes = [("w", "e1a", (3, 13, 0)), ("w", "e3b", (5, 2, 7)), ("w", "b4a", (100, 26, 40)),
              ("w", "d2a", (9, 4, 80)), ("w", "out", (0, 0, 11)), ("b", "d1b", (6,)), ("x", None, (0, 4, 3, 5))]
    for kind, name, idx in probes:
        arr = {"w": W.get(name), "b": B.get(name), "x": x0}[kind]
        grad = {"w": Wt.get(name), "b": Bt.get(name), "x": xt}[kind].grad.numpy()[idx]
        h = 1e-6 * max(1.0, abs(arr[idx]))
        old = arr[idx]
        arr[idx] = old + h
        lp = loss(W, B, x0)
        arr[idx] = old - h
        lm = loss(W, B, x0)
        arr[idx] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad) <= 1e-6 * max(1.0, abs(grad)), (kind, name, idx, fd, grad)
