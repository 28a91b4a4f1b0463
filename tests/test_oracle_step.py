"""Pins of the oracle's time stepping against closed forms, invariants, Fourier analysis and brute
force (Section 2.1, Eqs. 4-6).  The Fourier symbol below is assembled here, independently of the
oracle's stencil loops, from the staggered positions of Section 2.1."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import sh, stepper as st
from paper_2004_02833_gb300 import synth


def _problem(N, shape, sa, ss, q, h, dt, bc, coupling_cache):
    mats, slots = coupling_cache(N)
    return st.Problem(N, np.broadcast_to(sa, shape).copy(), np.broadcast_to(ss, shape).copy(),
                      np.broadcast_to(q, shape).copy(), h, dt, bc, mats=mats, slots=slots)


# ----------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("bc", ["periodic", "vacuum"])
def test_p0_closed_form(bc, coupling_cache):
    # N = 0 leaves u_0' = -sigma_a u_0 + q per cell; Eq. (5) solves it exactly, so after t:
    # u_0 e^{-sigma_a t} + q (1 - e^{-sigma_a t}) / sigma_a.
    shape = (3, 4, 5)
    sa, _, q = synth.random_media(shape, 11, 0.1, 3.0)
    P = _problem(0, shape, sa, 0.0, q, 0.2, 0.05, bc, coupling_cache)
    u = synth.random_state(0, shape, 12)
    k = 7
    t = k * P.dt
    want = u[0] * np.exp(-sa * t) + q * (-np.expm1(-sa * t)) / sa
    got = P.run(u, k)[0]
    assert np.abs(got - want).max() < 1e-14


def test_uniform_state_decays(coupling_cache):
    # Periodic, homogeneous media, every moment uniform in space: all differences vanish and each
    # step multiplies u_0 by e^{-sigma_a dt} and every other moment by e^{-(sigma_a+sigma_s) dt}.
    N, shape = 3, (4, 4, 4)
    sa, ss = 0.3, 1.7
    P = _problem(N, shape, sa, ss, 0.0, 0.25, 0.08, "periodic", coupling_cache)
    vals = np.linspace(-1.0, 2.0, P.n_c)
    u = np.broadcast_to(vals[:, None, None, None], (P.n_c,) + shape).copy()
    k = 5
    got = P.run(u, k)
    f = np.full(P.n_c, np.exp(-(sa + ss) * k * P.dt))
    f[0] = np.exp(-sa * k * P.dt)
    assert np.abs(got - (vals * f)[:, None, None, None]).max() < 1e-14


def test_conservation_of_u0():
    # Config 0 rules (P3, 32^3 periodic, sigma_a = 0, q = 0): sum of u_0 is conserved by every
    # substep (the u_0 update adds a sum of periodic differences), 40 steps.
    inst = synth.gaussian_pulse(3, 32)
    P = st.Problem(3, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, inst.bc)
    u = P.run(inst.full_state(), 40)
    assert abs(u[0].sum() - 1.0) < 1e-14
    assert np.abs(u[1:]).max() > 1e-6  # the pulse actually moved


def test_interpolation_linear_media(coupling_cache):
    # The mean of a linear field over the cells adjacent to a staggered point equals its value at
    # the point (interior points; reading of "interpolated", Section 3.2).
    n = 6
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    sig = 1.0 + 0.5 * x + 0.25 * y + 0.125 * z
    for slot in [(2, 1, 1), (1, 2, 2), (2, 2, 2), (1, 1, 1)]:
        avg = st.point_average(sig, slot, "vacuum")
        off = [(g - 1) * 0.5 for g in slot]
        want = 1.0 + 0.5 * (x + off[0]) + 0.25 * (y + off[1]) + 0.125 * (z + off[2])
        inner = (slice(0, n - 1),) * 3
        assert np.abs(avg[inner] - want[inner]).max() < 1e-14
        avg_p = st.point_average(sig, slot, "periodic")
        assert np.abs(avg_p[inner] - want[inner]).max() < 1e-14


def test_vacuum_equals_zeroed_ring(coupling_cache):
    # Vacuum reads 0 outside; the same evolution results from a periodic grid padded by one cell per
    # side whose padding is reset to 0 before every substep (homogeneous media).
    N, n = 3, 5
    shape, pshape = (n,) * 3, (n + 2,) * 3
    Pv = _problem(N, shape, 0.4, 0.9, 0.3, 0.2, 0.06, "vacuum", coupling_cache)
    Pp = _problem(N, pshape, 0.4, 0.9, 0.3, 0.2, 0.06, "periodic", coupling_cache)
    u = synth.random_state(N, shape, 5)
    up = np.zeros((Pp.n_c,) + pshape)
    inner = (slice(None),) + (slice(1, n + 1),) * 3
    up[inner] = u

    def zero_ring(v):
        w = np.zeros_like(v)
        w[inner] = v[inner]
        return w

    for _ in range(3):
        u = Pv.step(u)
        for cls, tau in ((1, 0.5 * Pp.dt), (0, Pp.dt), (1, 0.5 * Pp.dt)):
            up = Pp.substep(zero_ring(up), cls, tau)
    assert np.abs(up[inner] - u).max() < 1e-14


# ----------------------------------------------------------------------------- Fourier analysis
def _factors(c, tau):
    alpha = np.exp(-c * tau)
    beta = tau if c == 0 else -np.expm1(-c * tau) / c
    return alpha, beta


def _symbol(P, k, sa, ss):
    """Amplification matrix of one step for the mode e^{i k . x_a} in physical staggered positions.
    A half-grid centred difference of e^{i k x} at a staggered point is (2i/h) sin(k h / 2)."""
    n = P.n_c
    sig = [2j * np.sin(k[d] * P.h[d] / 2.0) / P.h[d] for d in range(3)]
    K = sum(sig[d] * P.mats[d] for d in range(3))
    c = np.full(n, sa + ss)
    c[0] = sa

    def sub(cls, tau):
        G = np.eye(n, dtype=complex)
        for a in np.nonzero(P.cls == cls)[0]:
            al, be = _factors(c[a], tau)
            G[a] = -be * K[a]
            G[a, a] += al
        return G

    return sub(1, P.dt / 2) @ sub(0, P.dt) @ sub(1, P.dt / 2), K + np.diag(c)


def _positions(P, shape):
    """x_a(i) = (i + g/2) h on each axis (slot g = 1 -> (i+1/2)h, g = 2 -> (i+1)h)."""
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return [(X + P.slots[a, 0] / 2.0) * P.h[0] for a in range(P.n_c)], \
           [(Y + P.slots[a, 1] / 2.0) * P.h[1] for a in range(P.n_c)], \
           [(Z + P.slots[a, 2] / 2.0) * P.h[2] for a in range(P.n_c)]


@pytest.mark.parametrize("N,kint", [(1, (1, 0, 0)), (3, (1, 2, 3)), (7, (3, 1, 2))])
def test_single_mode_matches_symbol(N, kint, coupling_cache):
    n = 8
    shape = (n, n, n)
    sa, ss = 0.2, 0.7
    P = _problem(N, shape, sa, ss, 0.0, 1.0 / n, 0.3 / n, "periodic", coupling_cache)
    k = [2 * np.pi * kint[d] / (n * P.h[d]) for d in range(3)]
    G, _ = _symbol(P, k, sa, ss)
    rng = np.random.default_rng(0)
    uh = rng.standard_normal(P.n_c) + 1j * rng.standard_normal(P.n_c)
    X, Y, Z = _positions(P, shape)
    phase = np.array([np.exp(1j * (k[0] * X[a] + k[1] * Y[a] + k[2] * Z[a])) for a in range(P.n_c)])
    steps = 5
    got = P.run(np.real(uh[:, None, None, None] * phase), steps)
    want = np.real((np.linalg.matrix_power(G, steps) @ uh)[:, None, None, None] * phase)
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("N,kint", [(3, (1, 2, 3)), (7, (2, 1, 3))])
def test_single_mode_matches_symbol_non_cubic_cells(N, kint, coupling_cache):
    # cells hx != hy != hz on a 10 x 6 x 8 grid: each axis' difference divides by its own h
    # (Section 2.1), so the mode's symbol carries (2i/h_d) sin(k_d h_d / 2) per axis
    shape = (8, 6, 10)
    h = (0.1, 0.13, 0.17)
    sa, ss = 0.2, 0.7
    P = _problem(N, shape, sa, ss, 0.0, h, 0.03, "periodic", coupling_cache)
    n = (shape[2], shape[1], shape[0])
    k = [2 * np.pi * kint[d] / (n[d] * P.h[d]) for d in range(3)]
    G, _ = _symbol(P, k, sa, ss)
    rng = np.random.default_rng(5)
    uh = rng.standard_normal(P.n_c) + 1j * rng.standard_normal(P.n_c)
    X, Y, Z = _positions(P, shape)
    phase = np.array([np.exp(1j * (k[0] * X[a] + k[1] * Y[a] + k[2] * Z[a])) for a in range(P.n_c)])
    got = P.run(np.real(uh[:, None, None, None] * phase), 4)
    want = np.real((np.linalg.matrix_power(G, 4) @ uh)[:, None, None, None] * phase)
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("N", [1, 3, 7])
def test_lossless_modes_have_unit_amplification(N, coupling_cache):
    # sigma = 0: every eigenvalue of the step lies on the unit circle for dt < h/3 (Section 2.1
    # convergence condition), for every wave vector of an 8^3 grid.
    n = 8
    P = _problem(N, (n, n, n), 0.0, 0.0, 0.0, 1.0 / n, 0.3 / n, "periodic", coupling_cache)
    rng = np.random.default_rng(1)
    for _ in range(12):
        k = 2 * np.pi * rng.integers(0, n, 3) / (n * P.h[0])
        G, _ = _symbol(P, k, 0.0, 0.0)
        ev = np.abs(np.linalg.eigvals(G))
        assert np.abs(ev - 1.0).max() < 1e-12


@pytest.mark.parametrize("N", [1, 3])
def test_second_order_in_time(N, coupling_cache):
    # Eq. (6) is second order in time: at fixed h and k the step power approaches the exact
    # semi-discrete propagator exp(-t A(k)) with error ~ dt^2.
    n = 16
    h = 1.0 / n
    sa, ss = 0.3, 0.8
    k = [2 * np.pi * 1.0, 2 * np.pi * 2.0, 0.0]
    errs = []
    T = 0.24
    for m in (16, 32, 64, 128):
        dt = T / m
        P = _problem(N, (2, 2, 2), sa, ss, 0.0, h, dt, "periodic", coupling_cache)
        G, A = _symbol(P, k, sa, ss)
        errs.append(np.abs(np.linalg.matrix_power(G, m) - sla.expm(-T * A)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.1), rates


# ----------------------------------------------------------------------------- brute force 4^3
@pytest.fixture(scope="module")
def brute(coupling_cache):
    N, n = 3, 4
    shape = (n, n, n)
    sa, ss = 0.25, 0.6
    P = _problem(N, shape, sa, ss, 0.0, 1.0 / n, 0.3 / n, "periodic", coupling_cache)
    size = P.n_c * n ** 3
    T = np.empty((size, size))
    for j in range(size):
        e = np.zeros(size)
        e[j] = 1.0
        T[:, j] = P.step(e.reshape((P.n_c,) + shape)).ravel()
    return P, T, shape, sa, ss


def test_step_matrix_block_fourier(brute):
    # T maps every mode family {e_b e^{i k . x_a}} by the amplification matrix G(k).
    P, T, shape, sa, ss = brute
    n = shape[0]
    X, Y, Z = _positions(P, shape)
    worst = 0.0
    for kz in range(n):
        for ky in range(n):
            for kx in range(n):
                k = [2 * np.pi * kk / (n * P.h[0]) for kk in (kx, ky, kz)]
                G, _ = _symbol(P, k, sa, ss)
                V = np.zeros((T.shape[0], P.n_c), dtype=complex)
                for a in range(P.n_c):
                    ph = np.exp(1j * (k[0] * X[a] + k[1] * Y[a] + k[2] * Z[a])).ravel()
                    block = np.zeros((P.n_c, ph.size), dtype=complex)
                    block[a] = ph
                    V[:, a] = block.ravel()
                worst = max(worst, np.abs(T @ V - V @ G).max())
    assert worst < 1e-13
    assert np.abs(np.linalg.eigvals(T)).max() <= 1.0 + 1e-12


def test_adjoint_is_transpose(brute):
    # The oracle's discrete adjoint of one step equals the transpose of the brute-force matrix.
    P, T, shape, sa, ss = brute
    rng = np.random.default_rng(7)
    u0 = rng.standard_normal((P.n_c,) + shape)
    lam = rng.standard_normal((P.n_c,) + shape)
    got, *_ = P.backward(u0, 1, lam)
    assert np.abs(got.ravel() - T.T @ lam.ravel()).max() < 1e-13


@pytest.mark.parametrize("bc", ["periodic", "vacuum"])
def test_adjoint_dot_product_and_media_gradient(bc, coupling_cache):
    # <S x, y> = <x, S^T y> for three steps on random media, and the media gradients of
    # J = sum w u_0 agree with central differences.
    N, shape = 3, (4, 5, 6)
    sa, ss, q = synth.random_media(shape, 21)
    P = _problem(N, shape, sa, ss, q, 0.2, 0.05, bc, coupling_cache)
    Pl = _problem(N, shape, sa, ss, 0.0 * q, 0.2, 0.05, bc, coupling_cache)
    rng = np.random.default_rng(22)
    x = rng.standard_normal((P.n_c,) + shape)
    y = rng.standard_normal((P.n_c,) + shape)
    Sx = Pl.run(x, 3)
    STy, *_ = Pl.backward(x, 3, y)
    assert abs(np.vdot(Sx, y) - np.vdot(x, STy)) < 1e-12 * np.abs(Sx).sum()

    w = rng.uniform(0, 1, shape)
    J, g_sa, g_ss, g_q = P.gradient(x, 3, w)
    eps = 1e-6
    for (name, g) in (("sa", g_sa), ("ss", g_ss), ("q", g_q)):
        for cell in [(0, 0, 0), (3, 4, 5), (1, 2, 3)]:
            args = {"sa": sa, "ss": ss, "q": q}
            p, m = dict(args), dict(args)
            p[name] = args[name].copy()
            p[name][cell] += eps
            m[name] = args[name].copy()
            m[name][cell] -= eps
            Jp = np.sum(w * _problem(N, shape, p["sa"], p["ss"], p["q"], 0.2, 0.05, bc,
                                     coupling_cache).run(x, 3)[0])
            Jm = np.sum(w * _problem(N, shape, m["sa"], m["ss"], m["q"], 0.2, 0.05, bc,
                                     coupling_cache).run(x, 3)[0])
            fd = (Jp - Jm) / (2 * eps)
            assert abs(fd - g[cell]) < 1e-7 * max(1.0, abs(fd)), (name, cell, fd, g[cell])


def test_cfl_rejected(coupling_cache):
    with pytest.raises(ValueError):
        _problem(1, (2, 2, 2), 0.0, 0.0, 0.0, 0.3, 0.1, "periodic", coupling_cache)


@pytest.mark.parametrize("N", [3, 7])
def test_anisotropic_scattering_decays_each_order_by_its_own_rate(N, coupling_cache):
    # Section 2: a spatially uniform state has no transport, so each moment of order l >= 1 decays
    # by exp(-(sigma_a + sigma_s - Sigma_sl) t) per step (Sigma_sl = f_l sigma_s) and u_0 by
    # exp(-sigma_a t); here f_l = g^l (a Henyey-Greenstein phase function's moments).
    shape = (3, 4, 5)
    sa, ss, gHG = 0.3, 1.7, 0.6
    f = tuple(gHG ** l for l in range(N + 1))
    mats, slots = coupling_cache(N)
    P = st.Problem(N, np.full(shape, sa), np.full(shape, ss), np.zeros(shape), 0.1, 0.03, "periodic",
                   mats=mats, slots=slots, scat=f)
    rng = np.random.default_rng(3)
    amp = rng.uniform(0.5, 1.5, P.n_c)
    u = np.broadcast_to(amp[:, None, None, None], (P.n_c,) + shape).copy()
    k = 4
    got = P.run(u, k)
    t = k * P.dt
    for a in range(P.n_c):
        l = int(np.sqrt(a))
        rate = sa if a == 0 else sa + (1.0 - f[l]) * ss
        assert np.abs(got[a] - amp[a] * np.exp(-rate * t)).max() <= 1e-13 * amp[a]


def test_isotropic_scattering_moments_reproduce_the_isotropic_step(coupling_cache):
    # f_l = 0 for l >= 1 is isotropic scattering: the same step to the last bit
    N, shape = 3, (4, 5, 6)
    rng = np.random.default_rng(8)
    sa, ss, q = rng.uniform(0, 2, shape), rng.uniform(0, 2, shape), rng.uniform(0, 1, shape)
    mats, slots = coupling_cache(N)
    u = rng.standard_normal(((N + 1) ** 2,) + shape)
    a = st.Problem(N, sa, ss, q, 0.1, 0.03, "vacuum", mats=mats, slots=slots)
    b = st.Problem(N, sa, ss, q, 0.1, 0.03, "vacuum", mats=mats, slots=slots,
                   scat=(1.0,) + (0.0,) * N)
    assert np.array_equal(a.run(u, 3), b.run(u, 3))


def test_dE_matches_extended_precision():
    # E'(x) of Eq. (5)'s E(x) = (e^x - 1)/x enters the adjoint's dbeta/dc = -tau^2 E'(-c tau).  Pinned
    # against the closed form evaluated with 60 significant digits (no cancellation left at that
    # precision), over the arguments -c tau the media produce (c tau from 1e-14 to 50) and a few
    # positive ones: relative error <= 2e-15 everywhere, including 1e-3 <= |x| <= 1, where the FP64
    # closed form itself loses up to 1e-10.
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    xs = np.concatenate([-np.logspace(-14, 1.7, 300), np.logspace(-14, 0.5, 60), [0.0, -1.0, 1.0]])
    got = st._dE(xs)
    for x, g in zip(xs, got):
        X = mpmath.mpf(float(x))
        ref = mpmath.mpf(1) / 2 if X == 0 else (mpmath.exp(X) * (X - 1) + 1) / X**2
        assert abs((mpmath.mpf(float(g)) - ref) / ref) <= 2e-15, x


# ----------------------------------------------------------------------------- merged schedule
def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("bc", ["periodic", "vacuum"])
def test_two_odd_half_steps_are_one_odd_full_step(bc, coupling_cache):
    # With the even class frozen the residual r of the odd class does not change, and Eq. (5)
    # composes exactly: exp(-c t/2)^2 = exp(-c t) and (t/2) E(-c t/2) (1 + exp(-c t/2)) = t E(-c t).
    # Media with sigma near 0 and up to 10 cover both ends of E.
    shape = (4, 5, 6)
    sa, ss, q = synth.random_media(shape, 31, 0.0, 10.0)
    sa[0, 0, :] = 0.0
    ss[0, 0, :3] = 0.0
    P = _problem(7, shape, sa, ss, q, 0.1, 0.03, bc, coupling_cache)
    u = synth.random_state(7, shape, 32)
    halves = P.substep(P.substep(u, 1, 0.5 * P.dt), 1, 0.5 * P.dt)
    full = P.substep(u, 1, P.dt)
    assert _rel(halves, full) <= 1e-13


def _merged_segments(P, u, k, m):
    # the library's merged form of k steps, in segments of at most m steps: odd half pass, then
    # even and odd full passes, closing with an even full pass and an odd half pass per segment
    s = 0
    while s < k:
        n = min(m, k - s)
        u = P.substep(u, 1, 0.5 * P.dt)
        for j in range(n):
            u = P.substep(u, 0, P.dt)
            u = P.substep(u, 1, P.dt if j < n - 1 else 0.5 * P.dt)
        s += n
    return u


@pytest.mark.parametrize("k,m", [(5, 5), (7, 3), (4, 1)])
def test_merged_schedule_equals_eq6(k, m, coupling_cache):
    # Eq. (6) taken literally (three substeps per step) against its merged form, whole or cut into
    # segments (the step kernels' schedule, and the staged adjoint's)
    shape = (5, 4, 6)
    sa, ss, q = synth.random_media(shape, 33, 0.0, 4.0)
    P = _problem(5, shape, sa, ss, q, 0.1, 0.03, "vacuum", coupling_cache)
    u = synth.random_state(5, shape, 34)
    assert _rel(_merged_segments(P, u, k, m), P.run(u, k)) <= 1e-13
