"""Mistakes planted in the oracle, one at a time, on the CPU: each must be caught by a pin that the
unmodified oracle passes (the Fourier symbol of the staggered step, Section 2.1 and Eq. 6, on
non-cubic cells; the closed-form decay of a uniform state, Eq. 5 and Section 2; for the basis and
coupling of Section 2, orthonormality, the P1 wave speeds and the Gauss nodes of the m = 0 block of
Mz).  This shows the pins fix the oracle's arithmetic, not only its shape."""
import math

import numpy as np
import pytest
import scipy.special as sps

from oracle import sh, stepper as st
from test_oracle_step import _positions, _symbol

H = (0.1, 0.13, 0.17)
DT = 0.03
SHAPE = (8, 6, 10)


def _fourier_error(mats, slots, N=3, kint=(1, 2, 3), steps=3, oracle_mats=None):
    """max |oracle - closed form| for one Fourier mode; the symbol comes from the unmodified
    coupling matrices `mats`, the oracle runs with `oracle_mats` (default `mats`) and whatever is
    patched in."""
    sa, ss = 0.2, 0.7
    z = np.zeros(SHAPE)
    P = st.Problem(N, z + sa, z + ss, z, H, DT, "periodic", mats=mats if oracle_mats is None else oracle_mats,
                   slots=slots)
    n = (SHAPE[2], SHAPE[1], SHAPE[0])
    k = [2 * np.pi * kint[d] / (n[d] * H[d]) for d in range(3)]
    ref = st.Problem(N, z + sa, z + ss, z, H, DT, "periodic", mats=tuple(m.copy() for m in mats),
                     slots=slots)
    G, _ = _symbol(ref, k, sa, ss)
    rng = np.random.default_rng(11)
    uh = rng.standard_normal(P.n_c) + 1j * rng.standard_normal(P.n_c)
    X, Y, Z = _positions(ref, SHAPE)
    phase = np.array([np.exp(1j * (k[0] * X[a] + k[1] * Y[a] + k[2] * Z[a])) for a in range(P.n_c)])
    got = P.run(np.real(uh[:, None, None, None] * phase), steps)
    want = np.real((np.linalg.matrix_power(G, steps) @ uh)[:, None, None, None] * phase)
    return float(np.abs(got - want).max())


def _decay_error(mats, slots, N=3, scat=None):
    """max relative deviation of a uniform state from its closed-form per-order decay."""
    sa, ss = 0.3, 1.7
    shape = (3, 4, 5)
    P = st.Problem(N, np.full(shape, sa), np.full(shape, ss), np.zeros(shape), 0.1, DT, "periodic",
                   mats=mats, slots=slots, scat=scat)
    amp = np.random.default_rng(3).uniform(0.5, 1.5, P.n_c)
    got = P.run(np.broadcast_to(amp[:, None, None, None], (P.n_c,) + shape).copy(), 4)
    t = 4 * DT
    f = scat if scat is not None else (1.0,) + (0.0,) * N
    err = 0.0
    for a in range(P.n_c):
        l = int(np.sqrt(a))
        rate = sa if a == 0 else sa + (1.0 - f[l]) * ss
        err = max(err, float(np.abs(got[a] - amp[a] * np.exp(-rate * t)).max() / amp[a]))
    return err


def _swap_direction(self, u_b, target_slot, d):
    if target_slot != 2:
        return (st.shift(u_b, d, +1, self.bc) - u_b) / self.h[d]
    return (u_b - st.shift(u_b, d, -1, self.bc)) / self.h[d]


def _no_h(self, u_b, target_slot, d):
    if target_slot == 2:
        return st.shift(u_b, d, +1, self.bc) - u_b
    return u_b - st.shift(u_b, d, -1, self.bc)


def _h_of_x_everywhere(self, u_b, target_slot, d):
    if target_slot == 2:
        return (st.shift(u_b, d, +1, self.bc) - u_b) / self.h[0]
    return (u_b - st.shift(u_b, d, -1, self.bc)) / self.h[0]


def _classes_swapped(self, u):
    u = self.substep(u, 0, 0.5 * self.dt)
    u = self.substep(u, 1, self.dt)
    return self.substep(u, 0, 0.5 * self.dt)


def _full_odd_steps(self, u):
    u = self.substep(u, 1, self.dt)
    u = self.substep(u, 0, self.dt)
    return self.substep(u, 1, self.dt)


def _explicit_euler(self, u, cls, tau):
    out = u.copy()
    for a in np.nonzero(self.cls == cls)[0]:
        out[a] = u[a] + tau * (self.residual(u, a) - self.c[a] * u[a])
    return out


def _dropped_source_term(self, u, a):
    r = np.zeros(u.shape[1:])
    for d in range(3):
        row = self.mats[d][a]
        for b in np.nonzero(row)[0][:-1]:  # the last coupling of every row is lost
            r -= row[b] * self.derivative(u[b], self.slots[a, d], d)
    return r


FOURIER_MUTATIONS = [
    ("difference direction swapped", "derivative", _swap_direction),
    ("1/h dropped", "derivative", _no_h),
    ("one cell size for every axis", "derivative", _h_of_x_everywhere),
    ("half steps on the even class", "step", _classes_swapped),
    ("odd substeps of full length", "step", _full_odd_steps),
    ("Eq. 5 replaced by an explicit Euler step", "substep", _explicit_euler),
    ("a coupling term dropped", "residual", _dropped_source_term),
]


def test_unmodified_oracle_passes_both_checks(coupling_cache):
    mats, slots = coupling_cache(3)
    assert _fourier_error(mats, slots) < 1e-13
    assert _decay_error(mats, slots) < 1e-13
    assert _decay_error(mats, slots, scat=tuple(0.6 ** l for l in range(4))) < 1e-13


@pytest.mark.parametrize("name,attr,fn", FOURIER_MUTATIONS, ids=[m[0] for m in FOURIER_MUTATIONS])
def test_planted_stepping_mistake_is_caught(coupling_cache, monkeypatch, name, attr, fn):
    mats, slots = coupling_cache(3)
    monkeypatch.setattr(st.Problem, attr, fn)
    assert _fourier_error(mats, slots) > 1e-6, name


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_planted_sign_error_in_a_coupling_matrix_is_caught(coupling_cache, axis):
    # the oracle runs with one M_d negated; the symbol keeps the true matrices
    mats, slots = coupling_cache(3)
    bad = tuple(-m if d == axis else m for d, m in enumerate(mats))
    assert _fourier_error(mats, slots, oracle_mats=bad) > 1e-6


@pytest.mark.parametrize("mistake", ["u_0 decays with sigma_s too", "per-order scattering ignored"])
def test_planted_collision_mistake_is_caught(coupling_cache, monkeypatch, mistake):
    mats, slots = coupling_cache(3)
    scat = None
    if mistake == "u_0 decays with sigma_s too":
        orig = st.Problem._collision

        def bad(self):
            c = orig(self)
            c[0] = st.point_average(self.sigma_a + self.sigma_s, (1, 1, 1), self.bc)
            return c

        monkeypatch.setattr(st.Problem, "_collision", bad)
    else:
        scat = tuple(0.6 ** l for l in range(4))
        orig_init = st.Problem.__post_init__

        def bad_init(self):
            self.scat = None
            orig_init(self)

        monkeypatch.setattr(st.Problem, "__post_init__", bad_init)
    assert _decay_error(mats, slots, scat=scat) > 1e-6, mistake


# ---------------------------------------------------------------- basis and coupling (Section 2)
def _basis_checks(N=3):
    """(Gram error, P1 wave-speed error, Gauss-node error of the m = 0 block of Mz)."""
    g = float(np.abs(sh.gram(N) - np.eye((N + 1) ** 2)).max())
    Mx, My, Mz = sh.coupling(1)
    r3 = 1.0 / math.sqrt(3.0)
    p1 = max(abs(Mx[0, 3] - r3), abs(My[0, 1] - r3), abs(Mz[0, 2] - r3))
    mz = sh.coupling(N)[2]
    idx = [l * l + l for l in range(N + 1)]
    ev = np.sort(np.linalg.eigvalsh(mz[np.ix_(idx, idx)]))
    gw = float(np.abs(ev - np.sort(np.polynomial.legendre.leggauss(N + 1)[0])).max())
    return g, p1, gw


def _real_sh_variant(sqrt2=True, condon_shortley=False, swap_cos_sin=False):
    def real_sh(N, mu, phi):
        mu = np.asarray(mu, dtype=np.float64)
        phi = np.asarray(phi, dtype=np.float64)
        out = np.empty(((N + 1) ** 2,) + mu.shape)
        for c, (l, m) in enumerate(sh.components(N)):
            am = abs(m)
            p = sps.lpmv(am, l, mu) * (1.0 if condon_shortley else (-1.0) ** am)
            k = math.sqrt(2.0) if sqrt2 else 1.0
            cos_t, sin_t = (np.sin, np.cos) if swap_cos_sin else (np.cos, np.sin)
            if m == 0:
                out[c] = sh._norm(l, 0) * p
            elif m > 0:
                out[c] = k * sh._norm(l, am) * p * cos_t(am * phi)
            else:
                out[c] = k * sh._norm(l, am) * p * sin_t(am * phi)
        return out
    return real_sh


def _norm_without_factorials(l, m):
    return math.sqrt((2 * l + 1) / (4.0 * math.pi))


def _coupling_x_y_swapped(N):
    mu, ph, w = sh.quadrature(N)
    Y = sh.real_sh(N, mu, ph)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    mats = []
    for om in (s * np.sin(ph), s * np.cos(ph), mu):
        M = (Y * (w * om)) @ Y.T
        M[np.abs(M) < sh.ZERO_TOL] = 0.0
        mats.append(M)
    return tuple(mats)


_orig_quadrature = sh.quadrature


def _coarse_quadrature(N, extra=2):
    return _orig_quadrature(max(N - 3, 0), 0)


BASIS_MUTATIONS = [
    ("sqrt(2) of the m != 0 functions dropped", "real_sh", _real_sh_variant(sqrt2=False)),
    ("Condon-Shortley phase kept", "real_sh", _real_sh_variant(condon_shortley=True)),
    ("cos and sin types swapped", "real_sh", _real_sh_variant(swap_cos_sin=True)),
    ("(l-m)!/(l+m)! dropped from N_l^m", "_norm", _norm_without_factorials),
    ("Omega_x and Omega_y swapped", "coupling", _coupling_x_y_swapped),
    ("quadrature too coarse to be exact", "quadrature", _coarse_quadrature),
]


def test_unmodified_basis_passes_the_checks():
    assert max(_basis_checks()) < 1e-12


@pytest.mark.parametrize("name,attr,fn", BASIS_MUTATIONS, ids=[m[0] for m in BASIS_MUTATIONS])
def test_planted_basis_mistake_is_caught(monkeypatch, name, attr, fn):
    monkeypatch.setattr(sh, attr, fn)
    assert max(_basis_checks()) > 1e-6, name


# ---------------------------------------------------------------- media points and vacuum boundary
def _interp_error():
    """max deviation of the point mean of a linear field from its value at the staggered point."""
    n = 6
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    sig = 1.0 + 0.5 * x + 0.25 * y + 0.125 * z
    inner = (slice(0, n - 1),) * 3
    err = 0.0
    for slot in [(2, 1, 1), (1, 2, 2), (2, 2, 2)]:
        off = [(g - 1) * 0.5 for g in slot]
        want = 1.0 + 0.5 * (x + off[0]) + 0.25 * (y + off[1]) + 0.125 * (z + off[2])
        err = max(err, float(np.abs(st.point_average(sig, slot, "vacuum")[inner] - want[inner]).max()))
    return err


def _vacuum_error(mats, slots):
    """vacuum run against a periodic run on a padded grid whose padding is zeroed every substep."""
    N, n = 3, 5
    shape, pshape = (n,) * 3, (n + 2,) * 3
    Pv = st.Problem(N, np.full(shape, 0.4), np.full(shape, 0.9), np.full(shape, 0.3), 0.2, 0.06,
                    "vacuum", mats=mats, slots=slots)
    Pp = st.Problem(N, np.full(pshape, 0.4), np.full(pshape, 0.9), np.full(pshape, 0.3), 0.2, 0.06,
                    "periodic", mats=mats, slots=slots)
    u = np.random.default_rng(5).standard_normal((Pv.n_c,) + shape)
    up = np.zeros((Pp.n_c,) + pshape)
    inner = (slice(None),) + (slice(1, n + 1),) * 3
    up[inner] = u
    for _ in range(2):
        u = Pv.step(u)
        for cls, tau in ((1, 0.5 * Pp.dt), (0, Pp.dt), (1, 0.5 * Pp.dt)):
            ring = np.zeros_like(up)
            ring[inner] = up[inner]
            up = Pp.substep(ring, cls, tau)
    return float(np.abs(up[inner] - u).max())


def _point_average_lower_neighbour(sig, slot, bc):
    total = np.array(sig, dtype=np.float64)
    count = np.ones_like(total)
    for d in range(3):
        if slot[d] == 2:
            total = total + st.shift(total, d, -1, bc)
            count = count + st.shift(count, d, -1, bc)
    return total / count


_orig_shift = st.shift


def _shift_wraps_always(f, d, s, bc):
    return _orig_shift(f, d, s, st.PERIODIC)


def test_unmodified_media_and_boundary_pass(coupling_cache):
    mats, slots = coupling_cache(3)
    assert _interp_error() < 1e-14
    assert _vacuum_error(mats, slots) < 1e-14


def test_planted_interpolation_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(st, "point_average", _point_average_lower_neighbour)
    assert _interp_error() > 1e-6


def test_planted_vacuum_mistake_is_caught(coupling_cache, monkeypatch):
    mats, slots = coupling_cache(3)
    monkeypatch.setattr(st, "shift", _shift_wraps_always)
    assert _vacuum_error(mats, slots) > 1e-6


def _dE_closed_form_near_zero(x):
    """E'(x) by the closed form down to |x| = 1e-3 (the cancellation the series avoids)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-3
    xs = x[small]
    out[small] = 0.5 + xs / 3.0 + xs**2 / 8.0 + xs**3 / 30.0 + xs**4 / 144.0
    xl = x[~small]
    out[~small] = (np.exp(xl) * (xl - 1.0) + 1.0) / (xl * xl)
    return out


def test_planted_inaccurate_dE_is_caught(monkeypatch):
    # the extended-precision pin of E' (Eq. 5) catches the closed form evaluated near zero
    from test_oracle_step import test_dE_matches_extended_precision

    pytest.importorskip("mpmath")
    monkeypatch.setattr(st, "_dE", _dE_closed_form_near_zero)
    with pytest.raises(AssertionError):
        test_dE_matches_extended_precision()
