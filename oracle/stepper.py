"""Serial FP64 time stepping of the staggered P_N system, written from Section 2.1 of the paper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

State layout: ``u[c, z, y, x]`` in the component order c = l*l + l + m of ``oracle.sh``; cell index
(i, j, k) is 0-based.  A component with slot g = 1 along an axis sits at (i + 1/2) h on that axis, one
with g = 2 at (i + 1) h (the paper's G_{1..} / G_{2..} grids of Section 2.1, shifted to 0-based).

What is computed (paper passage in brackets):
  * half-grid centred differences [Section 2.1, the difference formula before Eq. 4]: for a target a
    and a source b coupled along axis d,
        g_{a,d} = 2 :  D_d u_b(i) = (u_b(i + e_d) - u_b(i)) / h_d
        g_{a,d} = 1 :  D_d u_b(i) = (u_b(i) - u_b(i - e_d)) / h_d ;
  * the frozen-dual scalar ODEs of Eq. (4) solved exactly by Eq. (5),
        u <- u + tau (r - c u) E(-c tau),   r = q_a - sum_d sum_b M_d[a, b] D_d u_b,
        E(x) = (exp(x) - 1) / x,  E(0) = 1;
  * the Strang step of Eq. (6):  S^o_{dt/2} o S^e_{dt} o S^o_{dt/2}, taken literally (no merging);
  * C = diag(c) with c = sigma_a for u_0 and c = sigma_a + sigma_s for every other component
    (Section 2, Sigma_tl with isotropic scattering; "c_k for k >= 1 are identical", Section 3.2);
    q enters the u_0 equation only (isotropic source);
  * anisotropic scattering (optional ``scat``): Section 2's Sigma_tl = Sigma_a + Sigma_s0 -
    Sigma_sl per moment order l, with Sigma_sl = f_l * sigma_s (f_0 = 1, so sigma_s = Sigma_s0):
    c = sigma_a + (1 - f_l) sigma_s for a component of order l.

Readings where the paper is silent:
  * media on staggered points [Section 3.2 says only "interpolated"]: the arithmetic mean of
    sigma over the 2^k cells adjacent to the point (k = number of 2-slots); periodic: indices wrap;
    vacuum: the mean over the in-domain cells only.  c, and from it the substep factors, are
    computed from the averaged sigma;
  * boundaries: periodic [Section 2.1] wraps indices; vacuum (not in the paper) reads every
    out-of-domain value of every component as 0;
  * which class is halved: Eq. (6) literally (odd = odd l, half steps; even = even l incl. u_0).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import sh

PERIODIC = "periodic"
VACUUM = "vacuum"

# array axis of a field f[z, y, x] that carries the physical axis d = 0 (x), 1 (y), 2 (z)
_AX = (2, 1, 0)


def shift(f: np.ndarray, d: int, s: int, bc: str) -> np.ndarray:
    """Values f(i + s e_d) on the cell index grid; periodic wraps, vacuum reads 0 outside."""
    ax = _AX[d]
    if bc == PERIODIC:
        return np.roll(f, -s, axis=ax)
    out = np.zeros_like(f)
    n = f.shape[ax]
    src = [slice(None)] * f.ndim
    dst = [slice(None)] * f.ndim
    if s > 0:
        src[ax] = slice(s, n)
        dst[ax] = slice(0, n - s)
    else:
        src[ax] = slice(0, n + s)
        dst[ax] = slice(-s, n)
    out[tuple(dst)] = f[tuple(src)]
    return out


def point_average(sig: np.ndarray, slot, bc: str) -> np.ndarray:
    """Mean of a per-cell field over the cells adjacent to the staggered point of `slot` (reading)."""
    total = np.array(sig, dtype=np.float64)
    count = np.ones_like(total)
    for d in range(3):
        if slot[d] == 2:
            total = total + shift(total, d, +1, bc)
            count = count + shift(count, d, +1, bc)
    return total / count


def E(x: np.ndarray) -> np.ndarray:
    """E(x) = (exp(x) - 1)/x with E(0) = 1 (Eq. 5); expm1 keeps small |x| accurate."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x != 0.0
    out[nz] = np.expm1(x[nz]) / x[nz]
    return out


@dataclass
class Problem:
    """One P_N instance: order N, per-cell media [z, y, x], spacing, time step, boundary."""

    N: int
    sigma_a: np.ndarray
    sigma_s: np.ndarray
    q: np.ndarray
    h: tuple
    dt: float
    bc: str = PERIODIC
    mats: tuple = field(default=None, repr=False)
    slots: np.ndarray = field(default=None, repr=False)
    scat: tuple = None    # f_l, l = 0..N, of anisotropic scattering (None: isotropic)

    def __post_init__(self):
        self.sigma_a = np.asarray(self.sigma_a, dtype=np.float64)
        self.sigma_s = np.asarray(self.sigma_s, dtype=np.float64)
        self.q = np.asarray(self.q, dtype=np.float64)
        if np.isscalar(self.h):
            self.h = (float(self.h),) * 3
        self.h = tuple(float(v) for v in self.h)
        if self.bc not in (PERIODIC, VACUUM):
            raise ValueError(f"unknown boundary {self.bc}")
        # Section 2.1: convergence is proven for dt < min(h)/3.
        if not self.dt < min(self.h) / 3.0:
            raise ValueError("dt must be below min(h)/3")
        if self.mats is None:
            self.mats = sh.coupling(self.N)
        if self.slots is None:
            self.slots = sh.placement(self.N, self.mats)
        self.cls = sh.parity_class(self.slots)
        if self.scat is not None:
            self.scat = tuple(float(v) for v in self.scat)
            if len(self.scat) != self.N + 1 or self.scat[0] != 1.0:
                raise ValueError("scat holds f_0 = 1, f_1, ..., f_N")
        self.c = self._collision()

    @property
    def n_c(self) -> int:
        return (self.N + 1) ** 2

    def _collision(self) -> np.ndarray:
        """c at each component's own points: sigma_a for u_0, sigma_a + sigma_s otherwise
        (sigma_a + (1 - f_l) sigma_s for a component of order l with anisotropic scattering)."""
        c = np.empty((self.n_c,) + self.sigma_a.shape, dtype=np.float64)
        tot = self.sigma_a + self.sigma_s
        cache = {}
        for a in range(self.n_c):
            key = tuple(self.slots[a])
            if a == 0:
                c[a] = point_average(self.sigma_a, key, self.bc)
                continue
            l = int(np.sqrt(a))  # c = l*l + l + m
            ck = key if self.scat is None else key + (l,)
            if ck not in cache:
                field_ = tot if self.scat is None else self.sigma_a + (1.0 - self.scat[l]) * self.sigma_s
                cache[ck] = point_average(field_, key, self.bc)
            c[a] = cache[ck]
        return c

    def derivative(self, u_b: np.ndarray, target_slot: int, d: int) -> np.ndarray:
        """D_d u_b at the points of a target whose slot along d is `target_slot` (Section 2.1)."""
        if target_slot == 2:
            return (shift(u_b, d, +1, self.bc) - u_b) / self.h[d]
        return (u_b - shift(u_b, d, -1, self.bc)) / self.h[d]

    def residual(self, u: np.ndarray, a: int) -> np.ndarray:
        """r_a = q_a - sum_d sum_b M_d[a, b] D_d u_b  (right-hand side of Eq. 4)."""
        r = self.q.copy() if a == 0 else np.zeros(u.shape[1:])
        for d in range(3):
            row = self.mats[d][a]
            for b in np.nonzero(row)[0]:
                r -= row[b] * self.derivative(u[b], self.slots[a, d], d)
        return r

    def substep(self, u: np.ndarray, cls: int, tau: float) -> np.ndarray:
        """S^{cls}_tau: every component of class `cls` by Eq. (5); the dual class is frozen."""
        out = u.copy()
        for a in np.nonzero(self.cls == cls)[0]:
            r = self.residual(u, a)
            ca = self.c[a]
            out[a] = u[a] + tau * (r - ca * u[a]) * E(-ca * tau)
        return out

    def step(self, u: np.ndarray) -> np.ndarray:
        """One full step of Eq. (6): odd half step, even full step, odd half step."""
        u = self.substep(u, 1, 0.5 * self.dt)
        u = self.substep(u, 0, self.dt)
        return self.substep(u, 1, 0.5 * self.dt)

    def run(self, u: np.ndarray, k: int) -> np.ndarray:
        u = np.array(u, dtype=np.float64)
        for _ in range(k):
            u = self.step(u)
        return u

    # ------------------------------------------------------------------ discrete adjoint
    # The transpose of every substep, written out as its own operation.  A substep on class A is
    #     u_A' = alpha_A u_A + beta_A r_A,   r_A = q_A - sum_d M_d^{AB} D_d u_B,   u_B' = u_B,
    # with alpha = 1 - c tau E(-c tau) = exp(-c tau) and beta = tau E(-c tau) (Eq. 5 rearranged).
    # Given lam' = dJ/du', the pull-back is
    #     lam_A = alpha_A lam'_A,
    #     lam_B = lam'_B - sum_a sum_d M_d[a, b] D_{d,a}^T (beta_a lam'_a),
    # where D^T of a forward difference is the negated backward difference with the same
    # boundary rule (and vice versa), and the media receive
    #     dJ/dc_a += lam'_a (dalpha/dc u_a + dbeta/dc r_a),   dJ/dq += beta_0 lam'_0.

    def derivative_T(self, g: np.ndarray, target_slot: int, d: int) -> np.ndarray:
        """Transpose of `derivative` (same boundary rule)."""
        if target_slot == 2:
            return (shift(g, d, -1, self.bc) - g) / self.h[d]
        return (g - shift(g, d, +1, self.bc)) / self.h[d]

    def substep_adjoint(self, u: np.ndarray, lam: np.ndarray, cls: int, tau: float, grads: dict):
        """Pull lam back through S^{cls}_tau applied to the pre-substep state u; add media grads."""
        out = lam.copy()
        for a in np.nonzero(self.cls == cls)[0]:
            ca = self.c[a]
            x = -ca * tau
            alpha = 1.0 + x * E(x)
            beta = tau * E(x)
            r = self.residual(u, a)
            dalpha = -tau * alpha
            dbeta = -tau * tau * _dE(x)
            grads["c"][a] += lam[a] * (dalpha * u[a] + dbeta * r)
            if a == 0:
                grads["q"] += beta * lam[0]
            out[a] = alpha * lam[a]
            bl = beta * lam[a]
            for d in range(3):
                row = self.mats[d][a]
                for b in np.nonzero(row)[0]:
                    out[b] -= row[b] * self.derivative_T(bl, self.slots[a, d], d)
        return out

    def forward_states(self, u0: np.ndarray, k: int):
        """All substep states of k literal Strang steps and the (class, tau) of each substep."""
        states = [np.array(u0, dtype=np.float64)]
        plan = []
        for _ in range(k):
            for cls, tau in ((1, 0.5 * self.dt), (0, self.dt), (1, 0.5 * self.dt)):
                plan.append((cls, tau))
                states.append(self.substep(states[-1], cls, tau))
        return states, plan

    def backward(self, u0: np.ndarray, k: int, lam_final: np.ndarray):
        """Pull lam_final = dJ/du(after k steps) back to dJ/du(initial) and the media gradients.

        Returns (lam_initial, dJ/dsigma_a, dJ/dsigma_s, dJ/dq).  dJ/dc at every component's points
        is spread to the cells by the transpose of the point averaging.
        """
        states, plan = self.forward_states(u0, k)
        lam = np.array(lam_final, dtype=np.float64)
        grads = {"c": np.zeros_like(self.c), "q": np.zeros_like(self.q)}
        for (cls, tau), u in zip(reversed(plan), reversed(states[:-1])):
            lam = self.substep_adjoint(u, lam, cls, tau, grads)
        g_sa = np.zeros_like(self.sigma_a)
        g_ss = np.zeros_like(self.sigma_s)
        # u_0 sits on G111: its c is the cell's own sigma_a.
        g_sa += point_average_T(grads["c"][0], (1, 1, 1), self.bc)
        for a in range(1, self.n_c):
            g = point_average_T(grads["c"][a], tuple(self.slots[a]), self.bc)
            g_sa += g
            g_ss += g
        return lam, g_sa, g_ss, grads["q"]

    def gradient(self, u0: np.ndarray, k: int, w: np.ndarray):
        """J = sum_cells w * u_0 after k steps; returns (J, dJ/dsigma_a, dJ/dsigma_s, dJ/dq)."""
        if self.scat is not None:
            raise NotImplementedError("the adjoint takes isotropic scattering")
        J = float(np.sum(w * self.run(u0, k)[0]))
        lam = np.zeros((self.n_c,) + self.sigma_a.shape)
        lam[0] = w
        _, g_sa, g_ss, g_q = self.backward(u0, k, lam)
        return J, g_sa, g_ss, g_q


def _dE(x: np.ndarray) -> np.ndarray:
    """E'(x), the derivative of E(x) = (exp(x) - 1)/x of Eq. (5).

    Differentiating the series E(x) = sum_k x^k / (k+1)! gives E'(x) = sum_k (k+1) x^k / (k+2)!,
    summed term by term for |x| < 1 (22 terms: the next is below 1e-21 of the sum); for |x| >= 1
    the closed form (exp(x) (x - 1) + 1) / x^2, whose numerator no longer cancels.  (The closed form
    near 0 loses about eps / x^2 of its value to cancellation: 1e-10 at |x| = 1e-3.)
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1.0
    xs = x[small]
    acc = np.zeros_like(xs)
    term_pow = np.ones_like(xs)
    fact = 2.0  # (k+2)! for k = 0
    for k in range(22):
        acc = acc + (k + 1) * term_pow / fact
        term_pow = term_pow * xs
        fact = fact * (k + 3)
    out[small] = acc
    xl = x[~small]
    out[~small] = (np.exp(xl) * (xl - 1.0) + 1.0) / (xl * xl)
    return out


def point_average_T(g: np.ndarray, slot, bc: str) -> np.ndarray:
    """Transpose of `point_average`: spread g(point)/count to each adjacent cell."""
    ones = np.ones_like(g)
    count = ones.copy()
    for d in range(3):
        if slot[d] == 2:
            count = count + shift(count, d, +1, bc)
    share = g / count
    # each point gathers cells i + {0,1} e_d for the 2-slot axes; its transpose scatters back
    out = share
    for d in range(3):
        if slot[d] == 2:
            out = out + shift(out, d, -1, bc)
    return out
