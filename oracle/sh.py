"""Real spherical harmonics, the P_N coupling matrices and the sub-grid placement.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows Section 2 of the paper:
  * moments psi_l^m = int conj(Y_l^m) psi dOmega with
    Y_l^m = (-1)^m sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) e^{i m phi} P_l^m(mu)  (Section 2, after Eq. 2);
  * the real-valued 3D system  u_t + Mx u_x + My u_y + Mz u_z + C u = q  (Eq. 3), whose symmetric
    sparse matrices are  M_d[a, b] = int_{S^2} Omega_d Y_a Y_b dOmega  in a real orthonormal basis;
  * the staggered placement of Section 2.1: u_0 lives on G111 and a derivative along axis d of a
    component on a (1,.,.) grid updates a component on the matching (2,.,.) grid and vice versa.

Readings of what the paper leaves open (the "appropriate substitutions" to a real basis):
  * polar axis z, mu = cos(theta) = Omega_z, Omega = (sqrt(1-mu^2) cos phi, sqrt(1-mu^2) sin phi, mu);
  * real basis without the Condon-Shortley phase:
        m > 0 : sqrt(2) N_l^m P_l^m(mu) cos(m phi)
        m = 0 : N_l^0 P_l(mu)
        m < 0 : sqrt(2) N_l^|m| P_l^|m|(mu) sin(|m| phi)
    with P_l^m(mu) = (1-mu^2)^{m/2} d^m/dmu^m P_l(mu) (no (-1)^m) and N_l^m the factor above;
  * component index c = l*l + l + m, l = 0..N, m = -l..l;
  * entries with |value| < 1e-10 are exact zeros of the integral and are set to 0 (at N = 39 the
    rule leaves ~1e-13 of rounding on them, while the smallest true entry is ~9e-3).

The integrals are evaluated by a product rule that is exact for the integrands: Gauss-Legendre in
mu (the mu-part is a polynomial of degree <= 2N+2) times the uniform rule in phi (a trigonometric
polynomial of degree <= 2N+1).  The associated Legendre functions come from scipy.special.lpmv
(a library routine; its Condon-Shortley sign is removed here).
"""
from __future__ import annotations

import math
from collections import deque
from fractions import Fraction

import numpy as np
import scipy.special as sps


ZERO_TOL = 1e-10


def components(N: int) -> list[tuple[int, int]]:
    """(l, m) of every component in the index order c = l*l + l + m (Section 2)."""
    return [(l, m) for l in range(N + 1) for m in range(-l, l + 1)]


def _norm(l: int, m: int) -> float:
    """N_l^m = sqrt((2l+1)/(4 pi) * (l-m)!/(l+m)!) for m >= 0 (Section 2)."""
    ratio = Fraction(math.factorial(l - m), math.factorial(l + m))
    return math.sqrt((2 * l + 1) / (4.0 * math.pi) * float(ratio))


def real_sh(N: int, mu: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics, shape (n_c, *mu.shape), order c = l*l + l + m."""
    mu = np.asarray(mu, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    out = np.empty(((N + 1) ** 2,) + mu.shape, dtype=np.float64)
    for c, (l, m) in enumerate(components(N)):
        am = abs(m)
        # scipy's lpmv carries the Condon-Shortley factor (-1)^m; the basis here does not.
        p = (-1.0) ** am * sps.lpmv(am, l, mu)
        if m == 0:
            out[c] = _norm(l, 0) * p
        elif m > 0:
            out[c] = math.sqrt(2.0) * _norm(l, am) * p * np.cos(am * phi)
        else:
            out[c] = math.sqrt(2.0) * _norm(l, am) * p * np.sin(am * phi)
    return out


def quadrature(N: int, extra: int = 2) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Product rule on S^2 exact for the integrands of degree <= 2N+2: nodes (mu, phi), weights."""
    n_mu = N + 2 + extra
    n_phi = 2 * N + 4 + 2 * extra
    x, w = np.polynomial.legendre.leggauss(n_mu)
    ph = 2.0 * math.pi * np.arange(n_phi) / n_phi
    MU, PH = np.meshgrid(x, ph, indexing="ij")
    W = np.outer(w, np.full(n_phi, 2.0 * math.pi / n_phi))
    return MU.ravel(), PH.ravel(), W.ravel()


def gram(N: int) -> np.ndarray:
    """int Y_a Y_b dOmega by the same product rule (must be the identity)."""
    mu, ph, w = quadrature(N)
    Y = real_sh(N, mu, ph)
    return (Y * w) @ Y.T


def coupling(N: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Mx, My, Mz of Eq. (3): M_d[a, b] = int Omega_d Y_a Y_b dOmega (dense, index order c)."""
    mu, ph, w = quadrature(N)
    Y = real_sh(N, mu, ph)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    omegas = (s * np.cos(ph), s * np.sin(ph), mu)
    mats = []
    for om in omegas:
        M = (Y * (w * om)) @ Y.T
        M[np.abs(M) < ZERO_TOL] = 0.0
        mats.append(M)
    return tuple(mats)


def placement(N: int, mats=None) -> np.ndarray:
    """Sub-grid slot (1 or 2) of every component along x, y, z; shape (n_c, 3).

    Section 2.1: u_0 sits on G111; a nonzero M_d[a, b] means a d-derivative of b updates a, so
    a and b sit on grids that differ exactly in slot d.  The slots are propagated from u_0 over
    the coupling graph; a conflict (a placement that is not possible) raises.
    """
    if mats is None:
        mats = coupling(N)
    n = (N + 1) ** 2
    slots = np.zeros((n, 3), dtype=np.int64)
    slots[0] = (1, 1, 1)
    seen = np.zeros(n, dtype=bool)
    seen[0] = True
    queue = deque([0])
    while queue:
        a = queue.popleft()
        for d, M in enumerate(mats):
            for b in np.nonzero(M[a])[0]:
                want = slots[a].copy()
                want[d] = 3 - want[d]
                if seen[b]:
                    if not np.array_equal(slots[b], want):
                        raise ValueError(f"placement conflict at component {b}")
                else:
                    slots[b] = want
                    seen[b] = True
                    queue.append(b)
    if not seen.all():
        raise ValueError("coupling graph does not reach every component")
    return slots


def parity_class(slots: np.ndarray) -> np.ndarray:
    """0 for the 'even' grids G111, G221, G122, G212 and 1 for the 'odd' ones (Section 2.1)."""
    return (np.sum(slots == 2, axis=1) % 2).astype(np.int64)
