"""Pins of the oracle's basis, coupling matrices and placement against facts the paper and the
mathematics fix (not against the oracle's own formulas)."""
import math

import os

import numpy as np
import pytest

from oracle import sh

ORDERS = [1, 3, 7, 15]


def _idx(l, m):
    return l * l + l + m


@pytest.mark.parametrize("N", ORDERS + [39])
def test_basis_orthonormal(N):
    # Section 2: the moments are taken against an orthonormal SH basis.
    G = sh.gram(N)
    assert np.abs(G - np.eye(len(G))).max() < 1e-12


@pytest.mark.parametrize("N", ORDERS)
def test_coupling_symmetric(coupling_cache, N):
    # Eq. (3): "the symmetric system matrices Mx, My, Mz".
    (mats, _) = coupling_cache(N)
    for M in mats:
        assert np.array_equal(M != 0, M.T != 0)
        assert np.abs(M - M.T).max() < 1e-14


@pytest.mark.parametrize("N", ORDERS)
def test_mz_m0_block_is_paper_recursion(coupling_cache, N):
    # Section 2 (slab P_N): d_x of (l+1)/(2l+1) psi_{l+1} + l/(2l+1) psi_{l-1}.  The m = 0 block of Mz
    # in the orthonormal basis is that tridiagonal matrix after the scaling psi_l ~ u_l / sqrt(2l+1).
    (mats, _) = coupling_cache(N)
    Mz = mats[2]
    idx = [_idx(l, 0) for l in range(N + 1)]
    B = Mz[np.ix_(idx, idx)]
    s = np.sqrt(2.0 * np.arange(N + 1) + 1.0)
    T = (B / s[:, None]) * s[None, :]
    want = np.zeros_like(T)
    for l in range(N + 1):
        if l + 1 <= N:
            want[l, l + 1] = (l + 1) / (2 * l + 1)
        if l - 1 >= 0:
            want[l, l - 1] = l / (2 * l + 1)
    assert np.abs(T - want).max() < 1e-14


@pytest.mark.parametrize("N", ORDERS)
def test_mz_m0_eigenvalues_are_gauss_nodes(coupling_cache, N):
    # Golub-Welsch: the symmetric Jacobi matrix of the Legendre recurrence has the N+1 Gauss nodes
    # as eigenvalues (the P_N wave speeds along z).
    (mats, _) = coupling_cache(N)
    idx = [_idx(l, 0) for l in range(N + 1)]
    ev = np.sort(np.linalg.eigvalsh(mats[2][np.ix_(idx, idx)]))
    nodes, _ = np.polynomial.legendre.leggauss(N + 1)
    assert np.abs(ev - np.sort(nodes)).max() < 1e-13


@pytest.mark.parametrize("N", ORDERS)
def test_rotation_invariance(coupling_cache, N):
    # P_N preserves rotational invariance (Section 1): Mx, My, Mz are similar (same spectrum).
    (mats, _) = coupling_cache(N)
    ev = [np.sort(np.linalg.eigvalsh(M)) for M in mats]
    assert np.abs(ev[0] - ev[2]).max() < 1e-12
    assert np.abs(ev[1] - ev[2]).max() < 1e-12


def test_p1_wave_speed(coupling_cache):
    # P1: int Omega_d Y_00 Y_1 = 1/sqrt(3) for the Y_1 aligned with axis d.
    (mats, _) = coupling_cache(1)
    Mx, My, Mz = mats
    r3 = 1.0 / math.sqrt(3.0)
    assert abs(Mx[0, _idx(1, 1)] - r3) < 1e-15
    assert abs(My[0, _idx(1, -1)] - r3) < 1e-15
    assert abs(Mz[0, _idx(1, 0)] - r3) < 1e-15
    assert np.count_nonzero(Mx[0]) == np.count_nonzero(My[0]) == np.count_nonzero(Mz[0]) == 1


@pytest.mark.parametrize("N", [7, 15, 39])
def test_row_sparsity_matches_paper(coupling_cache, N):
    # Section 3.2 (unrolled multiplications): rows of Mx and My have one to four nonzeros, rows of
    # Mz zero to two; ten products per row at most.
    (mats, _) = coupling_cache(N)
    nx, ny, nz = [(M != 0).sum(1) for M in mats]
    assert nx.min() == 1 and nx.max() == 4
    assert ny.min() == 1 and ny.max() == 4
    assert nz.min() == 0 and nz.max() == 2
    assert (nx + ny + nz).max() == 10


def test_zero_threshold_gap(coupling_cache):
    # The rule leaves rounding on structural zeros; the drop threshold sits in a wide gap.
    (mats, _) = coupling_cache(39)
    for M in mats:
        assert np.abs(M[M != 0]).min() > 5e-3


def _parity_slots(N):
    """Slots from the reflection parity of each real SH (independent of the coupling matrices):
    x -> -x maps phi -> pi - phi, y -> -y maps phi -> -phi, z -> -z maps mu -> -mu."""
    out = []
    for l, m in sh.components(N):
        am = abs(m)
        if m >= 0:  # cos type (and m = 0)
            px, py = (-1) ** am, 1
        else:       # sin type
            px, py = -((-1) ** am), -1
        pz = (-1) ** (l + am)
        out.append([1 if p == 1 else 2 for p in (px, py, pz)])
    return np.array(out)


@pytest.mark.parametrize("N", ORDERS + [39])
def test_placement(coupling_cache, N):
    # Section 2.1: u_0 on G111; each d-derivative switches slot d; placement always possible.
    (mats, slots) = coupling_cache(N)
    assert tuple(slots[0]) == (1, 1, 1)
    assert np.array_equal(slots, _parity_slots(N))
    for d, M in enumerate(mats):
        a, b = np.nonzero(M)
        diff = slots[a] != slots[b]
        assert diff[:, d].all()
        assert not np.delete(diff, d, axis=1).any()
    # "even" grids G111, G221, G122, G212 hold exactly the even-l components
    ls = np.array([l for l, _ in sh.components(N)])
    even = {(1, 1, 1), (2, 2, 1), (1, 2, 2), (2, 1, 2)}
    is_even = np.array([tuple(s) in even for s in slots])
    assert np.array_equal(is_even, ls % 2 == 0)
    assert np.array_equal(sh.parity_class(slots), ls % 2)


def _printed_flop_model():
    """(N, FLOP per LCUP) as printed in Section 4.1.1 (tests/golden/flop_model.txt)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "flop_model.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return [(int(n), float(v)) for n, v in rows]


@pytest.mark.parametrize("N,printed", _printed_flop_model())
def test_flop_model_class_sizes(coupling_cache, N, printed):
    # Section 4.1.1 prints 392 + 40 v_e + 50 v_o FLOP per cell and 68.3 / 50.5 / 45.1 FLOP/LCUP.  The
    # printed values come out only with 40 per odd-grid and 50 per even-grid component (reading:
    # the two labels are swapped), which pins the class sizes of the placement.
    (mats, slots) = coupling_cache(N)
    cls = sh.parity_class(slots)
    n_even, n_odd = int((cls == 0).sum()), int((cls == 1).sum())
    per = (392 + 40 * n_odd + 50 * n_even) / (N + 1) ** 2
    assert abs(per - printed) <= 0.05 + 1e-9
