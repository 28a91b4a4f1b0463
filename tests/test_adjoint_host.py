"""The staged adjoint's per-cell arithmetic compiled for the host (nvcc, no GPU) and run over
bounds-checked memory: the factor derivatives of Eq. (5) and the pull-back through one pass,
which recovers the pass's residual from its stored pre- and post-pass states instead of re-running
the stencil, against the oracle's discrete adjoint of that substep: the media-gradient sums per
sub-grid slot and for u_0, dJ/dq, w = beta lam, with and without a pending factor applied first.
FP32 states and factors; the bound 1e-5 of each field's largest value (the FP32 bound of the
adjoint tests, for one pass)."""
import os
import subprocess

import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import synth

from test_fused_host import CSRC, HERE, ROOT, _nvcc


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("pull_host") / "emulate_pull")
    cmd = [nvcc, "-std=c++17", "-O1", "-diag-suppress", "20011", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           os.path.join(HERE, "host", "emulate_pull.cu"), os.path.join(CSRC, "model.cpp"), "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    return exe


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


CASES = [
    # N, shape (nz, ny, nx), bc, class of the pass, half step, pending factor (-1 none, 0 dt, 1 dt/2)
    (3, (4, 5, 8), "vacuum", 0, 0, -1),
    (3, (3, 4, 8), "periodic", 1, 1, -1),
    (7, (4, 5, 4), "periodic", 1, 1, 1),
    (7, (3, 4, 8), "vacuum", 0, 0, 0),
    (15, (2, 3, 4), "vacuum", 1, 0, -1),
]


@pytest.mark.parametrize("N,shape,bc,cls,half,pre", CASES)
def test_pull_back_on_host_vs_oracle(emulator, tmp_path, N, shape, bc, cls, half, pre):
    inst, u = synth.random_instance(N, shape, seed=1800 + N, bc=bc)
    lam = np.random.default_rng(1801 + N).standard_normal(u.shape)
    P = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, bc)
    tau = 0.5 * inst.dt if half else inst.dt
    upre = f32(u)
    upost = f32(P.substep(upre, cls, tau))
    lam32 = f32(lam)
    nz, ny, nx = shape
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    np.concatenate([upre.ravel(), upost.ravel(), lam32.ravel(), inst.sigma_a.ravel(), inst.sigma_s.ravel(),
                    inst.q.ravel()]).tofile(fin)
    res = subprocess.run([emulator, str(N), str(cls), str(nx), str(ny), str(nz), str(0 if bc == "periodic" else 1),
                          repr(inst.h), repr(inst.dt), str(half), str(pre), fin, fout],
                         capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    n_c, V = u.shape[0], nz * ny * nx
    out = np.fromfile(fout)
    w = out[:n_c * V].reshape(u.shape)
    lam_out = out[n_c * V:2 * n_c * V].reshape(u.shape)
    gacc = out[2 * n_c * V:(2 * n_c + 9) * V].reshape((9,) + shape)
    gq = out[(2 * n_c + 9) * V:].reshape(shape)

    m = P.cls == cls
    lam_eff = lam32.copy()
    if pre >= 0:  # the pending factor of the class, applied first (u_0's own at dt)
        fa = np.exp(-P.c * (0.5 * inst.dt if pre else inst.dt))
        fa[0] = np.exp(-P.c[0] * inst.dt)
        lam_eff[m] = fa[m] * lam32[m]
    grads = {"c": np.zeros_like(P.c), "q": np.zeros_like(P.q)}
    P.substep_adjoint(upre, lam_eff, cls, tau, grads)
    beta = tau * st.E(-P.c * tau)
    beta[0] = inst.dt * st.E(-P.c[0] * inst.dt)  # u_0 (class 0) always takes the full step
    # the media-gradient sums per sub-grid slot code (u_0 apart) and for u_0
    code = (P.slots[:, 0] - 1) + 2 * (P.slots[:, 1] - 1) + 4 * (P.slots[:, 2] - 1)
    want = np.zeros((9,) + shape)
    for a in np.nonzero(m)[0]:
        want[8 if a == 0 else code[a]] += grads["c"][a]
    scale = np.abs(want).max()
    assert scale > 0 and np.abs(gacc - want).max() <= 1e-5 * scale
    if cls == 0:
        assert np.abs(gq - grads["q"]).max() <= 1e-5 * np.abs(grads["q"]).max()
    else:
        assert not np.any(gq)
    assert np.abs(w[m] - (beta * lam_eff)[m]).max() <= 1e-6 * np.abs(beta * lam_eff)[m].max()
    assert not np.any(w[~m])
    # lam: the class scaled by a pending factor where one was given, else untouched
    assert np.abs(lam_out - lam_eff).max() <= 1e-6 * np.abs(lam_eff).max()
