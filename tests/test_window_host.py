"""The register-window kernel's per-cell body compiled for the host (nvcc, no GPU) and run over
bounds-checked memory: one substep of either class against the oracle's substep, for N up to 15,
both boundaries, full and half steps, FP32 and BF16 storage, down to one cell, cubic and
non-cubic cells (the body's scaled form), isotropic and anisotropic scattering (its per-order
factor planes, Section 2)."""
import os
import subprocess

import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import synth

from test_fused_host import CSRC, HERE, ROOT, _bf16_round, _nvcc


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("window_host") / "emulate_window")
    cmd = [nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           os.path.join(HERE, "host", "emulate_window.cu"), os.path.join(CSRC, "model.cpp"), "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    return exe


CASES = [
    # N, shape (nz, ny, nx), bc, target class, half step, storage[, (hy / h, hz / h)[, g: f_l = g^l]]
    (1, (5, 4, 7), "periodic", 0, 0, "fp32"),
    (3, (5, 4, 7), "vacuum", 0, 0, "fp32", (1.3, 1.7)),
    (7, (4, 5, 6), "periodic", 1, 1, "fp32", (1.7, 1.3)),
    (15, (3, 4, 5), "vacuum", 1, 0, "fp32", (1.3, 1.3)),
    (7, (4, 4, 4), "vacuum", 0, 0, "bf16", (1.25, 2.0)),
    (3, (5, 4, 7), "periodic", 0, 0, "fp32", (1.0, 1.0), 0.6),
    (7, (4, 5, 6), "vacuum", 1, 1, "fp32", (1.0, 1.0), -0.4),
    (15, (3, 4, 5), "periodic", 0, 0, "fp32", (1.3, 1.7), 0.85),
    (7, (4, 4, 4), "periodic", 1, 0, "bf16", (1.0, 1.0), 0.5),
    (3, (5, 4, 7), "vacuum", 1, 0, "fp32"),
    (3, (3, 6, 5), "vacuum", 1, 1, "fp32"),
    (7, (5, 4, 7), "periodic", 1, 0, "fp32"),
    (7, (5, 4, 7), "vacuum", 0, 0, "fp32"),
    (7, (4, 4, 4), "periodic", 1, 1, "bf16"),
    (15, (3, 4, 5), "vacuum", 0, 0, "fp32"),
    (15, (3, 4, 5), "periodic", 1, 1, "fp32"),
    (3, (1, 1, 1), "periodic", 0, 0, "fp32"),
]


@pytest.mark.parametrize("case", CASES)
def test_window_body_on_host_vs_oracle(emulator, tmp_path, case):
    N, shape, bc, cls, half, prec = case[:6]
    inst, u = synth.random_instance(N, shape, seed=600 + N, bc=bc)
    nz, ny, nx = shape
    # non-cubic cells: h along x, h_y, h_z as given (dt stays below min(h) / 3)
    h3 = (inst.h, inst.h * case[6][0], inst.h * case[6][1]) if len(case) > 6 else None
    g = case[7] if len(case) > 7 else None
    scat = tuple(g ** l for l in range(N + 1)) if g is not None else None
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    np.concatenate([u.ravel(), inst.sigma_a.ravel(), inst.sigma_s.ravel(), inst.q.ravel()]).tofile(fin)
    extra = [repr(h3[1]), repr(h3[2])] if h3 else []
    if g is not None:
        extra.append(repr(g))
    res = subprocess.run([emulator, str(N), str(cls), str(nx), str(ny), str(nz),
                          str(0 if bc == "periodic" else 1), repr(inst.h), repr(inst.dt), str(half),
                          prec, fin, fout] + extra, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    got = np.fromfile(fout).reshape(u.shape)
    P = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, h3 if h3 and h3[1:] != (inst.h, inst.h) else inst.h,
                   inst.dt, bc, scat=scat)
    u_in = u.astype(np.float32).astype(np.float64) if prec == "fp32" else _bf16_round(u)
    ref = P.substep(u_in, cls, 0.5 * inst.dt if half else inst.dt)
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    assert np.isfinite(got).all()
    assert err <= (1e-5 if prec == "fp32" else 2e-2), err
