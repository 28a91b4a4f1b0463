"""The fused step kernel's phases compiled for the host (nvcc, no GPU) and run over bounds-checked
memory: one pass (even full step, then the odd step) against the oracle's two substeps, on grids
with ragged 32 x 8 tiles, several z chunks, one cell, both boundaries, FP32 and BF16 storage."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2004_02833_gb300", "csrc")


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fused_host") / "emulate_fused")
    cmd = [nvcc, "-std=c++17", "-O1", "-diag-suppress", "20011", "-I", os.path.join(ROOT, "include"),
           "-I", CSRC, os.path.join(HERE, "host", "emulate_fused.cu"), os.path.join(CSRC, "model.cpp"),
           "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    return exe


def _bf16_round(u):
    # round to nearest even at 8 mantissa bits (the storage rounding of the input state)
    b = np.asarray(u, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


CASES = [
    # N, shape (nz, ny, nx), bc, odd half step, storage, planes per z chunk
    (1, (4, 12, 70), "periodic", 1, "fp32", 1),
    (3, (7, 17, 40), "vacuum", 1, "fp32", 3),
    (5, (5, 9, 35), "periodic", 0, "fp32", 2),
    (7, (5, 9, 35), "vacuum", 0, "fp32", 2),
    (7, (3, 4, 5), "periodic", 1, "fp32", 4),
    (7, (1, 1, 1), "periodic", 0, "fp32", 1),
    (9, (3, 9, 33), "vacuum", 0, "fp32", 2),
    (5, (6, 8, 32), "periodic", 0, "bf16", 5),
]


@pytest.mark.parametrize("N,shape,bc,half,prec,zc", CASES)
def test_fused_phases_on_host_vs_oracle(emulator, tmp_path, N, shape, bc, half, prec, zc):
    inst, u = synth.random_instance(N, shape, seed=500 + N, bc=bc)
    nz, ny, nx = shape
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    np.concatenate([u.ravel(), inst.sigma_a.ravel(), inst.sigma_s.ravel(), inst.q.ravel()]).tofile(fin)
    res = subprocess.run([emulator, str(N), str(zc), str(nx), str(ny), str(nz),
                          str(0 if bc == "periodic" else 1), repr(inst.h), repr(inst.dt), str(half),
                          prec, fin, fout], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    got = np.fromfile(fout).reshape(u.shape)
    P = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, bc)
    u_in = u.astype(np.float32).astype(np.float64) if prec == "fp32" else _bf16_round(u)
    ref = P.substep(P.substep(u_in, 0, inst.dt), 1, 0.5 * inst.dt if half else inst.dt)
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    # FP32: the method's FP32 bound; BF16: two passes of storage rounding (2^-9 each) plus FP32
    assert np.isfinite(got).all()
    assert err <= (1e-5 if prec == "fp32" else 2e-2), err
