"""The TMA-staged kernel's stage plan and column work compiled for the host (nvcc, no GPU) and run
over bounds-checked memory: every box the producer would issue is copied as the TMA unit copies
it (zero outside the tensor, x aligned to 16 bytes, inside its region and buffer), the consumers
of each stage run with their rotating accumulator window, CTA by CTA in the kernel's tile walk
with several tiles per CTA, and one pass is compared with the oracle's substep.  Full and partial
tiles, both boundaries, both classes, full and half steps, FP32 and BF16 storage; and the
adjoint's transposed-coupling mode (ADJ_SOURCES, with and without a folded factor) against the
oracle's pull-back through a substep."""
import os
import subprocess

import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import synth

from test_fused_host import CSRC, HERE, ROOT, _bf16_round, _nvcc

VARIANTS = {  # (order, tile x, y, z, stage buffers, box length step), as in stage_variants.h
    7: (7, 32, 2, 2, 4, 1),
    15: (15, 32, 3, 3, 3, 1),
    39: (39, 40, 2, 2, 2, 1),
}


@pytest.fixture(scope="module")
def emulators(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("stage_host")
    out = {}
    for key, (n, tx, ty, tz, nb, eq) in VARIANTS.items():
        exe = str(d / f"emulate_stage_{key}")
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1", "-diag-suppress", "20011",
               "-I", os.path.join(ROOT, "include"), "-I", CSRC, f"-DRTPN_SN={n}", f"-DRTPN_STX={tx}",
               f"-DRTPN_STY={ty}", f"-DRTPN_STZ={tz}", f"-DRTPN_SNB={nb}", f"-DRTPN_SEM={eq}",
               os.path.join(HERE, "host", "emulate_stage.cu"), os.path.join(CSRC, "model.cpp"), "-o", exe]
        res = subprocess.run(cmd, capture_output=True, text=True)
        assert res.returncode == 0, res.stderr[-2000:]
        out[key] = exe
    return out


CASES = [
    # variant, shape (nz, ny, nx) with nx a multiple of 8, bc, target class, half step, storage, SMs
    (7, (5, 6, 72), "periodic", 0, 0, "fp32", 3),
    (7, (7, 5, 40), "vacuum", 1, 1, "fp32", 4),
    (7, (3, 3, 8), "periodic", 1, 0, "bf16", 2),
    (15, (7, 8, 64), "vacuum", 0, 0, "fp32", 5),
    (15, (4, 4, 40), "periodic", 1, 1, "bf16", 3),
    (39, (3, 5, 80), "periodic", 0, 0, "fp32", 4),
    (39, (4, 3, 48), "vacuum", 1, 0, "bf16", 2),
    (39, (2, 2, 8), "periodic", 1, 1, "fp32", 1),
]


@pytest.mark.parametrize("key,shape,bc,cls,half,prec,sms", CASES)
def test_stage_plan_and_columns_on_host_vs_oracle(emulators, tmp_path, key, shape, bc, cls, half, prec, sms):
    N = VARIANTS[key][0]
    inst, u = synth.random_instance(N, shape, seed=700 + N, bc=bc)
    nz, ny, nx = shape
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    np.concatenate([u.ravel(), inst.sigma_a.ravel(), inst.sigma_s.ravel(), inst.q.ravel()]).tofile(fin)
    res = subprocess.run([emulators[key], str(cls), str(nx), str(ny), str(nz), str(0 if bc == "periodic" else 1),
                          repr(inst.h), repr(inst.dt), str(half), prec, str(sms), fin, fout],
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    got = np.fromfile(fout).reshape(u.shape)
    P = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, bc)
    u_in = u.astype(np.float32).astype(np.float64) if prec == "fp32" else _bf16_round(u)
    ref = P.substep(u_in, cls, 0.5 * inst.dt if half else inst.dt)
    assert np.isfinite(got).all()
    if prec == "fp32":
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    else:  # one pass rounds its class once: within one BF16 ulp (2^-8 relative) of the oracle
        m = P.cls == cls
        assert np.all(np.abs(got[m] - ref[m]) <= 2.0 ** -8 * np.abs(ref[m]) + 1e-6 * np.abs(ref).max())
        assert np.array_equal(got[~m], u_in[~m])


ADJ_CASES = [
    # variant, shape (nz, ny, nx), bc, target class, alpha folded in, half step (the alpha's tau)
    (7, (5, 6, 72), "vacuum", 0, False, 0),
    (7, (4, 5, 40), "periodic", 1, True, 1),
    (15, (4, 5, 64), "periodic", 0, True, 0),
    (39, (3, 4, 40), "vacuum", 1, False, 0),
]


@pytest.mark.parametrize("key,shape,bc,cls,alpha,half", ADJ_CASES)
def test_adjoint_transposed_coupling_on_host_vs_oracle(emulators, tmp_path, key, shape, bc, cls, alpha, half):
    # the adjoint's pass onto class B = cls (mode ADJ_SOURCES): lam_B <- a lam_B + K w / h, which is
    # the oracle's pull-back lam_B - K^T (beta lam_A) through a substep on the other class A with
    # beta lam_A = w; a = 1, or the factor of a later substep on class B (folded in)
    N = VARIANTS[key][0]
    inst, u = synth.random_instance(N, shape, seed=900 + N, bc=bc)
    rng = np.random.default_rng(901 + N)
    lam, w = rng.standard_normal(u.shape), rng.standard_normal(u.shape)
    nz, ny, nx = shape
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    np.concatenate([lam.ravel(), w.ravel(), inst.sigma_a.ravel(), inst.sigma_s.ravel(), inst.q.ravel()]).tofile(fin)
    res = subprocess.run([emulators[key], str(cls), str(nx), str(ny), str(nz), str(0 if bc == "periodic" else 1),
                          repr(inst.h), repr(inst.dt), str(half), "fp32", "3", fin, fout,
                          "adjsrc_alpha" if alpha else "adjsrc"], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    got = np.fromfile(fout).reshape(u.shape)
    P = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, bc)
    a_cls, b = 1 - cls, P.cls == cls
    w32 = w.astype(np.float32).astype(np.float64)
    lam32 = lam.astype(np.float32).astype(np.float64)
    tau = inst.dt  # any tau: the oracle's pull-back is given lam_A = w / beta
    beta = tau * st.E(-P.c * tau)
    lam_in = lam32.copy()
    lam_in[P.cls == a_cls] = w32[P.cls == a_cls] / beta[P.cls == a_cls]
    grads = {"c": np.zeros_like(P.c), "q": np.zeros_like(P.q)}
    ref = P.substep_adjoint(u, lam_in, a_cls, tau, grads)  # ref_B = lam_B - K^T w
    if alpha:
        # the factor of class B at the alpha's tau (u_0, class 0, keeps its own at dt)
        tb = 0.5 * inst.dt if half else inst.dt
        fa = np.exp(-P.c * tb)
        fa[0] = np.exp(-P.c[0] * inst.dt)
        ref[b] = ref[b] - lam32[b] + fa[b] * lam32[b]
    assert np.abs(got[b] - ref[b]).max() <= 1e-5 * np.abs(ref[b]).max()
    assert np.array_equal(got[~b], lam32[~b])
