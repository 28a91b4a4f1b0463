"""Non-cubic cells (hx, hy, hz): the GPU path against the oracle, whose differences divide by the
cell size of their own axis (Section 2.1), for the kernels that take them (staged, generic, the
window kernel up to N = 15) and the adjoint; the fused and batched kernels and the P39 window
kernel refuse them.  Same bounds as the cubic tests."""
import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import rtpn, synth

pytestmark = pytest.mark.gpu

H3 = (0.1, 0.13, 0.17)   # dt = 0.03 < min(h) / 3
from test_gpu_parity import TOL, assert_parity  # noqa: E402


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def problem(inst, coupling_cache, h=H3):
    mats, slots = coupling_cache(inst.N)
    return st.Problem(inst.N, inst.sigma_a, inst.sigma_s, inst.q, h, inst.dt, inst.bc, mats=mats,
                      slots=slots)


CASES = [
    # N, shape (nz, ny, nx), bc, kernel, precision, expected kernel id
    (3, (5, 6, 7), "vacuum", "generic", "fp64", 1),
    (7, (6, 7, 9), "periodic", "generic", "fp32", 1),
    (7, (5, 6, 32), "vacuum", "stage", "fp32", 3),      # the staged kernel (compiled for N = 7)
    (7, (5, 6, 32), "vacuum", "auto", "fp32", 2),       # below N = 15 the window kernel
    (5, (4, 5, 6), "periodic", "auto", "fp32", 2),
    (3, (6, 7, 9), "vacuum", "window", "bf16", 2),
    (9, (5, 4, 7), "periodic", "window", "fp32", 2),
    (15, (4, 5, 9), "vacuum", "window", "fp32", 2),
    (15, (3, 4, 6), "periodic", "window", "bf16", 2),
    (15, (7, 9, 40), "periodic", "stage", "fp32", 3),
    (15, (3, 5, 8), "vacuum", "stage", "bf16", 3),
    (39, (4, 5, 40), "vacuum", "auto", "fp32", 3),
]


@pytest.mark.parametrize("N,shape,bc,kernel,precision,kid", CASES)
def test_non_cubic_cells_vs_oracle(cuda_device, coupling_cache, N, shape, bc, kernel, precision, kid):
    inst, u0 = synth.random_instance(N, shape, seed=1000 + N, bc=bc)
    P = problem(inst, coupling_cache)
    ref = P.run(u0, 3)
    with rtpn.Context(N, shape, H3[0], bc, precision, inst.dt) as ctx:
        if kernel != "auto":
            ctx.set_kernel(kernel)
        ctx.set_spacing(*H3)
        info = ctx.info()
        assert info.kernel == kid and (info.h, info.hy, info.hz) == H3
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        ctx.step(3)
        got = ctx.get_moments()
    assert_parity(got, ref, precision, P, u0, 3)


def test_spacing_back_to_cubic_is_bitwise_unchanged(cuda_device):
    inst, u0 = synth.random_instance(7, (5, 6, 33), seed=11, bc="periodic")
    out = []
    for spacings in ([], [H3, (inst.h,) * 3]):
        with rtpn.Context(7, inst.shape, inst.h, inst.bc, "fp32", inst.dt) as ctx:
            for s in spacings:
                ctx.set_spacing(*s)
            assert ctx.info().kernel == 2
            ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
            ctx.set_moments(u0)
            ctx.step(4)
            out.append(ctx.get_moments())
    assert np.array_equal(out[0], out[1])


# FP64: the bound the task sets for FP64 parity, 1e-12, on J and on every gradient (both sides
# evaluate E' of Eq. 5 without cancellation).  FP32: the cubic bound.
@pytest.mark.parametrize("precision,kernel,tol", [("fp64", "generic", 1e-12), ("fp32", "stage", 1e-4)])
def test_adjoint_non_cubic_vs_oracle(cuda_device, coupling_cache, precision, kernel, tol):
    N, shape = (3, (5, 6, 8)) if kernel == "generic" else (15, (4, 5, 40))
    inst, u0 = synth.random_instance(N, shape, seed=1100 + N, bc="vacuum")
    w = np.random.default_rng(7).uniform(0.0, 1.0, shape)
    J_ref, gsa_ref, gss_ref, gq_ref = problem(inst, coupling_cache).gradient(u0, 3, w)
    with rtpn.Context(N, shape, H3[0], "vacuum", precision, inst.dt) as ctx:
        ctx.set_kernel(kernel)
        ctx.set_spacing(*H3)
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        J, (gsa, gss, gq) = ctx.adjoint(w, 3, ckpt_every=2)
    assert abs(J - J_ref) <= tol * abs(J_ref)
    assert rel(gsa, gsa_ref) <= tol and rel(gss, gss_ref) <= tol and rel(gq, gq_ref) <= tol


def test_non_cubic_rejections(cuda_device):
    with rtpn.Context(39, (3, 4, 8), 0.1, "periodic", "fp32", 0.03) as ctx:
        ctx.set_kernel("window")
        with pytest.raises(rtpn.RtpnError) as e:
            ctx.set_spacing(*H3)
        assert e.value.code == rtpn.EUNSUPPORTED and ctx.info().hy == 0.1
        ctx.set_kernel("auto")
        ctx.set_spacing(*H3)
        with pytest.raises(rtpn.RtpnError) as e:
            ctx.set_kernel("window")
        assert e.value.code == rtpn.EUNSUPPORTED
    with rtpn.Context(7, (3, 4, 32), 0.1, "periodic", "fp32", 0.03) as ctx:
        ctx.set_kernel("fused")
        with pytest.raises(rtpn.RtpnError) as e:
            ctx.set_spacing(*H3)
        assert e.value.code == rtpn.EUNSUPPORTED
        ctx.set_kernel("auto")
        with pytest.raises(rtpn.RtpnError) as e:
            ctx.set_spacing(0.1, 0.05, 0.1)   # dt = 0.03 >= 0.05 / 3
        assert e.value.code == rtpn.ECFL and ctx.info().hy == 0.1
        ctx.set_spacing(*H3)
        with pytest.raises(rtpn.RtpnError) as e:
            ctx.set_kernel("fused")
        assert e.value.code == rtpn.EUNSUPPORTED
        ctx.set_kernel("window")
        assert ctx.info().kernel == 2
    insts = synth.batch_instances(2, seed=3)
    b = rtpn.Batch([(i.N, i.shape, i.h, i.bc, i.dt) for i in insts], "fp32")
    try:
        with pytest.raises(rtpn.RtpnError) as e:
            b.instances[0].set_spacing(insts[0].h, 2 * insts[0].h, insts[0].h)
        assert e.value.code == rtpn.EUNSUPPORTED
    finally:
        b.close()
