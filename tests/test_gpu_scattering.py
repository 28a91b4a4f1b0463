"""Anisotropic scattering (Section 2: Sigma_tl = Sigma_a + Sigma_s0 - Sigma_sl, Sigma_sl = f_l sigma_s)
on the generic kernel and on the window kernel's anisotropic form (N <= 15) against the oracle,
element by element, FP64 <= 1e-12, FP32 <= 1e-5 relative and BF16 by the rounding model (the bounds
of the isotropic tests); and the refusals of the other kernels."""
import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import rtpn, synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
from test_gpu_parity import assert_parity  # noqa: E402


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def hg(N, g):
    """Legendre moments of a Henyey-Greenstein phase function: f_l = g^l."""
    return np.array([g ** l for l in range(N + 1)])


def oracle(inst, coupling_cache, scat, h=None):
    mats, slots = coupling_cache(inst.N)
    return st.Problem(inst.N, inst.sigma_a, inst.sigma_s, inst.q, inst.h if h is None else h, inst.dt,
                      inst.bc, mats=mats, slots=slots, scat=None if scat is None else tuple(scat))


CASES = [
    # N, shape (nz, ny, nx), bc, precision, g, kernel asked for, kernel expected (1 generic, 2 window)
    (3, (5, 6, 7), "vacuum", "fp64", 0.6, "auto", 1),
    (7, (4, 5, 9), "periodic", "fp64", -0.3, "auto", 1),
    (7, (6, 7, 33), "vacuum", "fp32", 0.85, "generic", 1),
    (7, (6, 7, 33), "vacuum", "fp32", 0.85, "auto", 2),
    (3, (5, 6, 7), "periodic", "fp32", -0.4, "auto", 2),
    (15, (3, 4, 8), "periodic", "fp32", 0.5, "auto", 2),
    (15, (4, 3, 9), "vacuum", "fp32", 0.9, "window", 2),
    (9, (4, 5, 6), "vacuum", "bf16", 0.7, "auto", 2),
]


@pytest.mark.parametrize("N,shape,bc,precision,g,kernel,kid", CASES)
def test_anisotropic_scattering_vs_oracle(cuda_device, coupling_cache, N, shape, bc, precision, g, kernel, kid):
    inst, u0 = synth.random_instance(N, shape, seed=1200 + N, bc=bc)
    f = hg(N, g)
    P = oracle(inst, coupling_cache, f)
    ref = P.run(u0, 3)
    with rtpn.Context(N, shape, inst.h, bc, precision, inst.dt) as ctx:
        if kernel != "auto":
            ctx.set_kernel(kernel)
        ctx.set_scattering(f)
        assert ctx.info().kernel == kid
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        ctx.step(3)
        got = ctx.get_moments()
    if precision == "bf16":
        assert_parity(got, ref, precision, P, u0, 3)
    else:
        assert rel(got, ref) <= TOL[precision], rel(got, ref)


def test_scattering_set_after_media_and_back_to_isotropic(cuda_device, coupling_cache):
    # the moments set after the media recompute the factors; None restores the isotropic step and
    # the automatic kernel choice
    inst, u0 = synth.random_instance(7, (5, 6, 32), seed=1300, bc="vacuum")
    f = hg(7, 0.7)
    P_aniso, P_iso = oracle(inst, coupling_cache, f), oracle(inst, coupling_cache, None)
    with rtpn.Context(7, inst.shape, inst.h, inst.bc, "fp32", inst.dt) as ctx:
        assert ctx.info().kernel == 2
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        ctx.set_scattering(f)
        ctx.step(2)
        ref = P_aniso.run(u0, 2)
        assert rel(ctx.get_moments(), ref) <= TOL["fp32"]
        ctx.set_scattering(None)
        assert ctx.info().kernel == 2
        ctx.step(2)
        ref = P_iso.run(ref, 2)
        assert rel(ctx.get_moments(), ref) <= TOL["fp32"]


@pytest.mark.parametrize("precision,kid", [("fp64", 1), ("fp32", 2)])
def test_anisotropic_scattering_on_non_cubic_cells(cuda_device, coupling_cache, precision, kid):
    # FP32: the window kernel's form with both the scaled differences and the per-order factors
    h3 = (0.1, 0.13, 0.17)
    inst, u0 = synth.random_instance(5, (4, 5, 6), seed=1400, bc="periodic")
    f = hg(5, 0.4)
    ref = oracle(inst, coupling_cache, f, h=h3).run(u0, 3)
    with rtpn.Context(5, inst.shape, h3[0], inst.bc, precision, inst.dt) as ctx:
        ctx.set_spacing(*h3)
        ctx.set_scattering(f)
        assert ctx.info().kernel == kid
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        ctx.step(3)
        got = ctx.get_moments()
    assert rel(got, ref) <= TOL[precision], rel(got, ref)


def test_scattering_moves_a_staged_context_to_the_window_kernel(cuda_device, coupling_cache):
    # N = 15 with 16-byte rows runs on the staged kernel; anisotropic moments move it to the window
    # kernel (the staged kernel's tile is no window tile), and None moves it back
    inst, u0 = synth.random_instance(15, (4, 5, 32), seed=1500, bc="periodic")
    f = hg(15, 0.6)
    P_aniso, P_iso = oracle(inst, coupling_cache, f), oracle(inst, coupling_cache, None)
    with rtpn.Context(15, inst.shape, inst.h, inst.bc, "fp32", inst.dt) as ctx:
        assert ctx.info().kernel == 3
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        ctx.set_scattering(f)
        assert ctx.info().kernel == 2
        ctx.step(2)
        ref = P_aniso.run(u0, 2)
        assert rel(ctx.get_moments(), ref) <= TOL["fp32"]
        ctx.set_scattering(None)
        assert ctx.info().kernel == 3
        ctx.step(2)
        ref = P_iso.run(ref, 2)
        assert rel(ctx.get_moments(), ref) <= TOL["fp32"]


def test_anisotropic_scattering_refusals(cuda_device):
    with rtpn.Context(7, (3, 4, 32), 0.1, "periodic", "fp32", 0.03) as ctx:
        for bad in (np.ones(7), np.r_[0.9, np.zeros(7)], np.r_[1.0, 1.5, np.zeros(6)]):
            with pytest.raises(rtpn.RtpnError) as e:
                ctx.set_scattering(bad)
            assert e.value.code == rtpn.EINVAL
        ctx.set_kernel("stage")
        with pytest.raises(rtpn.RtpnError) as e:
            ctx.set_scattering(hg(7, 0.5))
        assert e.value.code == rtpn.EUNSUPPORTED
        ctx.set_kernel("auto")
        ctx.set_scattering(hg(7, 0.5))
        for k in ("stage", "fused"):
            with pytest.raises(rtpn.RtpnError) as e:
                ctx.set_kernel(k)
            assert e.value.code == rtpn.EUNSUPPORTED
        ctx.set_media(np.zeros((3, 4, 32)), np.ones((3, 4, 32)), np.zeros((3, 4, 32)))
        with pytest.raises(rtpn.RtpnError) as e:
            ctx.adjoint(np.ones((3, 4, 32)), 2, ckpt_every=1)
        assert e.value.code == rtpn.EUNSUPPORTED
    with rtpn.Context(39, (3, 4, 8), 0.1, "periodic", "fp32", 0.03) as ctx:
        ctx.set_kernel("window")   # no anisotropic form at N = 39
        with pytest.raises(rtpn.RtpnError) as e:
            ctx.set_scattering(hg(39, 0.5))
        assert e.value.code == rtpn.EUNSUPPORTED
        ctx.set_kernel("auto")
        ctx.set_scattering(hg(39, 0.5))
        assert ctx.info().kernel == 1
    insts = synth.batch_instances(2, seed=3)
    b = rtpn.Batch([(i.N, i.shape, i.h, i.bc, i.dt) for i in insts], "fp32")
    try:
        with pytest.raises(rtpn.RtpnError) as e:
            b.instances[0].set_scattering(hg(insts[0].N, 0.5))
        assert e.value.code == rtpn.EUNSUPPORTED
    finally:
        b.close()
