"""The autograd form of the adjoint: torch.autograd.grad of the detector functional J against the
oracle's discrete adjoint, torch.autograd.gradcheck, and FP32 against the oracle.

J = sum w u_0 after k steps is differentiated with respect to per-cell sigma_a, sigma_s and q; the
gradients come from the library's rtpn_adjoint behind paper_2004_02833_gb300.autograd.
Bounds: as the plain adjoint tests (tests/test_gpu_adjoint.py), the same arithmetic.
"""
import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import rtpn, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def tensors(arrays, dtype, requires_grad=False):
    import torch

    return [torch.tensor(a, dtype=dtype, device="cuda", requires_grad=requires_grad) for a in arrays]


def test_autograd_p3_32_checkerboard_fp64_vs_oracle(cuda_device, coupling_cache):
    import torch

    from paper_2004_02833_gb300.autograd import detector_response

    inst = synth.checkerboard(3, 32)
    w = synth.detector_box(32)
    mats, slots = coupling_cache(3)
    P = st.Problem(3, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, inst.bc, mats=mats, slots=slots)
    k = 30
    J_ref, gsa_ref, gss_ref, gq_ref = P.gradient(inst.full_state(), k, w)
    sa, ss, q = tensors((inst.sigma_a, inst.sigma_s, inst.q), torch.float64, requires_grad=True)
    u0, wt = tensors((inst.full_state(), w), torch.float64)
    with rtpn.Context(3, inst.shape, inst.h, inst.bc, "fp64", inst.dt) as ctx:
        J = detector_response(ctx, sa, ss, q, u0, wt, k, ckpt_every=7)
        gsa, gss, gq = torch.autograd.grad(J, (sa, ss, q))
        assert J.dim() == 0 and J.is_cuda
        Jv = float(J.detach())
    assert J_ref > 0 and abs(Jv - J_ref) <= 1e-12 * J_ref
    for g, ref in ((gsa, gsa_ref), (gss, gss_ref), (gq, gq_ref)):
        assert rel(g.cpu().numpy(), ref) <= 1e-12


def test_autograd_scales_by_the_incoming_gradient(cuda_device):
    import torch

    from paper_2004_02833_gb300.autograd import detector_response

    inst, u = synth.random_instance(3, (4, 5, 8), seed=61, bc="periodic")
    w = np.random.default_rng(62).uniform(0.0, 1.0, inst.shape)
    sa, ss, q = tensors((inst.sigma_a, inst.sigma_s, inst.q), torch.float64, requires_grad=True)
    u0, wt = tensors((u, w), torch.float64)
    with rtpn.Context(3, inst.shape, inst.h, inst.bc, "fp64", inst.dt) as ctx:
        J = detector_response(ctx, sa, ss, q, u0, wt, 4, ckpt_every=3)
        (2.5 * J).backward()
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u)
        J_plain, (gsa, gss, gq) = ctx.adjoint(w, 4, ckpt_every=3)
    assert abs(float(J.detach()) - J_plain) <= 1e-13 * abs(J_plain)
    for t, g in ((sa, gsa), (ss, gss), (q, gq)):
        assert np.array_equal(t.grad.cpu().numpy(), 2.5 * g)


def test_autograd_gradcheck_fp64(cuda_device):
    import torch

    from paper_2004_02833_gb300.autograd import detector_response

    inst, u = synth.random_instance(1, (3, 4, 4), seed=63, bc="vacuum")
    w = np.random.default_rng(64).uniform(0.0, 1.0, inst.shape)
    sa, ss, q = tensors((inst.sigma_a + 0.5, inst.sigma_s + 0.5, inst.q), torch.float64, requires_grad=True)
    u0, wt = tensors((u, w), torch.float64)
    with rtpn.Context(1, inst.shape, inst.h, inst.bc, "fp64", inst.dt) as ctx:
        fn = lambda a, s, qq: detector_response(ctx, a, s, qq, u0, wt, 3, ckpt_every=2)
        assert torch.autograd.gradcheck(fn, (sa, ss, q), eps=1e-6, atol=1e-8, rtol=1e-6, fast_mode=True)


def test_autograd_fp32_staged_vs_oracle(cuda_device, coupling_cache):
    import torch

    from paper_2004_02833_gb300.autograd import detector_response

    N, shape = 15, (4, 5, 40)
    inst, u = synth.random_instance(N, shape, seed=65, bc="vacuum")
    w = np.random.default_rng(66).uniform(0.0, 1.0, shape)
    mats, slots = coupling_cache(N)
    P = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, inst.bc, mats=mats, slots=slots)
    J_ref, gsa_ref, gss_ref, gq_ref = P.gradient(u, 3, w)
    sa, ss, q = tensors((inst.sigma_a, inst.sigma_s, inst.q), torch.float32, requires_grad=True)
    u0, wt = tensors((u, w), torch.float32)
    with rtpn.Context(N, shape, inst.h, inst.bc, "fp32", inst.dt) as ctx:
        ctx.set_kernel("stage")
        J = detector_response(ctx, sa, ss, q, u0, wt, 3, ckpt_every=2)
        gsa, gss, gq = torch.autograd.grad(J, (sa, ss, q))
    assert gsa.dtype == torch.float32
    assert abs(float(J.detach()) - J_ref) <= 1e-4 * abs(J_ref)
    for g, ref in ((gsa, gsa_ref), (gss, gss_ref), (gq, gq_ref)):
        assert rel(g.cpu().double().numpy(), ref) <= 1e-4
