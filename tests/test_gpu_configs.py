"""The workloads at their full sizes, in the launch configuration bench.py times.

Where the oracle cannot run the whole workload, it computes one step from the same state at full
size (its cost is seconds), and long runs are compared with the GPU FP64 path, which the small
cases pin to the oracle at <= 1e-12.  Comparisons of large states are done component by component
on the device (torch is only the comparison plumbing here).
"""
import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import rtpn, synth

from test_gpu_parity import assert_parity, bf16_random_walk

pytestmark = pytest.mark.gpu


def make(inst, precision, kernel="auto"):
    ctx = rtpn.Context(inst.N, inst.shape, inst.h, inst.bc, precision, inst.dt)
    if kernel != "auto":
        ctx.set_kernel(kernel)
    ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
    return ctx


def device_rel_err(a, b, n_c, shape):
    """max |a - b| / max |b| over the full state, one component at a time on the device."""
    import torch

    ta = torch.empty(shape, dtype=torch.float64, device="cuda")
    tb = torch.empty(shape, dtype=torch.float64, device="cuda")
    num, den, num0, den0 = 0.0, 0.0, 0.0, 0.0
    for c in range(n_c):
        a.get_component(c, ta)
        b.get_component(c, tb)
        a.synchronize()
        b.synchronize()
        d = float((ta - tb).abs().max())
        r = float(tb.abs().max())
        num, den = max(num, d), max(den, r)
        if c == 0:
            num0, den0 = d, r
    return num / den, num0 / den0


def test_config1_one_step_vs_oracle_full_size(cuda_device):
    # P7, 128^3 checkerboard lattice, vacuum: one step from a dense random state, whole grid
    inst = synth.checkerboard(7, 128)
    u0 = synth.random_state(7, inst.shape, 5)
    ref = st.Problem(7, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, inst.bc).step(u0)
    for precision, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
        with make(inst, precision) as ctx:
            ctx.set_moments(u0)
            ctx.step(1)
            got = ctx.get_moments()
        assert np.abs(got - ref).max() / np.abs(ref).max() <= tol, precision


def test_config1_200_steps_fp32_vs_fp64(cuda_device):
    # P7 128^3 checkerboard, source in the central block, zero initial state, 200 steps
    inst = synth.checkerboard(7, 128)
    with make(inst, "fp64") as ref, make(inst, "fp32") as got:
        ref.step(200)
        got.step(200)
        err, err0 = device_rel_err(got, ref, 64, inst.shape)
        assert ref.count_nonfinite() == 0 and got.count_nonfinite() == 0
    assert err <= 1e-5 and err0 <= 1e-5, (err, err0)


def test_config2_small_instance_vs_oracle(cuda_device):
    # P39 on an independent 24^3 instance with the 200^3 rules, 100 steps: GPU FP64 vs the oracle
    inst = synth.random_blocks(39, 24, seed=2)
    u0 = inst.full_state()
    P = st.Problem(39, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, inst.bc)
    ref = P.run(u0, 100)
    for precision in ("fp64", "fp32", "bf16"):
        with make(inst, precision) as ctx:
            ctx.set_moments(u0)
            ctx.step(100)
            got = ctx.get_moments()
        assert_parity(got, ref, precision, P, u0, 100)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16", bf16_random_walk(100))])
def test_config2_full_size_vs_gpu_fp64(cuda_device, precision, tol):
    # P39 200^3 periodic, 100 steps: FP32 / BF16 storage vs the GPU FP64 path on the same input.
    # No oracle runs at this size, so BF16 is held to the random-walk size of its storage rounding
    # (an estimate, see bf16_random_walk); its rounding model is checked on the 24^3 instance.
    import torch

    inst = synth.random_blocks(39, 200, seed=2)
    u0 = torch.tensor(inst.u0, device="cuda")
    with make(inst, "fp64") as ref:
        ref.set_component(0, u0)
        ref.step(100)
        with make(inst, precision) as got:
            got.set_component(0, u0)
            got.step(100)
            err, err0 = device_rel_err(got, ref, 1600, inst.shape)
            s_ref, s_got = ref.sum_u0(), got.sum_u0()
    assert err <= tol and err0 <= tol, (err, err0)
    assert abs(s_got - s_ref) <= tol * abs(s_ref)


def test_config2_full_size_sampled_cells_vs_oracle(cuda_device):
    # P39 200^3 periodic in the bench's launch configuration (automatic kernel choice, FP32): one
    # step from the Gaussian u_0 plus eight seeded random components.  After one step a cell
    # depends on cells at most 4 away (three substeps, each reading one neighbour per axis, and the
    # point mean of the media), so the oracle steps an 11^3 crop around each sampled cell, with the
    # crop wrapped periodically, and its centre value is exact.
    import torch

    inst = synth.random_blocks(39, 200, seed=2)
    n_c = inst.n_c
    rng = np.random.default_rng(41)
    extra = {c: 0.1 * rng.standard_normal(inst.shape) for c in (1, 5, 17, 100, 400, 801, 1200, 1599)}
    samples = [(0, 0, 0), (199, 199, 199), (100, 57, 3), (31, 150, 199), (7, 0, 120)]  # (z, y, x)
    flat = torch.tensor([(z * 200 + y) * 200 + x for z, y, x in samples], device="cuda")
    got = np.zeros((len(samples), n_c))
    with make(inst, "fp32") as ctx:
        assert ctx.info().kernel == 3  # the staged kernel, as the bench runs it
        ctx.zero_moments()
        ctx.set_component(0, torch.tensor(inst.u0, device="cuda"))
        for c, v in extra.items():
            ctx.set_component(c, torch.tensor(v, device="cuda"))
        ctx.step(1)
        buf = torch.empty(inst.shape, dtype=torch.float64, device="cuda")
        for c in range(n_c):
            ctx.get_component(c, buf)
            ctx.synchronize()
            got[:, c] = buf.reshape(-1)[flat].cpu().numpy()
    r = 5
    worst = 0.0
    for k, (z, y, x) in enumerate(samples):
        iz, iy, ix = (np.arange(p - r, p + r + 1) % 200 for p in (z, y, x))
        crop = np.ix_(iz, iy, ix)
        u = np.zeros((n_c, 2 * r + 1, 2 * r + 1, 2 * r + 1))
        u[0] = inst.u0[crop]
        for c, v in extra.items():
            u[c] = v[crop]
        ref = st.Problem(39, inst.sigma_a[crop], inst.sigma_s[crop], inst.q[crop], inst.h, inst.dt,
                         "periodic").step(u)[:, r, r, r]
        worst = max(worst, np.abs(got[k] - ref).max() / np.abs(ref).max())
    assert worst <= 1e-5, worst
