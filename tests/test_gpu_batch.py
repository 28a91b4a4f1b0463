"""Batched form: one grouped launch per pass over independent instances of uneven order and size,
against the oracle per instance and against the per-instance launch loop."""
import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import rtpn, synth
from test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu


def small_instances(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i, N in enumerate([15, 1, 9, 3, 7, 5, 3, 1]):
        shape = tuple(int(v) for v in rng.integers(3, 21, 3))
        bc = "periodic" if i % 2 == 0 else "vacuum"
        inst, u = synth.random_instance(N, shape, seed=200 + i, bc=bc)
        out.append((inst, u))
    return out


def make_batch(items, precision="fp32"):
    b = rtpn.Batch([(i.N, i.shape, i.h, i.bc, i.dt) for i, _ in items], precision)
    for ctx, (inst, u) in zip(b.instances, items):
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u)
    return b


@pytest.mark.parametrize("tile", [(32, 4, 2), (16, 4, 4), (8, 8, 4), (32, 1, 1)])
def test_batch_matches_oracle(cuda_device, tile):
    items = small_instances()
    with make_batch(items) as b:
        b.set_tile(tile)
        assert b.tile() == tile
        b.step(3)
        got = [ctx.get_moments() for ctx in b.instances]
    for (inst, u), g in zip(items, got):
        ref = st.Problem(inst.N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, inst.bc).run(u, 3)
        assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max(), inst.N


def test_batch_grouped_equals_looped(cuda_device):
    items = small_instances(1)
    with make_batch(items) as b1, make_batch(items) as b2:
        b1.step(5)
        b2.step_looped(5)
        for c1, c2 in zip(b1.instances, b2.instances):
            a, r = c1.get_moments(), c2.get_moments()
            assert np.abs(a - r).max() <= 1e-6 * np.abs(r).max()


def test_batch_bf16(cuda_device):
    items = small_instances(2)
    with make_batch(items, "bf16") as b:
        b.step(2)
        got = [ctx.get_moments() for ctx in b.instances]
    for (inst, u), g in zip(items, got):
        P = st.Problem(inst.N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, inst.bc)
        assert_parity(g, P.run(u, 2), "bf16", P, u, 2)  # against the oracle's BF16 rounding model


def test_batch_rejects_unsupported(cuda_device):
    with pytest.raises(rtpn.RtpnError) as e:
        rtpn.Batch([(39, (4, 4, 4), 0.1, "periodic", None)])
    assert e.value.code == rtpn.EUNSUPPORTED
    with pytest.raises(rtpn.RtpnError) as e:
        rtpn.Batch([(3, (4, 4, 4), 0.1, "periodic", None)], "fp64")
    assert e.value.code == rtpn.EUNSUPPORTED
    with rtpn.Batch([(3, (4, 4, 4), 0.1, "periodic", None)]) as b:
        with pytest.raises(rtpn.RtpnError) as e:
            b.step(1)
        assert e.value.code == rtpn.ESTATE
        with pytest.raises(rtpn.RtpnError):
            b.set_tile((33, 1, 1))


def test_batched_workload_64_instances(cuda_device):
    # 64 instances, N in {1,3,5,9,15}, sides 24..96, Gaussian or checkerboard media, 100 FP32 steps:
    # grouped launch vs per-instance loop, and three instances against the GPU FP64 path.
    insts = synth.batch_instances(64, seed=3)
    items = [(i, i.full_state()) for i in insts]
    with make_batch(items) as b1, make_batch(items) as b2:
        b1.step(100)
        b2.step_looped(100)
        b1.synchronize()
        for k, (c1, c2) in enumerate(zip(b1.instances, b2.instances)):
            a, r = c1.get_component(0), c2.get_component(0)
            assert np.abs(a - r).max() <= 1e-6 * max(np.abs(r).max(), 1e-30), k
        for k in (0, 17, 63):
            inst = insts[k]
            with rtpn.Context(inst.N, inst.shape, inst.h, inst.bc, "fp64", inst.dt) as ref:
                ref.set_media(inst.sigma_a, inst.sigma_s, inst.q)
                ref.set_moments(inst.full_state())
                ref.step(100)
                want = ref.get_moments()
            got = b1.instances[k].get_moments()
            assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max(), k


def test_batch_autotune_keeps_state(cuda_device):
    items = small_instances(4)
    with make_batch(items) as b:
        before = [c.get_moments() for c in b.instances]
        tile, ms = b.autotune(reps=1)
        assert b.tile() == tile and ms > 0
        after = [c.get_moments() for c in b.instances]
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
