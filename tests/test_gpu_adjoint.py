"""Adjoint form: GPU discrete adjoint vs the oracle's discrete adjoint and vs central finite
differences of the GPU forward.

Bounds: FP64 storage: J, the final state and each gradient <= 1e-12 relative (max norm) to the
oracle, the bound the task sets for FP64 parity (both sides evaluate E' of Eq. 5, which enters
dbeta/dc, without the cancellation of its closed form near 0); FP32 storage <= 1e-4 relative to the
oracle's exact adjoint; FP32 adjoint vs FP64 central differences <= 1e-3.
"""
import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import rtpn, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("bc", ["periodic", "vacuum"])
@pytest.mark.parametrize("precision,tol,gtol", [("fp64", 1e-12, 1e-12), ("fp32", 1e-4, 1e-4)])
def test_adjoint_matches_oracle(cuda_device, coupling_cache, bc, precision, tol, gtol):
    N, shape = 3, (5, 6, 8)
    inst, u0 = synth.random_instance(N, shape, seed=41, bc=bc)
    w = np.random.default_rng(42).uniform(0.0, 1.0, shape)
    mats, slots = coupling_cache(N)
    P = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, bc, mats=mats, slots=slots)
    J_ref, gsa_ref, gss_ref, gq_ref = P.gradient(u0, 5, w)
    with rtpn.Context(N, shape, inst.h, bc, precision, inst.dt) as ctx:
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        J, (gsa, gss, gq) = ctx.adjoint(w, 5, ckpt_every=2)
        final = ctx.get_moments()
    assert abs(J - J_ref) <= tol * abs(J_ref)
    assert rel(gsa, gsa_ref) <= gtol and rel(gss, gss_ref) <= gtol and rel(gq, gq_ref) <= gtol
    assert rel(final, P.run(u0, 5)) <= max(tol, 1e-12)


@pytest.mark.parametrize("bc", ["periodic", "vacuum"])
def test_adjoint_staged_kernel_fp32_vs_oracle(cuda_device, coupling_cache, bc):
    # FP32 with the staged kernel: the forward recomputation and the transposed coupling of every
    # backward substep (lam_B += K w / h) run on it; full and partial tiles (nx = 40 > 32)
    N, shape = 15, (4, 5, 40)
    inst, u0 = synth.random_instance(N, shape, seed=43, bc=bc)
    w = np.random.default_rng(44).uniform(0.0, 1.0, shape)
    mats, slots = coupling_cache(N)
    P = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, bc, mats=mats, slots=slots)
    J_ref, gsa_ref, gss_ref, gq_ref = P.gradient(u0, 3, w)
    with rtpn.Context(N, shape, inst.h, bc, "fp32", inst.dt) as ctx:
        ctx.set_kernel("stage")
        assert ctx.info().kernel == 3
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        J, (gsa, gss, gq) = ctx.adjoint(w, 3, ckpt_every=2)
    assert abs(J - J_ref) <= 1e-4 * abs(J_ref)
    assert rel(gsa, gsa_ref) <= 1e-4 and rel(gss, gss_ref) <= 1e-4 and rel(gq, gq_ref) <= 1e-4


@pytest.mark.parametrize("bc", ["periodic", "vacuum"])
def test_adjoint_staged_kernel_many_tiles_vs_oracle(cuda_device, coupling_cache, bc):
    # more tiles than CTAs (one per SM), partial tiles in x and z: the per-tile media-gradient sums
    # of the staged pull-back must start from zero on every tile a CTA walks
    N, shape = 7, (9, 40, 72)
    inst, u0 = synth.random_instance(N, shape, seed=45, bc=bc)
    w = np.random.default_rng(46).uniform(0.0, 1.0, shape)
    mats, slots = coupling_cache(N)
    P = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, bc, mats=mats, slots=slots)
    J_ref, gsa_ref, gss_ref, gq_ref = P.gradient(u0, 2, w)
    with rtpn.Context(N, shape, inst.h, bc, "fp32", inst.dt) as ctx:
        ctx.set_kernel("stage", (32, 2, 2))
        assert ctx.info().kernel == 3
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        J, (gsa, gss, gq) = ctx.adjoint(w, 2, ckpt_every=1)
    assert abs(J - J_ref) <= 1e-4 * abs(J_ref)
    assert rel(gsa, gsa_ref) <= 1e-4 and rel(gss, gss_ref) <= 1e-4 and rel(gq, gq_ref) <= 1e-4


@pytest.mark.parametrize("k,ckpt", [(7, 3), (4, 4), (2, 5), (5, 1)])
def test_adjoint_staged_segments_vs_oracle(cuda_device, coupling_cache, k, ckpt):
    # the staged FP32 adjoint runs each checkpoint segment in the merged form of the step, written
    # out of place: segments of uneven length (7 = 3 + 3 + 1), one segment, a segment shorter than
    # the checkpoint interval and one step per segment, against the literal schedule of the oracle;
    # the final state (end of the last segment copied back) too
    N, shape = 7, (6, 5, 32)
    inst, u0 = synth.random_instance(N, shape, seed=47, bc="vacuum")
    w = np.random.default_rng(48).uniform(0.0, 1.0, shape)
    mats, slots = coupling_cache(N)
    P = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, "vacuum", mats=mats, slots=slots)
    J_ref, gsa_ref, gss_ref, gq_ref = P.gradient(u0, k, w)
    with rtpn.Context(N, shape, inst.h, "vacuum", "fp32", inst.dt) as ctx:
        ctx.set_kernel("stage")
        assert ctx.info().kernel == 3
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        before = ctx.info().steps_done
        J, (gsa, gss, gq) = ctx.adjoint(w, k, ckpt_every=ckpt)
        final = ctx.get_moments()
        assert ctx.info().steps_done == before + k
    assert np.abs(inst.q).max() > 0
    assert abs(J - J_ref) <= 1e-4 * abs(J_ref)
    assert rel(gsa, gsa_ref) <= 1e-4 and rel(gss, gss_ref) <= 1e-4 and rel(gq, gq_ref) <= 1e-4
    assert rel(final, P.run(u0, k)) <= 1e-5


def test_adjoint_workspace_kept_between_calls(cuda_device):
    # the staged adjoint keeps its work buffers and tensor maps: a second call with the same layout,
    # one with a smaller layout, one after rtpn_adjoint_release and one with a larger layout all give
    # the first call's result bit for bit (same inputs, same launches)
    N, shape = 7, (6, 5, 32)
    inst, u0 = synth.random_instance(N, shape, seed=51, bc="vacuum")
    w = np.random.default_rng(52).uniform(0.0, 1.0, shape)
    with rtpn.Context(N, shape, inst.h, "vacuum", "fp32", inst.dt) as ctx:
        ctx.set_kernel("stage")
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)

        def run(k, ckpt):
            ctx.set_moments(u0)
            J, g = ctx.adjoint(w, k, ckpt_every=ckpt)
            return J, np.stack(g)

        first = run(6, 3)
        for k, ckpt, release in ((6, 3, False), (2, 2, False), (6, 3, True), (6, 3, False), (9, 3, False)):
            if release:
                ctx.adjoint_release()
            got = run(k, ckpt)
            if (k, ckpt) == (6, 3):
                assert got[0] == first[0] and np.array_equal(got[1], first[1])
        ctx.adjoint_release()
        ctx.adjoint_release()  # a context without kept buffers


@pytest.mark.parametrize("kernel", ["stage", "generic"])
def test_adjoint_zero_steps(cuda_device, kernel):
    # k = 0: J is the detector on the current state, every gradient is zero, the state is unchanged
    N, shape = 7, (4, 4, 32)
    inst, u0 = synth.random_instance(N, shape, seed=49, bc="periodic")
    w = np.random.default_rng(50).uniform(0.0, 1.0, shape)
    with rtpn.Context(N, shape, inst.h, "periodic", "fp32", inst.dt) as ctx:
        ctx.set_kernel(kernel)
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        ctx.set_moments(u0)
        before = ctx.get_moments()
        J, grads = ctx.adjoint(w, 0, ckpt_every=3)
        after = ctx.get_moments()
    J_ref = float((w * before[0].astype(np.float64)).sum())
    assert abs(J - J_ref) <= 1e-12 * abs(J_ref)
    assert all(not np.any(g) for g in grads)
    assert np.array_equal(before, after)


def test_adjoint_p3_32_checkerboard_fp64(cuda_device, coupling_cache):
    # P3 on 32^3 in FP64: the lattice scaled to 32^3, vacuum, zero start, detector box scaled
    inst = synth.checkerboard(3, 32)
    w = synth.detector_box(32)
    mats, slots = coupling_cache(3)
    P = st.Problem(3, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, inst.bc, mats=mats, slots=slots)
    k = 30
    J_ref, gsa_ref, gss_ref, gq_ref = P.gradient(inst.full_state(), k, w)
    with rtpn.Context(3, inst.shape, inst.h, inst.bc, "fp64", inst.dt) as ctx:
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        J, (gsa, gss, gq) = ctx.adjoint(w, k, ckpt_every=7)
    assert J_ref > 0 and abs(J - J_ref) <= 1e-12 * J_ref
    assert rel(gsa, gsa_ref) <= 1e-12 and rel(gss, gss_ref) <= 1e-12 and rel(gq, gq_ref) <= 1e-12


def test_adjoint_fp32_vs_central_differences(cuda_device):
    # P15 on the [0,7]^3 lattice at 48^3 (long enough for the source to reach the detector):
    # the FP32 adjoint against central differences of the FP64 GPU forward at seeded cells.
    N, n, k = 15, 48, 100
    inst = synth.checkerboard(N, n)
    w = synth.detector_box(n)
    with rtpn.Context(N, inst.shape, inst.h, inst.bc, "fp32", inst.dt) as ctx:
        ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        J32, (gsa, gss, gq) = ctx.adjoint(w, k, ckpt_every=20)

    def J64(sa, ss, q):
        with rtpn.Context(N, inst.shape, inst.h, inst.bc, "fp64", inst.dt) as c:
            c.set_media(sa, ss, q)
            c.step(k)
            return float(np.sum(w * c.get_component(0)))

    base = J64(inst.sigma_a, inst.sigma_s, inst.q)
    assert base > 0 and abs(J32 - base) <= 1e-4 * base
    rng = np.random.default_rng(4)
    # cells between the source block (3,3,3) and the detector block (5,3,3)
    cells = [(int(z), int(y), int(x)) for z, y, x in
             zip(rng.integers(22, 26, 3), rng.integers(22, 26, 3), rng.integers(26, 34, 3))]
    for cell in cells:
        for name, g in (("sa", gsa), ("ss", gss), ("q", gq)):
            args = {"sa": inst.sigma_a, "ss": inst.sigma_s, "q": inst.q}
            eps = 1e-6 * max(float(args[name][cell]), 1.0)
            p = {kk: v.copy() for kk, v in args.items()}
            m = {kk: v.copy() for kk, v in args.items()}
            p[name][cell] += eps
            m[name][cell] -= eps
            fd = (J64(p["sa"], p["ss"], p["q"]) - J64(m["sa"], m["ss"], m["q"])) / (2 * eps)
            scale = max(abs(fd), 1e-3 * np.abs(g).max())
            assert abs(g[cell] - fd) <= 1e-3 * scale, (name, cell, g[cell], fd)


def test_adjoint_p15_96_config_vs_central_differences(cuda_device):
    # The adjoint workload at its stated size: P15 on the [0,7]^3 lattice at 96^3 cells, vacuum, 200
    # steps with checkpoints every 20, J = sum of u_0 over the 12^3 detector box.
    #  * the method: the FP64 adjoint (the oracle's discrete adjoint to 1e-12, tests above) against
    #    central differences of the FP64 forward (perturbation 1e-6 max(sigma, 1)) at 20 cells drawn
    #    by default_rng(4) from the region between the source block (3,3,3) and the detector block
    #    (5,3,3), all three media fields at each: <= 1e-5 relative.  A central difference with step
    #    1e-6 resolves a derivative only down to about (rounding of J) / step, ~1e-10 here, so for an
    #    entry below 1e-3 of its field's largest the check is normwise: <= 1e-5 of that largest;
    #  * the precision: the FP32 adjoint against the FP64 one over the whole grid, normwise, J to
    #    1e-4 and each gradient field to 1e-3 of its max.
    N, n, k = 15, 96, 200
    inst = synth.checkerboard(N, n)
    w = synth.detector_box(n)
    grads = {}
    for prec in ("fp32", "fp64"):
        with rtpn.Context(N, inst.shape, inst.h, inst.bc, prec, inst.dt) as ctx:
            ctx.set_media(inst.sigma_a, inst.sigma_s, inst.q)
            grads[prec] = ctx.adjoint(w, k, ckpt_every=20)
    J32, g32 = grads["fp32"]
    J64, g64 = grads["fp64"]
    assert J64 > 0 and abs(J32 - J64) <= 1e-4 * J64
    for a32, a64 in zip(g32, g64):
        assert rel(a32, a64) <= 1e-3
    rng = np.random.default_rng(4)
    cells = list(zip(rng.integers(41, 55, 20), rng.integers(41, 55, 20), rng.integers(41, 82, 20)))
    with rtpn.Context(N, inst.shape, inst.h, inst.bc, "fp64", inst.dt) as c64:

        def J(sa, ss, q):
            c64.set_media(sa, ss, q)
            c64.zero_moments()
            c64.step(k)
            return c64.detector(w)

        assert abs(J(inst.sigma_a, inst.sigma_s, inst.q) - J64) <= 1e-12 * J64
        for cell in [(int(z), int(y), int(x)) for z, y, x in cells]:
            for name, g in zip(("sa", "ss", "q"), g64):
                args = {"sa": inst.sigma_a, "ss": inst.sigma_s, "q": inst.q}
                eps = 1e-6 * max(float(args[name][cell]), 1.0)
                p = {kk: v.copy() for kk, v in args.items()}
                m = {kk: v.copy() for kk, v in args.items()}
                p[name][cell] += eps
                m[name][cell] -= eps
                fd = (J(p["sa"], p["ss"], p["q"]) - J(m["sa"], m["ss"], m["q"])) / (2 * eps)
                gmax = np.abs(g).max()
                scale = abs(fd) if abs(fd) >= 1e-3 * gmax else gmax
                assert abs(g[cell] - fd) <= 1e-5 * scale, (name, cell, g[cell], fd)
