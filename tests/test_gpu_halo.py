"""The z-slab decomposition on device state: 2 to 4 slab contexts on one GPU, ghost planes
refreshed device to device after every pass (rtpn_copy_planes), against one context over the whole
grid (Section 3's one-layer halos; Eq. 6's merged schedule on both sides).  FP64 on the generic
kernel to 1e-12 relative (the slabs compute every own cell from the same values as the single
context), FP32 on the window and the staged kernels to the FP32 bound."""
import numpy as np
import pytest

from paper_2004_02833_gb300 import halo, rtpn, synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = [
    # N, shape (nz, ny, nx), bc, slabs, precision, kernel, steps
    (3, (12, 7, 9), "periodic", 2, "fp64", "auto", 5),
    (3, (13, 6, 8), "vacuum", 3, "fp64", "auto", 4),
    (7, (16, 9, 10), "periodic", 4, "fp64", "auto", 3),
    (7, (11, 9, 10), "vacuum", 2, "fp32", "window", 4),
    (15, (10, 6, 40), "periodic", 3, "fp32", "stage", 3),
    (39, (8, 4, 40), "vacuum", 2, "fp32", "stage", 2),
]


@pytest.mark.parametrize("N,shape,bc,nslab,precision,kernel,steps", CASES)
def test_device_slabs_equal_one_context(cuda_device, N, shape, bc, nslab, precision, kernel, steps):
    inst, u0 = synth.random_instance(N, shape, seed=1200 + N, bc=bc)
    with rtpn.Context(N, shape, inst.h, bc, precision, inst.dt) as one:
        if kernel != "auto":
            one.set_kernel(kernel)
        one.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        one.set_moments(u0)
        one.step(steps)
        ref = one.get_moments()
    with halo.DeviceSlabs(N, shape, inst.h, bc, precision, inst.dt, nslab, kernel) as sl:
        sl.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        sl.set_moments(u0)
        sl.step(steps)
        got = sl.get_moments()
    assert rel(got, ref) <= (1e-12 if precision == "fp64" else 1e-6), rel(got, ref)


def test_copy_planes_rejects_mismatches(cuda_device):
    with rtpn.Context(3, (4, 5, 6), 0.1, "periodic", "fp64", 0.03) as a, \
            rtpn.Context(3, (4, 5, 7), 0.1, "periodic", "fp64", 0.03) as b, \
            rtpn.Context(3, (6, 5, 6), 0.1, "periodic", "fp64", 0.03) as c:
        with pytest.raises(rtpn.RtpnError):
            a.copy_planes_from(b, 0, 0, 1)      # nx differs
        with pytest.raises(rtpn.RtpnError):
            a.copy_planes_from(c, 5, 0, 2)      # past the source grid
        with pytest.raises(rtpn.RtpnError):
            a.copy_planes_from(a, 0, 1, 2)      # overlapping planes of one context
        u = synth.random_state(3, (6, 5, 6), 3)
        c.set_moments(u)
        a.zero_moments()
        a.copy_planes_from(c, 2, 1, 2, -1)      # planes 2, 3 of c into planes 1, 2 of a, every class
        got = a.get_moments()
    assert np.array_equal(got[:, 1:3], u[:, 2:4]) and not got[:, [0, 3]].any()
