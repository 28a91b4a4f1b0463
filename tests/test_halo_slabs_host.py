"""The slab decomposition on device state (halo.DeviceSlabs), its schedule and ghost-plane exchange,
run on the CPU with each slab's library context replaced by the oracle on that slab's planes:
the slabs together must equal one oracle run over the whole grid (Section 3's one-layer halos,
Eq. 6).  The GPU test (tests/test_gpu_halo.py) runs the same with the library's kernels and
rtpn_copy_planes."""
import numpy as np
import pytest

from oracle import stepper as st
from paper_2004_02833_gb300 import halo, synth


class OracleSlab:
    """The calls DeviceSlabs makes on a context, served by the oracle on the slab's own grid."""

    mats = {}

    def __init__(self, N, shape, h, bc, precision, dt):
        self.N, self.shape, self.h, self.bc, self.dt = N, tuple(shape), h, bc, dt
        self.P = None
        self.u = None

    def set_kernel(self, kernel):
        pass

    def close(self):
        pass

    def set_media(self, sa, ss, q):
        mats, slots = OracleSlab.mats[self.N]
        self.P = st.Problem(self.N, np.array(sa), np.array(ss), np.array(q), self.h, self.dt, self.bc,
                            mats=mats, slots=slots)

    def set_moments(self, u):
        self.u = np.array(u, dtype=np.float64)

    def get_moments(self):
        return self.u.copy()

    def substep(self, cls, half=False):
        self.u = self.P.substep(self.u, cls, 0.5 * self.dt if half else self.dt)

    def copy_planes_from(self, src, src_z, dst_z, nz, cls=-1):
        m = np.ones(self.u.shape[0], bool) if cls == -1 else self.P.cls == cls
        self.u[m, dst_z:dst_z + nz] = src.u[m, src_z:src_z + nz]


@pytest.mark.parametrize("N,shape,bc,nslab,k", [
    (3, (12, 4, 5), "periodic", 2, 3),
    (3, (11, 4, 4), "vacuum", 3, 2),
    (1, (8, 3, 3), "periodic", 4, 4),
])
def test_device_slabs_logic_equals_one_grid(monkeypatch, coupling_cache, N, shape, bc, nslab, k):
    OracleSlab.mats[N] = coupling_cache(N)
    monkeypatch.setattr(halo.rtpn, "Context", OracleSlab)
    inst, u0 = synth.random_instance(N, shape, seed=1700 + N, bc=bc)
    mats, slots = coupling_cache(N)
    ref = st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, bc, mats=mats,
                     slots=slots).run(u0, k)
    with halo.DeviceSlabs(N, shape, inst.h, bc, "fp64", inst.dt, nslab) as sl:
        sl.set_media(inst.sigma_a, inst.sigma_s, inst.q)
        sl.set_moments(u0)
        sl.step(k)
        got = sl.get_moments()
    assert float(np.abs(got - ref).max() / np.abs(ref).max()) <= 1e-13
