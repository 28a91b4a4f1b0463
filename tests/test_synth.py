"""The seeded input generators hold no method arithmetic; these check the reactor-like cube's
geometry against its stated construction (Section 5.2 stand-in)."""
import numpy as np

from paper_2004_02833_gb300 import synth


def test_reactor_like_geometry():
    n = 64
    sa, ss, q = synth.reactor_media(n)
    shell = n // 16
    assert np.all(ss == 1.0)
    # concrete on every face, `shell` cells thick; water inside; rods carry q = 2 and no absorption
    for face in (sa[:shell], sa[-shell:], sa[:, :shell], sa[:, -shell:], sa[:, :, :shell], sa[:, :, -shell:]):
        assert np.all(face == 5.0)
    inner = sa[shell:-shell, shell:-shell, shell:-shell]
    assert set(np.unique(inner)) == {0.0, 10.0}
    assert np.array_equal(q > 0, sa == 0.0) and set(np.unique(q)) == {0.0, 2.0}
    # rods run along z with square 5 x 5 cross-sections on a 10-cell pitch
    mid = n // 2
    row = q[mid, mid] > 0
    runs = np.diff(np.flatnonzero(np.diff(np.r_[0, row.astype(int), 0])))[::2]
    assert len(runs) >= 2 and np.all(runs[:-1] == 5)
    starts = np.flatnonzero(np.diff(np.r_[0, row.astype(int)]) == 1)
    assert np.all(np.diff(starts) == 10)
    col = q[:, mid, np.flatnonzero(row)[0]] > 0
    assert col.sum() > n // 2 and np.all(np.diff(np.flatnonzero(col)) == 1)


def test_reactor_like_instance():
    inst = synth.reactor_like(7, 32)
    assert inst.bc == "vacuum" and inst.h == 0.2 and abs(inst.dt - 0.06) < 1e-15
    assert inst.shape == (32, 32, 32) and not inst.u0.any()
