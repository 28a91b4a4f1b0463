"""The multi-rank form of the step on CPU: gloo ranks, each stepping its z slab (here with the oracle
as the local substep), refresh their ghost planes with `halo.SlabHalo.exchange` before every
substep; the slabs put together must equal the one-rank run bit for bit, periodic and vacuum.  The
ghost planes are filled with NaN before every exchange, so each face's component list must hold
every component that the substep reads across it."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

N, SHAPE, STEPS = 3, (7, 5, 6), 3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _run_slab(rank, world, bc, dist=None):
    import torch

    from oracle import stepper as st
    from paper_2004_02833_gb300 import halo, synth

    inst, u0 = synth.random_instance(N, SHAPE, seed=77, bc=bc)
    H = halo.SlabHalo(N, SHAPE[0], rank, world, bc == "periodic")
    planes = H.global_planes()
    P = st.Problem(N, inst.sigma_a[planes], inst.sigma_s[planes], inst.q[planes], inst.h, inst.dt, bc)
    u = torch.tensor(u0[:, planes])
    ghosts = ([0] if H.lower is not None else []) + ([H.local_nz - 1] if H.upper is not None else [])
    for _ in range(STEPS):
        for cls, tau in ((1, 0.5 * inst.dt), (0, inst.dt), (1, 0.5 * inst.dt)):
            # ghost planes are pure receive buffers: whatever the exchange does not fill is NaN, so a
            # component missing from a face's list shows up in the result (the local substep would
            # otherwise keep half of them right by itself)
            u[:, ghosts] = float("nan")
            H.exchange(u, cls, dist)
            with np.errstate(invalid="ignore"):
                u = torch.tensor(P.substep(u.numpy(), cls, tau))
    own = slice(H.lo, H.lo + (H.z1 - H.z0))
    return H.z0, H.z1, u.numpy()[:, own]


def _worker(rank, world, port, bc, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + _run_slab(rank, world, bc, dist))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _reference(bc):
    from oracle import stepper as st
    from paper_2004_02833_gb300 import synth

    inst, u0 = synth.random_instance(N, SHAPE, seed=77, bc=bc)
    return st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, bc).run(u0, STEPS)


def test_slabs_cover_the_domain():
    from paper_2004_02833_gb300 import halo

    assert halo.slabs(7, 3) == [(0, 3), (3, 5), (5, 7)]
    with pytest.raises(ValueError):
        halo.slabs(2, 3)


def test_faces_carry_a_quarter_of_the_moments():
    from paper_2004_02833_gb300 import halo

    H = halo.SlabHalo(7, 8, 0, 2, True)
    n_c = 64
    for A in (0, 1):
        up, lo = H.upper_sources[A], H.lower_sources[A]
        assert not set(up) & set(lo) and len(up) + len(lo) == (28 if A == 1 else 36)
        assert abs(len(up) - n_c / 4) <= 4 and abs(len(lo) - n_c / 4) <= 4


@pytest.mark.parametrize("bc", ["periodic", "vacuum"])
def test_one_rank_slab_equals_the_plain_run(bc):
    # a single periodic slab is its own neighbour: ghost copies stand in for the wrap
    z0, z1, u = _run_slab(0, 1, bc)
    assert (z0, z1) == (0, SHAPE[0])
    assert np.array_equal(u, _reference(bc))


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("bc", ["periodic", "vacuum"])
def test_gloo_ranks_equal_one_rank_bitwise(bc, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, bc, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _reference(bc)
    got = np.empty_like(ref)
    for _, z0, z1, u in out:
        got[:, z0:z1] = u
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------- blocks in x, y and z
def _run_block(rank, dims, bc, dist=None):
    import torch

    from oracle import stepper as st
    from paper_2004_02833_gb300 import halo, synth

    inst, u0 = synth.random_instance(N, SHAPE, seed=78, bc=bc)
    H = halo.BlockHalo(N, SHAPE, dims, rank, bc == "periodic")
    gx, gy, gz = (H.global_index(d) for d in range(3))
    box = np.ix_(gz, gy, gx)
    P = st.Problem(N, inst.sigma_a[box], inst.sigma_s[box], inst.q[box], inst.h, inst.dt, bc)
    u = torch.tensor(u0[(slice(None),) + box])
    own = H.own_slices()
    outside = torch.ones(u.shape[1:], dtype=torch.bool)
    outside[own] = False
    for _ in range(STEPS):
        for cls, tau in ((1, 0.5 * inst.dt), (0, inst.dt), (1, 0.5 * inst.dt)):
            # everything outside the own block (faces, edges, corners) is NaN until the exchange
            # fills the face layers a substep of class `cls` reads
            u[:, outside] = float("nan")
            H.exchange(u, cls, dist)
            with np.errstate(invalid="ignore"):
                u = torch.tensor(P.substep(u.numpy(), cls, tau))
    lo = [H.lo_hi[d][0] for d in range(3)]
    hi = [H.lo_hi[d][1] for d in range(3)]
    return (lo[2], hi[2], lo[1], hi[1], lo[0], hi[0]), u.numpy()[(slice(None),) + own]


def _block_worker(rank, dims, port, bc, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    world = dims[0] * dims[1] * dims[2]
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + _run_block(rank, dims, bc, dist))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _block_reference(bc):
    from oracle import stepper as st
    from paper_2004_02833_gb300 import synth

    inst, u0 = synth.random_instance(N, SHAPE, seed=78, bc=bc)
    return st.Problem(N, inst.sigma_a, inst.sigma_s, inst.q, inst.h, inst.dt, bc).run(u0, STEPS)


@pytest.mark.parametrize("bc", ["periodic", "vacuum"])
def test_one_block_equals_the_plain_run(bc):
    box, u = _run_block(0, (1, 1, 1), bc)
    assert box == (0, SHAPE[0], 0, SHAPE[1], 0, SHAPE[2])
    assert np.array_equal(u, _block_reference(bc))


@pytest.mark.parametrize("dims", [(2, 1, 1), (1, 2, 1), (2, 2, 1), (1, 2, 2)])
@pytest.mark.parametrize("bc", ["periodic", "vacuum"])
def test_gloo_blocks_equal_one_rank_bitwise(bc, dims):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = dims[0] * dims[1] * dims[2]
    procs = [ctx.Process(target=_block_worker, args=(r, dims, port, bc, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _block_reference(bc)
    got = np.full_like(ref, np.nan)
    for _, (z0, z1, y0, y1, x0, x1), u in out:
        got[:, z0:z1, y0:y1, x0:x1] = u
    assert np.array_equal(got, ref)


def test_block_faces_carry_a_quarter_of_the_moments_on_every_axis():
    from paper_2004_02833_gb300 import halo

    H = halo.BlockHalo(7, (8, 8, 8), (2, 2, 2), 0, True)
    for A in (0, 1):
        n_b = 28 if A == 1 else 36  # class B at N = 7: even l (28) for A = 1, odd l (36) for A = 0
        for d in range(3):
            up, lo = H.upper_sources[A][d], H.lower_sources[A][d]
            assert not set(up) & set(lo) and len(up) + len(lo) == n_b
            assert abs(len(up) - 16) <= 4 and abs(len(lo) - 16) <= 4
    # neighbours of rank 0 in a periodic 2 x 2 x 2 grid: rank + 1 along x, + 2 along y, + 4 along z
    assert H.upper == [1, 2, 4] and H.lower == [1, 2, 4]
