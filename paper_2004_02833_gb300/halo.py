"""Domain decomposition with one-layer halos, for running the step on several ranks.

The paper distributes the domain in blocks over MPI ranks and refreshes a one-cell ghost layer per
face before each sweep (Section 3).  `SlabHalo` splits z into slabs of whole planes, `BlockHalo`
splits x, y and z over a process grid; before a substep of class A (Eq. 5 with the dual class B
frozen) each rank fills its ghost layers with the class-B layers of its neighbours.  A half-grid difference along z reads one neighbour plane only
(Section 2.1): a target on z-slot 2 reads its sources (on z-slot 1) at i + 1, a target on z-slot 1
reads its sources (on z-slot 2) at i - 1.  So the upper ghost plane needs only the class-B
components on z-slot 1 and the lower one those on z-slot 2, about a quarter of the (N+1)^2 moments
per face and substep (the same holds along x and y with the x- and y-slots).

The exchange is point to point (``torch.distributed`` isend/irecv: gloo on the CPU, NCCL on GPUs),
not a collective, and it does not depend on how the local substep is computed.  Local arrays are
``[c][z][y][x]`` in the interface order c = l*l + l + m, with a ghost plane at z index 0 when the
slab has a lower neighbour and one at the last z index when it has an upper neighbour; with
periodic boundaries every slab has both (a single rank is its own neighbour).
"""
from __future__ import annotations

from dataclasses import dataclass

from . import rtpn


def slabs(nz: int, world: int) -> list[tuple[int, int]]:
    """[z0, z1) of every rank: nz planes split as evenly as possible (ranks < nz % world get one
    more)."""
    if world < 1 or nz < world:
        raise ValueError("need at least one z plane per rank")
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


@dataclass
class SlabHalo:
    """The halo of one rank's slab.  `upper_sources[A]` / `lower_sources[A]`: the interface indices
    of the class-(1 - A) components that a substep of class A reads across the upper / lower face."""

    N: int
    nz: int
    rank: int
    world: int
    periodic: bool

    def __post_init__(self):
        self.z0, self.z1 = slabs(self.nz, self.world)[self.rank]
        last = self.world - 1
        self.lower = self.rank - 1 if self.rank > 0 else (last if self.periodic else None)
        self.upper = self.rank + 1 if self.rank < last else (0 if self.periodic else None)
        n_c = (self.N + 1) ** 2
        info = [rtpn.component_info(self.N, c) for c in range(n_c)]
        self.upper_sources, self.lower_sources = {}, {}
        for A in (0, 1):
            B = 1 - A
            self.upper_sources[A] = [c for c, (_, _, s, k) in enumerate(info) if k == B and s[2] == 1]
            self.lower_sources[A] = [c for c, (_, _, s, k) in enumerate(info) if k == B and s[2] == 2]

    @property
    def lo(self) -> int:
        """z index of the first own plane in the local array."""
        return 1 if self.lower is not None else 0

    @property
    def local_nz(self) -> int:
        """z planes of the local array: own planes plus ghosts."""
        return (self.z1 - self.z0) + self.lo + (1 if self.upper is not None else 0)

    def global_planes(self) -> list[int]:
        """The global z plane of every local plane (ghosts wrapped when periodic)."""
        return [(self.z0 - self.lo + i) % self.nz for i in range(self.local_nz)]

    def exchange(self, u, A: int, dist=None) -> None:
        """Fills the ghost planes of the local state `u` (a torch tensor [c][z][y][x]) with the
        neighbours' planes that a substep of class A reads.  Every rank calls it before every
        substep; `dist` is torch.distributed (None: one rank only)."""
        import torch

        top, bot = u.shape[1] - 1, 0
        own_bot, own_top = self.lo, self.lo + (self.z1 - self.z0) - 1
        up_idx = torch.tensor(self.upper_sources[A], dtype=torch.long, device=u.device)
        lo_idx = torch.tensor(self.lower_sources[A], dtype=torch.long, device=u.device)
        # my lowest own plane goes to the lower neighbour's upper ghost, my highest own plane to
        # the upper neighbour's lower ghost
        send_down = u[up_idx, own_bot].contiguous() if self.lower is not None else None
        send_up = u[lo_idx, own_top].contiguous() if self.upper is not None else None
        recv_up = torch.empty_like(u[up_idx, 0]) if self.upper is not None else None
        recv_lo = torch.empty_like(u[lo_idx, 0]) if self.lower is not None else None
        if self.world == 1 or dist is None:
            if self.upper is not None:
                recv_up.copy_(send_down)
            if self.lower is not None:
                recv_lo.copy_(send_up)
        else:
            # tag 0: a plane travelling down (into an upper ghost), tag 1: travelling up
            reqs = []
            if self.upper is not None:
                reqs.append(dist.irecv(recv_up, src=self.upper, tag=0))
                reqs.append(dist.isend(send_up, dst=self.upper, tag=1))
            if self.lower is not None:
                reqs.append(dist.irecv(recv_lo, src=self.lower, tag=1))
                reqs.append(dist.isend(send_down, dst=self.lower, tag=0))
            for r in reqs:
                r.wait()
        if self.upper is not None:
            u[up_idx, top] = recv_up
        if self.lower is not None:
            u[lo_idx, bot] = recv_lo


def _split(n: int, parts: int) -> list[tuple[int, int]]:
    return slabs(n, parts)


@dataclass
class BlockHalo:
    """The halo of one rank's block in a px x py x pz process grid (rank = (kz * py + ky) * px + kx,
    x fastest), the block decomposition of the paper (Section 3) with one ghost layer per face.
    Along every axis d the upper ghost layer receives the class-B components on d-slot 1 and the
    lower one those on d-slot 2 (`upper_sources[A][d]`, `lower_sources[A][d]`).  A difference runs
    along one axis only, so faces suffice: edge and corner ghost cells of the state are never read
    (the media of the whole ghosted box are input data, taken from the global arrays)."""

    N: int
    shape: tuple          # global (nz, ny, nx)
    dims: tuple           # process grid (px, py, pz)
    rank: int
    periodic: bool

    def __post_init__(self):
        px, py, pz = self.dims
        if px * py * pz < 1 or self.rank >= px * py * pz:
            raise ValueError("rank outside the process grid")
        self.coords = (self.rank % px, (self.rank // px) % py, self.rank // (px * py))
        n = (self.shape[2], self.shape[1], self.shape[0])  # along x, y, z
        self.lo_hi = [_split(n[d], self.dims[d])[self.coords[d]] for d in range(3)]
        self.lower, self.upper = [], []
        for d in range(3):
            k, p = self.coords[d], self.dims[d]
            lower = k - 1 if k > 0 else (p - 1 if self.periodic else None)
            upper = k + 1 if k < p - 1 else (0 if self.periodic else None)
            self.lower.append(None if lower is None else self._rank_with(d, lower))
            self.upper.append(None if upper is None else self._rank_with(d, upper))
        n_c = (self.N + 1) ** 2
        info = [rtpn.component_info(self.N, c) for c in range(n_c)]
        self.upper_sources, self.lower_sources = {}, {}
        for A in (0, 1):
            B = 1 - A
            self.upper_sources[A] = [[c for c, (_, _, s, k) in enumerate(info) if k == B and s[d] == 1]
                                     for d in range(3)]
            self.lower_sources[A] = [[c for c, (_, _, s, k) in enumerate(info) if k == B and s[d] == 2]
                                     for d in range(3)]

    def _rank_with(self, d: int, k: int) -> int:
        c = list(self.coords)
        c[d] = k
        px, py, _ = self.dims
        return (c[2] * py + c[1]) * px + c[0]

    def first(self, d: int) -> int:
        """Local index of the first own cell along axis d (1 with a lower ghost layer)."""
        return 1 if self.lower[d] is not None else 0

    def own(self, d: int) -> int:
        return self.lo_hi[d][1] - self.lo_hi[d][0]

    def local_n(self, d: int) -> int:
        return self.own(d) + self.first(d) + (1 if self.upper[d] is not None else 0)

    def global_index(self, d: int) -> list[int]:
        """The global cell index along axis d of every local index (ghosts wrapped when periodic)."""
        n = (self.shape[2], self.shape[1], self.shape[0])[d]
        return [(self.lo_hi[d][0] - self.first(d) + i) % n for i in range(self.local_n(d))]

    def own_slices(self):
        """Slices of the own cells in a local [.., z, y, x] array."""
        return tuple(slice(self.first(d), self.first(d) + self.own(d)) for d in (2, 1, 0))

    def ghost_slices(self):
        """One index tuple per ghost face of a local [c, z, y, x] array."""
        out = []
        for d in range(3):
            ax = 3 - d
            for present, at in ((self.lower[d] is not None, 0), (self.upper[d] is not None, self.local_n(d) - 1)):
                if present:
                    idx = [slice(None)] * 4
                    idx[ax] = at
                    out.append(tuple(idx))
        return out

    def exchange(self, u, A: int, dist=None) -> None:
        """Fills the face ghost layers of the local state `u` (torch [c][z][y][x]) that a substep of
        class A reads, axis by axis; `dist` is torch.distributed (None: one rank only)."""
        import torch

        world = self.dims[0] * self.dims[1] * self.dims[2]
        for d in range(3):
            ax = 3 - d  # array axis of x, y, z in [c, z, y, x]
            if self.lower[d] is None and self.upper[d] is None:
                continue
            own_lo = self.first(d)
            own_hi = own_lo + self.own(d) - 1
            inner = [slice(self.first(e), self.first(e) + self.own(e)) for e in range(3)]

            def layer(at, comps):
                idx = [slice(None)] * 4
                idx[0] = torch.tensor(comps, dtype=torch.long, device=u.device)
                for e in range(3):
                    idx[3 - e] = at if e == d else inner[e]
                return tuple(idx)

            up_c, lo_c = self.upper_sources[A][d], self.lower_sources[A][d]
            send_down = u[layer(own_lo, up_c)].contiguous() if self.lower[d] is not None else None
            send_up = u[layer(own_hi, lo_c)].contiguous() if self.upper[d] is not None else None
            recv_up = torch.empty_like(u[layer(own_lo, up_c)]) if self.upper[d] is not None else None
            recv_lo = torch.empty_like(u[layer(own_hi, lo_c)]) if self.lower[d] is not None else None
            if world == 1 or dist is None or self.upper[d] == self.rank:
                # one block along a periodic axis is its own neighbour: a local copy
                if recv_up is not None:
                    recv_up.copy_(send_down)
                if recv_lo is not None:
                    recv_lo.copy_(send_up)
            else:
                reqs = []
                if self.upper[d] is not None:
                    reqs.append(dist.irecv(recv_up, src=self.upper[d], tag=2 * d))
                    reqs.append(dist.isend(send_up, dst=self.upper[d], tag=2 * d + 1))
                if self.lower[d] is not None:
                    reqs.append(dist.irecv(recv_lo, src=self.lower[d], tag=2 * d + 1))
                    reqs.append(dist.isend(send_down, dst=self.lower[d], tag=2 * d))
                for r in reqs:
                    r.wait()
            if recv_up is not None:
                u[layer(self.local_n(d) - 1, up_c)] = recv_up
            if recv_lo is not None:
                u[layer(0, lo_c)] = recv_lo


class DeviceSlabs:
    """The z-slab decomposition on library contexts: one context per slab on the current device,
    each holding its own planes plus the ghost planes of `SlabHalo`, advanced pass by pass
    (``Context.substep``) with the ghost planes refreshed device to device after every pass
    (``Context.copy_planes_from``, rtpn_copy_planes): after a pass on class A, each face's ghost
    receives the neighbour's outermost own plane of class A, which the next pass (on the other
    class) reads.  The passes follow the library's merged schedule of Eq. (6), so the slabs
    together take the same steps as one context over the whole grid.  The values a context
    computes on its own ghost planes are never used: the exchange overwrites them first.

    On one GPU this is the exchange pattern of the multi-GPU decomposition with the transport a
    device copy; across GPUs the same planes travel by point-to-point sends (``SlabHalo``).
    """

    def __init__(self, N: int, shape, h: float, bc: str, precision: str, dt: float, slabs_: int,
                 kernel: str = "auto"):
        nz, ny, nx = shape
        self.shape = tuple(shape)
        self.periodic = bc == "periodic"
        self.halos = [SlabHalo(N, nz, r, slabs_, self.periodic) for r in range(slabs_)]
        self.ctx = []
        for hl in self.halos:
            c = rtpn.Context(N, (hl.local_nz, ny, nx), h, bc, precision, dt)
            if kernel != "auto":
                c.set_kernel(kernel)
            self.ctx.append(c)

    def close(self):
        for c in self.ctx:
            c.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        for c in self.ctx:
            c.set_stream(stream)

    def set_media(self, sigma_a, sigma_s, q):
        """Per-cell media of the whole grid [z][y][x] (host arrays); each slab takes its planes,
        ghosts included."""
        for hl, c in zip(self.halos, self.ctx):
            zs = hl.global_planes()
            c.set_media(sigma_a[zs], sigma_s[zs], q[zs])

    def set_moments(self, u):
        """The whole state [c][z][y][x] (interface order, host array); ghosts included."""
        for hl, c in zip(self.halos, self.ctx):
            c.set_moments(u[:, hl.global_planes()])

    def get_moments(self):
        """The whole state from the slabs' own planes (host FP64)."""
        import numpy as np

        out = None
        for hl, c in zip(self.halos, self.ctx):
            part = c.get_moments()
            if out is None:
                out = np.empty((part.shape[0],) + self.shape)
            out[:, hl.z0:hl.z1] = part[:, hl.lo:hl.lo + (hl.z1 - hl.z0)]
        return out

    def _exchange(self, cls: int):
        for r, hl in enumerate(self.halos):
            if hl.upper is None:
                continue
            up = self.halos[hl.upper]
            mine, theirs = self.ctx[r], self.ctx[hl.upper]
            own_top = hl.lo + (hl.z1 - hl.z0) - 1
            # my highest own plane -> the upper neighbour's lower ghost (local plane 0), and its
            # lowest own plane -> my upper ghost (my last local plane)
            theirs.copy_planes_from(mine, own_top, 0, 1, cls)
            mine.copy_planes_from(theirs, up.lo, hl.local_nz - 1, 1, cls)

    def _pass(self, cls: int, half: bool):
        for c in self.ctx:
            c.substep(cls, half)
        self._exchange(cls)

    def step(self, k: int = 1):
        """k steps of Eq. (6) in the merged schedule: odd dt/2, then (even dt, odd dt) k - 1 times,
        even dt, odd dt/2."""
        if k <= 0:
            return
        self._pass(1, True)
        for s in range(k):
            self._pass(0, False)
            self._pass(1, s == k - 1)

    def synchronize(self):
        for c in self.ctx:
            c.synchronize()
