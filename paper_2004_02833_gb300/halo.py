"""Slab decomposition along z with one-plane halos, for running the step on several ranks.

The paper distributes the domain in blocks over MPI ranks and refreshes a one-cell ghost layer per
face before each sweep (Section 3).  Here the unit is a slab of whole z planes per rank; before a
substep of class A (Eq. 5 with the dual class B frozen) each rank fills its ghost planes with the
class-B planes of its neighbours.  A half-grid difference along z reads one neighbour plane only
(Section 2.1): a target on z-slot 2 reads its sources (on z-slot 1) at i + 1, a target on z-slot 1
reads its sources (on z-slot 2) at i - 1.  So the upper ghost plane needs only the class-B
components on z-slot 1 and the lower one those on z-slot 2, about a quarter of the (N+1)^2 moments
per face and substep.

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
