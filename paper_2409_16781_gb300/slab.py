"""Z-slab decomposition of one lattice over several GPUs, one process each.

arXiv 2409.16781 names multi-GPU runs as future work (Sec. 6).  The update
is local (each cell pulls from its 18 neighbours only), so a lattice splits
into slabs of whole z-planes: rank r owns planes [z0, z1) and keeps one
ghost plane below and one above (lb_options.halo_z).  A step pulls only the
five c_z = +1 populations from the ghost plane below and the five c_z = -1
populations from the ghost plane above, so after every step each rank
sends its lowest own plane's c_z = -1 populations down and its highest own
plane's c_z = +1 populations up (a ring: z is periodic), 5*nx*ny values each
way, and unpacks what it receives into its ghost planes (lb_halo_pack /
lb_halo_unpack).  The exchange is point-to-point (torch.distributed
send/recv: NCCL between GPUs, gloo between CPU processes), never a
collective; the FP64 mass and momentum are summed over ranks with one
all-reduce of four doubles.  Done this way, the slabs take bitwise the steps
of the whole lattice.

This module is the host side of that scheme: the plane ranges, the ghosted
flag and field slices, and the exchange.  The exchange works with any local
lattice that can pack and unpack its halo into torch tensors (the CUDA
lattice of this package, or a CPU stand-in in the tests).
"""
from __future__ import annotations

import numpy as np


def slab_range(nz: int, world: int, rank: int):
    """Own z-planes [z0, z1) of `rank`: nz planes split into `world` runs
    whose lengths differ by at most one (the longer runs first)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    if nz < world:
        raise ValueError(f"{nz} planes cannot be split over {world} ranks")
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


def ghosted(a: np.ndarray, z0: int, z1: int, axis: int = 0) -> np.ndarray:
    """Planes z0-1 .. z1 of `a` along `axis` (periodic wrap): the own planes
    [z0, z1) with one ghost plane below and one above."""
    nz = a.shape[axis]
    idx = [(z0 - 1) % nz] + list(range(z0, z1)) + [z1 % nz]
    return np.ascontiguousarray(np.take(a, idx, axis=axis))


class SlabExchange:
    """The per-step halo exchange of one rank's slab with its z-neighbours.

    `local` provides halo_pack(send_lo, send_hi) and halo_unpack(recv_lo,
    recv_hi) on tensors it allocated (halo_buffers()).  With one rank the
    slab is its own neighbour both ways (periodic z) and no message is sent.
    """

    def __init__(self, rank: int = 0, world: int = 1, group=None, device=None):
        """device: where the all-reduce of sum() runs (a CUDA device for
        NCCL; None = the host, for gloo)."""
        self.rank, self.world, self.group = int(rank), int(world), group
        self.device = device
        self.up = (self.rank + 1) % self.world
        self.down = (self.rank - 1) % self.world

    def __call__(self, local):
        send_lo, send_hi, recv_lo, recv_hi = local.halo_buffers()
        local.halo_pack(send_lo, send_hi)
        if self.world == 1:
            local.halo_unpack(send_hi, send_lo)
            return
        import torch.distributed as dist
        # the message going up lands in the upper rank's lower ghost plane,
        # the one going down in the lower rank's upper ghost plane; with two
        # ranks both go to the same peer and are told apart by their tag
        # (gloo) or by their order (NCCL matches a peer's sends and receives
        # in issue order: up first, then down, on both sides)
        ops = [dist.P2POp(dist.isend, send_hi, self.up, self.group, 0),
               dist.P2POp(dist.isend, send_lo, self.down, self.group, 1),
               dist.P2POp(dist.irecv, recv_lo, self.down, self.group, 0),
               dist.P2POp(dist.irecv, recv_hi, self.up, self.group, 1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        local.halo_unpack(recv_lo, recv_hi)

    def sum(self, values):
        """Element-wise FP64 sum of `values` over the ranks (one all-reduce)."""
        import torch
        t = torch.tensor(np.asarray(values, dtype=np.float64), dtype=torch.float64,
                         device=self.device if self.device is not None else "cpu")
        if self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()


class SlabLattice:
    """This rank's z-slab of an nx x ny x nz lattice, advanced by liblbgb.

    Global arrays (flags, initial fields) are passed whole to every rank;
    each takes its own planes plus ghosts.  `exchange` defaults to the ranks
    of torch.distributed (one rank when it is not initialised).
    """

    def __init__(self, nx, ny, nz, tau, u_lid=(0.0, 0.0, 0.0), flags=None, storage="f32",
                 force=(0.0, 0.0, 0.0), rank=None, world=None, group=None, exchange=None,
                 device=None, stream=None, kernel=0, block=0):
        import torch
        from .lattice import Lattice
        if rank is None or world is None:
            import torch.distributed as dist
            on = dist.is_available() and dist.is_initialized()
            rank = dist.get_rank(group) if on else 0
            world = dist.get_world_size(group) if on else 1
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.rank, self.world = int(rank), int(world)
        self.z0, self.z1 = slab_range(self.nz, self.world, self.rank)
        self.nzl = self.z1 - self.z0 + 2
        fl = None
        if flags is not None:
            fl = ghosted(np.asarray(flags, dtype=np.uint8).reshape(self.nz, self.ny, self.nx), self.z0, self.z1)
        self.lattice = Lattice(self.nx, self.ny, self.nzl, tau, u_lid=u_lid, flags=fl, storage=storage,
                               force=force, device=device, stream=stream, kernel=kernel, block=block,
                               halo_z=True)
        if exchange is None:
            import torch.distributed as dist
            nccl = dist.is_available() and dist.is_initialized() and dist.get_backend(group) == "nccl"
            exchange = SlabExchange(self.rank, self.world, group, self.lattice.device if nccl else None)
        self.exchange = exchange
        nb = self.lattice.halo_bytes()
        dev = self.lattice.device
        self._bufs = tuple(torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(4))
        self.halo()

    # the local-lattice side of SlabExchange
    def halo_buffers(self):
        return self._bufs

    def halo_pack(self, send_lo, send_hi):
        self.lattice.halo_pack(send_lo, send_hi)

    def halo_unpack(self, recv_lo, recv_hi):
        self.lattice.halo_unpack(recv_lo, recv_hi)

    def halo(self):
        """The halo exchange of the current state (after a step or an
        initialisation of the local lattice)."""
        import torch
        with torch.cuda.stream(self.lattice.stream):
            self.exchange(self)

    # ------------------------------------------------------------------
    def init_fields(self, rho=None, u=None):
        """Equilibrium from global fields rho (nz, ny, nx) and u (3, nz, ny, nx)."""
        r = None if rho is None else ghosted(np.asarray(rho, dtype=np.float64), self.z0, self.z1)
        v = None if u is None else ghosted(np.asarray(u, dtype=np.float64), self.z0, self.z1, axis=1)
        self.lattice.init_fields(r, v)
        self.halo()

    def step(self, n: int = 1):
        """n steps, each followed by the halo exchange."""
        for _ in range(int(n)):
            self.lattice.step(1)
            self.halo()

    def totals(self):
        """Global FP64 (mass, momentum[3]): this slab's sums, all-reduced."""
        m, p = self.lattice.totals()
        s = self.exchange.sum([m, p[0], p[1], p[2]])
        return float(s[0]), s[1:4].copy()

    def own_moments(self):
        """(rho, u) of this slab's own planes: (z1-z0, ny, nx), (3, z1-z0, ny, nx)."""
        rho, u = self.lattice.moments()
        return rho[1:-1], u[:, 1:-1]

    def own_populations(self):
        """Populations of the own planes: (19, z1-z0, ny, nx)."""
        return self.lattice.populations()[:, 1:-1]
