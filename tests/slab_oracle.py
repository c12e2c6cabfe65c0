"""A z-slab of the FP64 oracle, for the CPU tests of the slab decomposition.

It plays the part of the CUDA lattice's slab (lb_options.halo_z) in
paper_2409_16781_gb300.slab.SlabExchange: the oracle advances the slab with
its ghost planes like any lattice, and halo_pack / halo_unpack move the same
values lb_halo_pack / lb_halo_unpack move -- the five c_z = -1 populations of
the lowest own plane and the five c_z = +1 populations of the highest own
plane out, into the c_z = +1 populations of the lower ghost plane and the
c_z = -1 populations of the upper ghost plane -- found here from the
oracle's own velocity set.  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2409_16781_gb300.slab import ghosted, slab_range


class OracleSlab:
    def __init__(self, nx, ny, nz, tau, u_lid, flags, force, rank, world):
        import torch
        self.nx, self.ny, self.nz = nx, ny, nz
        self.z0, self.z1 = slab_range(nz, world, rank)
        self.nzl = self.z1 - self.z0 + 2
        self.flags = ghosted(np.asarray(flags, dtype=np.uint8).reshape(nz, ny, nx), self.z0, self.z1)
        self.ora = O.Lattice(nx, ny, self.nzl, tau, u_lid=u_lid, flags=self.flags, force=force)
        c, _ = O.velocity_set()
        self.up = [i for i in range(19) if c[i][2] == 1]
        self.dn = [i for i in range(19) if c[i][2] == -1]
        assert len(self.up) == 5 and len(self.dn) == 5
        self._bufs = tuple(torch.zeros((5, ny, nx), dtype=torch.float64) for _ in range(4))

    def halo_buffers(self):
        return self._bufs

    def halo_pack(self, send_lo, send_hi):
        import torch
        A = self.ora.A
        for k in range(5):
            send_lo[k].copy_(torch.from_numpy(A[self.dn[k], 1].copy()))
            send_hi[k].copy_(torch.from_numpy(A[self.up[k], self.nzl - 2].copy()))

    def halo_unpack(self, recv_lo, recv_hi):
        A = self.ora.A
        for k in range(5):
            A[self.up[k], 0] = recv_lo[k].numpy()
            A[self.dn[k], self.nzl - 1] = recv_hi[k].numpy()

    def init_fields(self, rho, u):
        self.ora.init_fields(ghosted(rho, self.z0, self.z1), ghosted(u, self.z0, self.z1, axis=1))

    def step(self):
        self.ora.step(1)

    def own_populations(self):
        return self.ora.A[:, 1:-1].copy()

    def own_totals(self):
        """FP64 mass and momentum of the own planes' fluid cells."""
        rho, u = self.ora.moments()
        fluid = self.flags == O.FLUID
        fluid[0] = False
        fluid[-1] = False
        mass = float(rho[fluid].sum())
        mom = np.array([float((rho * u[a])[fluid].sum()) for a in range(3)])
        return mass, mom
