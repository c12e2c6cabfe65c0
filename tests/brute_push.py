"""Brute-force D3Q19 BGK stepper for tiny lattices (pure Python, float64).

An independent formulation used only to pin the oracle on small inputs: the
state is a dict {cell: [19 post-collision values]} over fluid cells, the
velocity set is the textbook table written out literally (Qian, d'Humieres &
Lallemand 1992) in an order of its own, streaming is written as a PUSH
(each value travels to x + c_i, or is reflected back to x as the opposite
direction when x + c_i is solid), and the equilibrium and Guo source are
written in terms of the sound speed c_s.  None of this is shared with the
oracle (pull, enumerated velocity set, numeric coefficients).
"""
from __future__ import annotations

CS2 = 1.0 / 3.0
# (c, w): rest, 6 faces, 12 edges of the cube -- D3Q19
TABLE = [((0, 0, 0), 1.0 / 3.0)]
for a in range(3):
    for s in (1, -1):
        c = [0, 0, 0]
        c[a] = s
        TABLE.append((tuple(c), 1.0 / 18.0))
for a, b in ((0, 1), (0, 2), (1, 2)):
    for sa in (1, -1):
        for sb in (1, -1):
            c = [0, 0, 0]
            c[a] = sa
            c[b] = sb
            TABLE.append((tuple(c), 1.0 / 36.0))
VEL = [t[0] for t in TABLE]
WGT = [t[1] for t in TABLE]
OPP = [VEL.index(tuple(-v for v in c)) for c in VEL]


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def feq(rho, u):
    uu = _dot(u, u)
    out = []
    for c, w in TABLE:
        cu = _dot(c, u)
        out.append(w * rho * (1 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2)))
    return out


def guo(tau, rho, u, g):
    F = [rho * g[0], rho * g[1], rho * g[2]]
    out = []
    for c, w in TABLE:
        cu = _dot(c, u)
        v = [(c[a] - u[a]) / CS2 + cu * c[a] / (CS2 * CS2) for a in range(3)]
        out.append((1 - 1 / (2 * tau)) * w * _dot(v, F))
    return out


class Brute:
    def __init__(self, nx, ny, nz, tau, u_lid, g, flags):
        """flags: callable (x,y,z) -> 0 fluid, 1 wall, 2 lid, 3 far field.

        A far-field cell is the free stream: it absorbs what is pushed into
        it and pushes, in every direction, the equilibrium of density 1
        moving at u_lid."""
        self.n = (nx, ny, nz)
        self.tau = tau
        self.u_lid = tuple(u_lid)
        self.g = tuple(g)
        self.flag = flags
        self.fluid = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)
                      if flags(x, y, z) == 0]
        self.P = {}

    def step(self):
        nx, ny, nz = self.n
        incoming = {cell: [None] * 19 for cell in self.fluid}
        # push streaming with reflection at solid cells
        for (x, y, z) in self.fluid:
            post = self.P[(x, y, z)]
            for i, c in enumerate(VEL):
                t = ((x + c[0]) % nx, (y + c[1]) % ny, (z + c[2]) % nz)
                kind = self.flag(*t)
                if kind == 0:
                    incoming[t][i] = post[i]
                elif kind == 3:
                    pass  # absorbed by the free stream
                else:
                    val = post[i]
                    if kind == 2:
                        # a moving wall hands back momentum 2 w_i rho_w (c.u_w)/cs^2
                        val -= 2.0 * WGT[i] * 1.0 * _dot(c, self.u_lid) / CS2
                    incoming[(x, y, z)][OPP[i]] = val
        # far-field cells push the free-stream equilibrium into the fluid
        f_free = feq(1.0, self.u_lid)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    if self.flag(x, y, z) != 3:
                        continue
                    for i, c in enumerate(VEL):
                        t = ((x + c[0]) % nx, (y + c[1]) % ny, (z + c[2]) % nz)
                        if self.flag(*t) == 0:
                            incoming[t][i] = f_free[i]
        # collide
        newP = {}
        for cell in self.fluid:
            f = incoming[cell]
            rho = sum(f)
            j = [sum(f[i] * VEL[i][a] for i in range(19)) for a in range(3)]
            u = [j[a] / rho + self.g[a] / 2 for a in range(3)]
            fe = feq(rho, u)
            S = guo(self.tau, rho, u, self.g)
            newP[cell] = [f[i] - (f[i] - fe[i]) / self.tau + S[i] for i in range(19)]
        self.P = newP
