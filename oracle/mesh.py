"""Periodic rectilinear spectral-element mesh (Sec. III A).

Reading (the paper does not fix the mesh data structure): the periodic cubic
cell [0, a)^3 is split by per-axis breakpoints into n_x * n_y * n_z hexahedral
cells. Cell (ix, iy, iz) has index e = ix + n_x (iy + n_y iz). Each axis has
N_d = n_d p distinct periodic nodes; local node (i, j, k) of a cell, local
index i + (p+1)(j + (p+1) k), is global node gx + N_x (gy + N_y gz) with
g_d = (cell_d p + local_d) mod N_d.
"""
import numpy as np

from .fe1d import gll


class Mesh:
    def __init__(self, a, xb, p):
        self.a = float(a)
        self.xb = [np.asarray(b, float) for b in xb]
        self.p = int(p)
        self.nc = np.array([len(b) - 1 for b in self.xb])
        for b in self.xb:
            if abs(b[0]) > 0 or abs(b[-1] - a) > 1e-12 * a or np.any(np.diff(b) <= 0):
                raise ValueError("breakpoints must increase from 0 to a")
        self.N = self.nc * self.p
        self.nh = int(np.prod(self.N))
        self.ncells = int(np.prod(self.nc))
        self.P = self.p + 1
        self.nloc = self.P ** 3
        self.xi, self.wgll = gll(self.p)

    def cell_ijk(self, e):
        ix = e % self.nc[0]
        iy = (e // self.nc[0]) % self.nc[1]
        iz = e // (self.nc[0] * self.nc[1])
        return ix, iy, iz

    def cell_box(self, e):
        ix, iy, iz = self.cell_ijk(e)
        lo = np.array([self.xb[0][ix], self.xb[1][iy], self.xb[2][iz]])
        hi = np.array([self.xb[0][ix + 1], self.xb[1][iy + 1], self.xb[2][iz + 1]])
        return lo, hi

    def cell_nodes(self, e):
        """Global node ids of the cell's local nodes, in local order."""
        ix, iy, iz = self.cell_ijk(e)
        r = np.arange(self.P)
        gx = (ix * self.p + r) % self.N[0]
        gy = (iy * self.p + r) % self.N[1]
        gz = (iz * self.p + r) % self.N[2]
        return (gx[None, None, :] + self.N[0] * (gy[None, :, None] + self.N[1] * gz[:, None, None])).ravel()

    def node_coords(self):
        """(nh, 3) coordinates of the global nodes in [0, a)."""
        out = np.zeros((self.nh, 3))
        for e in range(self.ncells):
            lo, hi = self.cell_box(e)
            h = hi - lo
            x = [lo[d] + (self.xi + 1) / 2 * h[d] for d in range(3)]
            X = np.stack(np.meshgrid(x[0], x[1], x[2], indexing="ij"), -1)  # (P,P,P,3) [i,j,k]
            X = np.transpose(X, (2, 1, 0, 3)).reshape(-1, 3)                 # local order
            out[self.cell_nodes(e)] = np.mod(X, self.a)
        return out

    def lumped_mass(self):
        """Diagonal CFE overlap M^cc under GLL quadrature (Eq. orthCGLL denominator):
        m_l = sum over cells containing node l of w_i w_j w_k h_x h_y h_z / 8."""
        m = np.zeros(self.nh)
        w3 = (self.wgll[None, None, :] * self.wgll[None, :, None] * self.wgll[:, None, None]).ravel()
        for e in range(self.ncells):
            lo, hi = self.cell_box(e)
            np.add.at(m, self.cell_nodes(e), w3 * np.prod(hi - lo) / 8.0)
        return m

    def neighbours(self, e):
        """The 27 cells (periodic, with repeats for small meshes) around cell e."""
        ix, iy, iz = self.cell_ijk(e)
        out = []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    jx = (ix + dx) % self.nc[0]
                    jy = (iy + dy) % self.nc[1]
                    jz = (iz + dz) % self.nc[2]
                    out.append(jx + self.nc[0] * (jy + self.nc[1] * jz))
        return sorted(set(out))
