"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method itself. It only produces the
*inputs* a user of the OEFE solver would supply:

* the periodic cell, nuclear positions and charges (paper Sec. V systems,
  replaced by the synthetic cells described in ``CONFIGS``);
* per-axis mesh breakpoints graded toward the nuclei (the paper's meshes are
  "refined toward nuclei", Sec. V; the grading recipe is ours);
* radial tables R(r), R'(r) of the atomic orbitals used as enrichment
  (paper Eq. KSAtomicTrunc uses orbitals of the isolated atom from an external
  radial solver; here hydrogenic 1s/2s/2p with exponent Z stand in for them);
* a frozen effective potential V_eff(x) (a sum of Gaussian-smeared nuclear
  Coulomb potentials on the minimal image) evaluated at caller-given points;
* Monkhorst-Pack k-points with equal weights (paper Eq. rho);
* random starting vectors X0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.special import erf

# Enrichment function codes per atom, in order 1s, 2s, 2p_x, 2p_y, 2p_z.
# Each entry is (n, l, m) with m in {0: s, 1: x, 2: y, 3: z} for l = 1.
ORBITALS_1S_2P = ((1, 0, 0), (2, 0, 0), (2, 1, 1), (2, 1, 2), (2, 1, 3))


@dataclass
class Workload:
    name: str
    a: float                      # cubic cell edge (bohr)
    pos: np.ndarray               # (natoms, 3) nuclear positions (bohr)
    Z: np.ndarray                 # (natoms,) nuclear charges
    ncell: int                    # cells per axis
    p: int                        # FE polynomial order
    nv: list                      # vectors per k-point
    degree: int                   # Chebyshev degree per pass
    kgrid: tuple = (1, 1, 1)      # Monkhorst-Pack grid
    dtype: str = "f64"            # filter arithmetic of the plain path
    grading_ratio: float = 1.5
    sigma: float = 0.05           # Gaussian width of the smoothed nuclei
    r0: float = 3.0               # enrichment cutoff: h = 1 below r0
    rc: float = 4.0               # enrichment cutoff: h = 0 above rc
    ngrid: int = 2000             # radial table points on [0, rc]
    nq_cell: int = 0              # Gauss points per axis, plain cells (0: p+1)
    nq_enr: int = 0               # Gauss points per axis, enriched leaves (0: p+3)
    refine_depth: int = 6         # octree depth toward nuclei
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def natoms(self):
        return len(self.Z)

    @property
    def nelectrons(self):
        return int(np.sum(self.Z))

    def quad_params(self):
        return (self.nq_cell or self.p + 1, self.nq_enr or self.p + 3, self.refine_depth)


def _zincblende(a):
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    pos = np.concatenate([fcc, fcc + 0.25]) * a
    Z = np.array([14] * 4 + [6] * 4)
    return pos, Z


def config_c1():
    a = 10.26
    pos = np.array([[0.0, 0.0, 0.0], [a / 4, a / 4, a / 4]])
    return Workload("c1_fp64_gamma_2atom_8cube_p4", a, pos, np.array([6, 14]), 8, 4, [20], 20)


def config_c2():
    a = 8.5
    pos, Z = _zincblende(a)
    return Workload("c2_fp64_4k_8atom_16cube_p6", a, pos, Z, 16, 6, [64] * 4, 30,
                    kgrid=(2, 2, 1), dtype="c128")


def config_c3():
    w = config_c2()
    w.name = "c3_mixed_4k_8atom_16cube_p6"
    w.dtype = "c64"
    return w


def config_c4():
    a = 12.0
    rng = np.random.default_rng(1)
    sites, Z = [], []
    for s in (0.0, 0.5):
        for k in range(2):
            for j in range(2):
                for i in range(2):
                    sites.append([(i + s) * 6.0, (j + s) * 6.0, (k + s) * 6.0])
                    Z.append(6 if (i + j + k + int(2 * s)) % 2 == 0 else 14)
    pos = np.array(sites) + rng.uniform(-0.1, 0.1, (16, 3))
    pos = np.mod(pos, a)
    nv = [int(v) for v in rng.integers(96, 129, 8)]
    return Workload("c4_c64_8k_16atom_20cube_p6", a, pos, np.array(Z), 20, 6, nv, 30,
                    kgrid=(2, 2, 2), dtype="c64", seed=1)


def config_c5():
    a0 = 8.2
    cell, Zc = _zincblende(a0)
    pos, Z = [], []
    for k in range(2):
        for j in range(2):
            for i in range(2):
                pos.append(cell + a0 * np.array([i, j, k]))
                Z.append(Zc)
    pos = np.concatenate(pos)
    Z = np.concatenate(Z)
    # divacancy: drop the Z=14 site at the origin and its nearest Z=6 neighbour
    keep = np.ones(len(Z), bool)
    keep[0] = False
    d = np.linalg.norm(pos - pos[0], axis=1)
    d[Z != 6] = np.inf
    keep[int(np.argmin(d))] = False
    return Workload("c5_mixed_gamma_62atom_32cube_p6", 2 * a0, pos[keep], Z[keep], 32, 6,
                    [360], 50, dtype="f32")


def config_c3_small():
    """The c3 cell with an 8^3 graded mesh and one k-point: a profiling case
    whose cell matrices (~0.6 GB) still exceed the L2 cache."""
    w = config_c2()
    w.name = "c3small_8atom_8cube_p6_1k"
    w.ncell = 8
    w.nv = [64, 64]
    w.kgrid = (2, 1, 1)
    w.dtype = "c64"
    return w


def config_c3_mid():
    """The c3 cell on a 12^3 graded mesh with two k-points: a profiling case
    whose vectors (0.19 GB) and cell products (0.34 GB per k) exceed the L2
    cache like the full workload's, at 2 GB of split cell matrices per k."""
    w = config_c2()
    w.name = "c3mid_8atom_12cube_p6_2k"
    w.ncell = 12
    w.nv = [64, 64]
    w.kgrid = (2, 1, 1)
    w.dtype = "c64"
    return w


def config_c4_mid():
    """The 16-atom cell of the batched-k configuration (8 complex k-points, 97-123 vectors each) on
    a 12^3 graded mesh: the whole configuration at about a fifth of the mesh, since at 20^3 its
    operator data, vectors and batched-filter workspaces exceed one device's memory."""
    w = config_c4()
    w.name = "c4mid_c64_8k_16atom_12cube_p6"
    w.ncell = 12
    return w


def config_c5_mid():
    """The 62-atom divacancy supercell on a 16^3 graded mesh (about 0.9M nodes): a test case of the
    Gamma-point path with 360 vectors at an eighth of the large supercell's mesh."""
    w = config_c5()
    w.name = "c5mid_gamma_62atom_16cube_p6"
    w.ncell = 16
    return w


CONFIGS = {"c1": config_c1, "c3small": config_c3_small, "c3mid": config_c3_mid, "c2": config_c2, "c3": config_c3, "c4": config_c4, "c5": config_c5, "c5mid": config_c5_mid,
           "c4mid": config_c4_mid}


def graded_breakpoints(a, ncell, coords, ratio=1.5, tol=1e-3):
    """Per-axis cell boundaries (ncell+1 values, 0 .. a) refined toward nuclei.

    The distinct nuclear coordinates (mod a) on this axis become breakpoints.
    If there are at most ncell/2 of them, cells are shared out among the
    intervals in proportion to their length (largest remainder, at least 2
    each) and each interval is graded symmetrically from both ends with
    geometric ratio ``ratio``; otherwise the mesh is uniform.
    """
    c = np.sort(np.mod(np.asarray(coords, float), a))
    uniq = []
    for x in c:
        if not uniq or x - uniq[-1] > tol:
            uniq.append(x)
    if len(uniq) > 1 and (uniq[0] + a) - uniq[-1] <= tol:
        uniq.pop()
    if len(uniq) == 0 or len(uniq) > ncell // 2:
        return np.linspace(0.0, a, ncell + 1)
    # shift so the first breakpoint sits at 0: intervals start at nuclei
    if uniq[0] > tol:
        # the mesh must start at 0; keep 0 as an extra breakpoint
        uniq = [0.0] + uniq
    ends = uniq + [a]
    lengths = np.diff(ends)
    nint = len(lengths)
    share = lengths / a * ncell
    counts = np.maximum(np.floor(share).astype(int), 2)
    while counts.sum() > ncell:
        j = int(np.argmax(counts - share))
        counts[j] -= 1
    rem = share - np.floor(share)
    while counts.sum() < ncell:
        j = int(np.argmax(rem))
        counts[j] += 1
        rem[j] = -1
    out = [0.0]
    for L, n, x0 in zip(lengths, counts, ends[:-1]):
        half = [ratio ** i for i in range((n + 1) // 2)]
        w = half + half[::-1][(n % 2):]
        w = np.array(w) / np.sum(w) * L
        acc = x0
        for wi in w[:-1]:
            acc += wi
            out.append(acc)
        out.append(x0 + L)
    out = np.array(out)
    out[-1] = a
    return out


def mesh_breakpoints(w: Workload):
    """(3, ncell+1) per-axis breakpoints for a workload."""
    return np.stack([graded_breakpoints(w.a, w.ncell, w.pos[:, d], w.grading_ratio)
                     for d in range(3)])


def hydrogenic_radial(n, l, Z, r):
    """Analytic hydrogenic radial function R_nl and its derivative (atomic units)."""
    r = np.asarray(r, float)
    z32 = Z ** 1.5
    if (n, l) == (1, 0):
        e = np.exp(-Z * r)
        return 2 * z32 * e, -2 * Z * z32 * e
    if (n, l) == (2, 0):
        e = np.exp(-Z * r / 2)
        c = z32 / (2 * math.sqrt(2))
        f = (2 - Z * r)
        return c * f * e, c * (-Z * e - Z / 2 * f * e)
    if (n, l) == (2, 1):
        e = np.exp(-Z * r / 2)
        c = z32 / (2 * math.sqrt(6)) * Z
        return c * r * e, c * (e - Z / 2 * r * e)
    raise ValueError("only 1s, 2s, 2p radial functions are tabulated")


def radial_tables(Z, orbitals=ORBITALS_1S_2P, rc=4.0, ngrid=2000):
    """Tables R, dR of shape (natoms, nfun, ngrid) on the uniform grid [0, rc]."""
    r = np.linspace(0.0, rc, ngrid)
    R = np.zeros((len(Z), len(orbitals), ngrid))
    dR = np.zeros_like(R)
    for I, z in enumerate(Z):
        for j, (n, l, _m) in enumerate(orbitals):
            R[I, j], dR[I, j] = hydrogenic_radial(n, l, float(z), r)
    return R, dR


def orbital_lm_codes(orbitals=ORBITALS_1S_2P):
    """Angular code per function: 0 = s, 1/2/3 = p_x/p_y/p_z."""
    return np.array([m if l == 1 else 0 for (_n, l, m) in orbitals], dtype=np.int32)


def veff(points, a, pos, Z, sigma=0.05):
    """Frozen synthetic V_eff at points (npts, 3): sum over nuclei of the
    Gaussian-smeared Coulomb potential -Z erf(r / (sqrt(2) sigma)) / r on the
    minimal image (no lattice sum)."""
    pts = np.asarray(points, float)
    V = np.zeros(len(pts))
    s2 = math.sqrt(2.0) * sigma
    for R, z in zip(pos, Z):
        d = pts - R
        d -= a * np.round(d / a)
        r = np.sqrt(np.sum(d * d, axis=1))
        small = r < 1e-12
        rr = np.where(small, 1.0, r)
        v = -z * erf(rr / s2) / rr
        v[small] = -z * math.sqrt(2.0 / math.pi) / sigma
        V += v
    return V


def veff_device(points, a, pos, Z, sigma=0.05, device="cuda"):
    """The same V_eff as ``veff`` evaluated with torch on a device (large point sets); returns a
    float64 tensor on ``device``. Input generation only: the formula is that of ``veff``."""
    import torch
    pts = torch.as_tensor(np.asarray(points, float), dtype=torch.float64, device=device)
    V = torch.zeros(pts.shape[0], dtype=torch.float64, device=device)
    s2 = math.sqrt(2.0) * sigma
    for R, z in zip(np.asarray(pos, float), Z):
        d = pts - torch.as_tensor(R, dtype=torch.float64, device=device)
        d = d - a * torch.round(d / a)
        r = torch.sqrt(torch.sum(d * d, dim=1))
        small = r < 1e-12
        rr = torch.where(small, torch.ones_like(r), r)
        v = -float(z) * torch.special.erf(rr / s2) / rr
        v = torch.where(small, torch.full_like(v, -float(z) * math.sqrt(2.0 / math.pi) / sigma), v)
        V += v
    return V


def monkhorst_pack(a, q):
    """Full Monkhorst-Pack grid (no symmetry reduction), Cartesian bohr^-1, equal weights."""
    b = 2 * math.pi / a
    ks = []
    for r3 in range(q[2]):
        for r2 in range(q[1]):
            for r1 in range(q[0]):
                f = [(2 * (r + 1) - qq - 1) / (2 * qq) for r, qq in zip((r1, r2, r3), q)]
                ks.append([fi * b for fi in f])
    k = np.array(ks, float)
    return k, np.full(len(k), 1.0 / len(k))


def random_vectors(n, nv, complex_=False, seed=0, ld=None):
    """X0 uniform in [-1, 1]; for complex, the imaginary part is drawn next."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, (n, nv))
    if complex_:
        X = X + 1j * rng.uniform(-1.0, 1.0, (n, nv))
    if ld is not None and ld > nv:
        Xp = np.zeros((n, ld), X.dtype)
        Xp[:, :nv] = X
        X = Xp
    return X
