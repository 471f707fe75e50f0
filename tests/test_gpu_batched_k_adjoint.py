"""The batched-k configuration's patterns at scale, on its 16-atom cell with a 12^3 graded mesh:
all eight complex k-points with uneven vector counts (97-123) in one persistent tensor-core launch
per degree (graph-captured, replayed), and the adjoint of the band trace tr(X^+ H(V) X) with respect
to the quadrature-point potential against central finite differences (h = 1e-4) and against the
oracle's fields on a block of cells (Sec. IV; Eq. HOEFEelelements, H affine in V; Eq. rho)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c4mid():
    import paper_2010_09701_gb300 as P
    w = W.CONFIGS["c4mid"]()
    ctx = P.setup_workload(w, device=0)
    xyz, qw = ctx.quadrature_points()
    V = W.veff_device(xyz, w.a, w.pos, w.Z, w.sigma, device="cuda")
    ctx.build_hamiltonian(V, P.STORE_F64 | P.STORE_BF16X3)
    return w, ctx, V, xyz


# the batched and per-k launches sum the FP32 products in different orders; the filter amplifies
# that rounding (each is within the mixed filter's own tolerance of the exact filter, 2e-4)
TOL_BATCHED = 1e-4


def colerr(out, ref):
    return np.max(np.linalg.norm(out - ref, axis=0) / np.linalg.norm(ref, axis=0))


def test_eight_kpoints_uneven_one_launch_per_degree(c4mid):
    import paper_2010_09701_gb300 as P
    w, ctx, V, _ = c4mid
    nh, nO = ctx.ndof()
    n = nh + nO
    assert ctx.nk == 8 and len(set(w.nv)) > 1 and min(w.nv) >= 96 and max(w.nv) <= 128
    Xs = [torch.tensor(W.random_vectors(n, nv, complex_=True, seed=60 + k), dtype=torch.complex128, device="cuda")
          for k, nv in enumerate(w.nv)]
    v0 = torch.tensor(W.random_vectors(n, 1, complex_=True, seed=9), dtype=torch.complex128, device="cuda")
    b = [ctx.upper_bound(k, v0, 20) for k in range(8)]
    a, a0, deg = 0.0, -0.5 * 14.0 ** 2 - 1.0, 6
    flags = P.FILTER_BF16X3 | P.FILTER_LAST_FP64
    ref = []
    for k in range(8):   # per k-point, one launch per degree each
        Y = Xs[k].clone()
        ctx.chebyshev_filter(k, Y, deg, a, b[k], a0, flags=flags)
        ref.append(Y.cpu().numpy())
    for rep in range(2):   # every k in one launch per degree; the second call replays the graph
        Yb = [x.clone() for x in Xs]
        ctx.filter_batched(Yb, deg, [a] * 8, b, [a0] * 8, flags)
        for k in range(8):
            assert colerr(Yb[k].cpu().numpy(), ref[k]) < TOL_BATCHED, (rep, k)
    # the low-precision degrees 1..5: one timed tensor-core product launch per degree for all eight
    # k-points (eight per degree if each k-point had its own)
    ctx.kernel_timing([P.C64])
    Yb = [x.clone() for x in Xs]
    ctx.filter_batched(Yb, deg, [a] * 8, b, [a0] * 8, flags)
    ms, nl = ctx.kernel_time()
    ctx.kernel_timing([])
    assert nl == deg - 1 and ms > 0
    for k in range(8):
        assert colerr(Yb[k].cpu().numpy(), ref[k]) < TOL_BATCHED, k


def test_band_trace_adjoint_at_scale(c4mid):
    from paper_2010_09701_gb300.autograd import band_trace
    w, ctx, V, xyz = c4mid
    nh, nO = ctx.ndof()
    n = nh + nO
    ik = 5
    X = torch.tensor(W.random_vectors(n, w.nv[ik], complex_=True, seed=77), dtype=torch.complex128, device="cuda")
    Vt = V.clone().requires_grad_(True)
    E = band_trace(Vt, X, ctx, ik)
    E.backward()
    g = Vt.grad.detach().clone()
    rng = np.random.default_rng(3)
    nq = V.numel()

    def energy(Vp):
        return float(band_trace(Vp, X, ctx, ik))

    # central differences along directions: E is affine in V, so only the rounding of the trace
    # (about 1e-15 of |E|) separates them from the adjoint. Along a non-negative direction on every
    # point at h = 1e-4 the change is far above that rounding; along one supported on 64 random
    # points the change is tiny at h = 1e-4, so there the step is h = 1 (the same derivative)
    h = 1e-4
    d = torch.tensor(rng.uniform(0.0, 1.0, nq), dtype=torch.float64, device="cuda")
    fd = (energy(V + h * d) - energy(V - h * d)) / (2 * h)
    ad = float(torch.dot(d, g))
    assert abs(fd - ad) <= 1e-6 * abs(ad)
    idx = torch.tensor(rng.choice(nq, 64, replace=False), device="cuda")
    d = torch.zeros_like(V)
    d[idx] = torch.tensor(rng.uniform(0.5, 1.0, 64), dtype=torch.float64, device="cuda")
    fd = (energy(V + d) - energy(V - d)) / 2.0
    ad = float(torch.dot(d, g))
    assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-14 * abs(float(E.detach()))

    # the oracle's fields on a 2^3 block of cells around a nucleus: w_q sum_v |u_v(x_q)|^2 there
    from scipy.spatial import cKDTree
    from oracle.enrichment import Enrichment
    from oracle.mesh import Mesh
    from oracle.operators import Problem
    from oracle.quadrature import Quadrature
    mesh = Mesh(w.a, W.mesh_breakpoints(w), w.p)
    cells = [ix + w.ncell * (iy + w.ncell * iz) for iz in range(2) for iy in range(2) for ix in range(2)]
    near = sorted({f for e in cells for f in mesh.neighbours(e)})
    nqc, nqe, depth = w.quad_params()
    quad = Quadrature(mesh, w.pos, w.rc, nqc, nqe, depth, cells=near)
    R, dR = W.radial_tables(w.Z, rc=w.rc, ngrid=w.ngrid)
    enr = Enrichment(w.a, w.pos, W.orbital_lm_codes(), R, dR, w.r0, w.rc)
    k, _ = W.monkhorst_pack(w.a, w.kgrid)
    pr = Problem(mesh, quad, enr, k[ik], cells=cells)
    Xb = X.cpu().numpy()[pr.rows]
    go = solver.band_trace_grad_V(pr, Xb)
    pts = np.concatenate([quad.points[quad.offset[e]:quad.offset[e + 1]] for e in cells])
    gob = np.concatenate([go[quad.offset[e]:quad.offset[e + 1]] for e in cells])
    tree = cKDTree(np.asarray(xyz))
    dist, j = tree.query(pts)
    assert np.max(dist) < 1e-9   # the same point sets on both sides
    gb = g.cpu().numpy()[j]
    assert np.max(np.abs(gb - gob)) <= 1e-12 * np.max(np.abs(gob))
