"""GPU parity of the operator construction against the oracle: quadrature
points, lumped mass, M^oo, and the cell matrices H^O_e (Eq. HOEFEelelements,
T-transform of Eq. UOEFESplit)."""
import numpy as np
import pytest

import workloads as W
from gpu_cases import c1_pair, paired, rel

pytestmark = pytest.mark.gpu

KS = [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)]


def test_graded_mesh_matches_inputs():
    from paper_2010_09701_gb300 import Context
    ctx = Context(0)
    for name in ("c1", "c2", "c4", "c5"):
        w = W.CONFIGS[name]()
        xb = ctx.mesh_graded(w.a, w.ncell, w.p, w.pos, w.grading_ratio)
        assert np.allclose(xb, W.mesh_breakpoints(w), rtol=0, atol=1e-12 * w.a), name


@pytest.mark.parametrize("k", KS)
def test_quadrature_mass_and_moo(k):
    prs, ctx, V, _ = paired(ks=[k])
    pr = prs[0]
    xyz, w = ctx.quadrature_points()
    assert xyz.shape == pr.quad.points.shape
    assert np.max(np.abs(xyz - pr.quad.points)) <= 1e-14 * pr.mesh.a
    assert np.max(np.abs(w - pr.quad.weights)) <= 1e-14 * np.max(pr.quad.weights)
    m, Moo = ctx.overlap(0, complex_=pr.complex)
    assert rel(m, pr.m) < 1e-14
    assert rel(Moo, pr.Moo) < 1e-12


@pytest.mark.parametrize("k", KS)
def test_cell_matrices(k):
    prs, ctx, V, _ = paired(ks=[k])
    pr = prs[0]
    for e in range(pr.mesh.ncells):
        idx = ctx.cell_info(e)
        assert np.array_equal(idx, pr.index(e))
        H = ctx.cell_matrix(0, e, complex_=pr.complex)
        assert rel(H, pr.HO[e]) < 1e-12, e


@pytest.mark.parametrize("k", KS)
def test_cell_matrices_fp32_pair_build(k):
    # the per-step build in FP32-pair arithmetic (u = 2^-48, 2^5 times the FP64 unit): the FP64
    # tolerance scales by 32
    from paper_2010_09701_gb300 import F64_NATIVE, F64_PAIRS, STORE_F64, STORE_F64PAIR
    prs, ctx, V, Vd = paired(ks=[k])
    pr = prs[0]
    ctx.set_f64_products(F64_PAIRS)
    ctx.build_hamiltonian(Vd, STORE_F64 | STORE_F64PAIR)
    for e in range(pr.mesh.ncells):
        assert rel(ctx.cell_matrix(0, e, complex_=pr.complex), pr.HO[e]) < 32e-12, e
    ctx.set_f64_products(F64_NATIVE)


def test_c1_pair_build_nucleus_cells():
    # the refined cells (many leaves, partial sums) of the first configuration, pair arithmetic
    from paper_2010_09701_gb300 import F64_NATIVE, F64_PAIRS, STORE_F64, STORE_F64PAIR
    prs, ctx, V, Vd = c1_pair()
    pr = prs[0]
    ctx.set_f64_products(F64_PAIRS)
    ctx.build_hamiltonian(Vd, STORE_F64 | STORE_F64PAIR)
    cells = [e for e in range(pr.mesh.ncells) if pr.quad.cls[e] == 2][:4] + [5, 100, 511]
    for e in cells:
        assert rel(ctx.cell_matrix(0, e), pr.HO[e]) < 32e-12, e
    ctx.set_f64_products(F64_NATIVE)


def test_c1_cell_matrices_nucleus_cells():
    prs, ctx, V, _ = c1_pair()
    pr = prs[0]
    cells = [e for e in range(pr.mesh.ncells) if pr.quad.cls[e] == 2][:4] + [5, 100, 511]
    for e in cells:
        H = ctx.cell_matrix(0, e)
        assert rel(H, pr.HO[e]) < 1e-12, e
    m, Moo = ctx.overlap(0)
    assert rel(Moo, pr.Moo) < 1e-12


def test_single_cell_and_no_enrichment():
    # n_c = 1: a cell's nodes repeat through the periodic wrap
    prs, ctx, V, _ = paired(a=5.0, n=1, p=4, Zs=(3,), pos=[[1.0, 1.5, 2.0]], quad=(5, 6, 2), r0=1.2, rc=2.0)
    H = ctx.cell_matrix(0, 0)
    assert rel(H, prs[0].HO[0]) < 1e-12
    prs, ctx, V, _ = paired(a=5.0, n=2, p=2, Zs=(), enrich=False, quad=(3, 3, 0), r0=1.2, rc=2.0)
    for e in range(8):
        assert rel(ctx.cell_matrix(0, e), prs[0].HO[e]) < 1e-12
