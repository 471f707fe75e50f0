"""Parity of the tensor-core (tcgen05, BF16x3) cell products against the
oracle: single degrees (the bare product), full filters, complex and real,
one to four M tiles of 128 rows and ragged vector blocks."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_cases import c1_pair, paired, to_gpu
from oracle import solver

pytestmark = pytest.mark.gpu

KS = [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)]
# BF16x3: each cell product carries ~3 * 2^-17 relative error per term
TOL_DEGREE1 = 3e-5
TOL_FILTER = 2e-4


def colerr(out, ref):
    return np.max(np.linalg.norm(out - ref, axis=0) / np.linalg.norm(ref, axis=0))


def bounds(pr):
    import scipy.linalg as sla
    ev = sla.eigh(pr.assemble_H().toarray(), pr.dense_M(), eigvals_only=True)
    return ev[6], ev[-1] * 1.01, ev[0] - 1.0


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("nv", [5, 64, 70])
def test_tensor_single_degree(k, nv):
    from paper_2010_09701_gb300 import FILTER_BF16X3
    prs, ctx, V, _ = paired(ks=[k])
    pr = prs[0]
    a, b, a0 = bounds(pr)
    X = W.random_vectors(pr.n, nv, complex_=pr.complex, seed=nv)
    ref = solver.chebyshev_filter(pr.apply_A, X, 1, a, b, a0)
    Xd = to_gpu(X, torch.complex64 if pr.complex else torch.float32)
    ctx.chebyshev_filter(0, Xd, 1, a, b, a0, flags=FILTER_BF16X3)
    out = Xd.cpu().numpy().astype(ref.dtype)
    err = colerr(out, ref)
    assert err < TOL_DEGREE1
    assert err > 1e-9          # the split products did run (not an FP64 path)


@pytest.mark.parametrize("k", KS)
def test_tensor_filter_last_fp64(k):
    from paper_2010_09701_gb300 import FILTER_BF16X3, FILTER_LAST_FP64
    prs, ctx, V, _ = paired(ks=[k])
    pr = prs[0]
    a, b, a0 = bounds(pr)
    X = W.random_vectors(pr.n, 24, complex_=pr.complex, seed=2)
    ref = solver.chebyshev_filter(pr.apply_A, X, 9, a, b, a0)
    Xd = to_gpu(X)
    ctx.chebyshev_filter(0, Xd, 9, a, b, a0, flags=FILTER_LAST_FP64 | FILTER_BF16X3)
    assert colerr(Xd.cpu().numpy(), ref) < TOL_FILTER


def test_tensor_c1_two_m_tiles():
    # graded 8^3 mesh, p = 4: n_aug up to 135 -> two 128-row M tiles, four K tiles
    from paper_2010_09701_gb300 import FILTER_BF16X3
    w = W.config_c1()
    prs, ctx, V, _ = c1_pair()
    pr = prs[0]
    X = W.random_vectors(pr.n, 20, seed=w.seed)
    a, b, a0 = 0.0, 600.0, -99.0
    ref = solver.chebyshev_filter(pr.apply_A, X, 3, a, b, a0)
    Xd = to_gpu(X, torch.float32)
    ctx.chebyshev_filter(0, Xd, 3, a, b, a0, flags=FILTER_BF16X3)
    assert colerr(Xd.cpu().numpy().astype(np.float64), ref) < TOL_FILTER


def test_tensor_four_m_tiles():
    # p = 6 with enrichment: n_aug > 384 -> npad = 512 (four M tiles)
    from paper_2010_09701_gb300 import FILTER_BF16X3
    pos = np.random.default_rng(5).uniform(0.0, 7.0, (9, 3))
    prs, ctx, V, _ = paired(a=7.0, n=2, p=6, Zs=(3,) * 9, pos=pos, quad=(7, 7, 1), r0=2.0, rc=3.0,
                            ks=[(0.2, 0.1, -0.3)])
    pr = prs[0]
    assert max(ctx.cell_info(e).size for e in range(8)) > 384
    X = W.random_vectors(pr.n, 16, complex_=True, seed=3)
    ref = solver.chebyshev_filter(pr.apply_A, X, 1, 0.0, 500.0, -50.0)
    Xd = to_gpu(X, torch.complex64)
    ctx.chebyshev_filter(0, Xd, 1, 0.0, 500.0, -50.0, flags=FILTER_BF16X3)
    assert colerr(Xd.cpu().numpy().astype(np.complex128), ref) < TOL_DEGREE1


KS2 = [(0.3, 0.0, 0.0), (-0.3, 0.1, 0.0)]


@pytest.mark.parametrize("last_fp64", [False, True])
def test_batched_multik_filter(last_fp64):
    # all k-points in one persistent launch per degree, uneven vector counts, graph replay
    from paper_2010_09701_gb300 import FILTER_BF16X3, FILTER_LAST_FP64
    prs, ctx, V, _ = paired(ks=KS2)
    nvs = [20, 37]
    Xs = [W.random_vectors(pr.n, nv, complex_=True, seed=10 + i) for i, (pr, nv) in enumerate(zip(prs, nvs))]
    bnds = [bounds(pr) for pr in prs]
    deg = 7
    refs = [solver.chebyshev_filter(pr.apply_A, X, deg, *bd) for pr, X, bd in zip(prs, Xs, bnds)]
    dt = torch.complex128 if last_fp64 else torch.complex64
    flags = FILTER_BF16X3 | (FILTER_LAST_FP64 if last_fp64 else 0)
    for rep in range(2):   # the second call replays the captured graph
        Xd = [to_gpu(X, dt) for X in Xs]
        ctx.filter_batched(Xd, deg, [bd[0] for bd in bnds], [bd[1] for bd in bnds], [bd[2] for bd in bnds], flags)
        for k in range(2):
            out = Xd[k].cpu().numpy().astype(np.complex128)
            assert colerr(out, refs[k]) < TOL_FILTER, (rep, k)
        # the batched path computes the same products as the per-k path (the FP32 recurrence of the
        # two node updates may round differently by an ulp, which the filter amplifies)
        Xs1 = to_gpu(Xs[1], dt)
        ctx.chebyshev_filter(1, Xs1, deg, *bnds[1], flags=flags)
        assert colerr(Xd[1].cpu().numpy().astype(np.complex128), Xs1.cpu().numpy().astype(np.complex128)) < 2e-5


def test_autotune_then_batched_real():
    from paper_2010_09701_gb300 import FILTER_BF16X3
    prs, ctx, V, _ = paired()
    pr = prs[0]
    X = W.random_vectors(pr.n, 70, seed=4)
    ms = ctx.filter_autotune([to_gpu(X, torch.float32)])
    # real vectors: five candidates, the TMA kernel with 64 and with 128 vectors per tile included
    assert np.all(ms[:4] > 0) and ms[4] == 0 and ms[5] > 0
    a, b, a0 = bounds(pr)
    ref = solver.chebyshev_filter(pr.apply_A, X, 5, a, b, a0)
    Xd = to_gpu(X, torch.float32)
    ctx.filter_batched([Xd], 5, a, b, a0, FILTER_BF16X3)
    assert colerr(Xd.cpu().numpy().astype(np.float64), ref) < TOL_FILTER
    # with timing on, the captured graph carries one event pair per degree
    from paper_2010_09701_gb300 import F32, launch_count
    ctx.kernel_timing([F32])
    Xd = to_gpu(X, torch.float32)
    ctx.filter_batched([Xd], 5, a, b, a0, FILTER_BF16X3)
    ms, n = ctx.kernel_time()
    ctx.kernel_timing([])
    assert n == 5 and ms > 0
    assert colerr(Xd.cpu().numpy().astype(np.float64), ref) < TOL_FILTER
    # a replay of the captured graph counts each of its kernels: per degree the cell product,
    # the node update and the two enrichment kernels
    Xd = to_gpu(X, torch.float32)
    ctx.filter_batched([Xd], 5, a, b, a0, FILTER_BF16X3)   # capture (timing changed the graph key)
    Xd.copy_(to_gpu(X, torch.float32))                    # same buffer: the next call replays
    l0 = launch_count()
    ctx.filter_batched([Xd], 5, a, b, a0, FILTER_BF16X3)
    assert launch_count() - l0 >= 5 * 4
    assert colerr(Xd.cpu().numpy().astype(np.float64), ref) < TOL_FILTER


def test_upper_bound_tensor_products():
    from paper_2010_09701_gb300 import FILTER_BF16X3
    import scipy.linalg as sla
    prs, ctx, V, _ = paired(ks=[(0.25, -0.4, 0.1)])
    pr = prs[0]
    ev = sla.eigh(pr.assemble_H().toarray(), pr.dense_M(), eigvals_only=True)
    v0 = to_gpu(W.random_vectors(pr.n, 1, complex_=True, seed=3))
    b64 = ctx.upper_bound(0, v0, 30)
    b16 = ctx.upper_bound(0, v0, 30, FILTER_BF16X3)
    # theta_max + beta_last is a valid but loose bound; the low-precision run keeps it valid
    assert ev[-1] * (1 - 1e-4) <= b16 < 1.5 * ev[-1]
    assert ev[-1] * (1 - 1e-8) <= b64 < 1.5 * ev[-1]


@pytest.mark.parametrize("nv", [1, 8])
@pytest.mark.parametrize("deg", [1, 6])
def test_batched_small_vector_blocks(nv, deg):
    # fewer vectors than a warp's lanes: the batched node update must not rely on idle lanes; a
    # single mixed degree is one FP64 degree
    from paper_2010_09701_gb300 import FILTER_BF16X3, FILTER_LAST_FP64
    prs, ctx, V, _ = paired(ks=[KS[1]])
    pr = prs[0]
    a, b, a0 = bounds(pr)
    X = W.random_vectors(pr.n, nv, complex_=True, seed=30 + nv)
    ref = solver.chebyshev_filter(pr.apply_A, X, deg, a, b, a0)
    Xd = to_gpu(X)
    ctx.filter_batched([Xd], deg, a, b, a0, FILTER_BF16X3 | FILTER_LAST_FP64)
    assert colerr(Xd.cpu().numpy(), ref) < (1e-12 if deg == 1 else TOL_FILTER)
    X32 = to_gpu(X, torch.complex64)
    ctx.filter_batched([X32], deg, a, b, a0, FILTER_BF16X3)
    assert colerr(X32.cpu().numpy().astype(np.complex128), ref) < TOL_FILTER


def test_release_workspace_then_filter_again():
    # freeing the cached scratch drops the captured graph too; the next calls rebuild both
    from paper_2010_09701_gb300 import FILTER_BF16X3, FILTER_LAST_FP64
    prs, ctx, V, _ = paired(ks=[KS[1]])
    pr = prs[0]
    a, b, a0 = bounds(pr)
    X = W.random_vectors(pr.n, 12, complex_=True, seed=44)
    ref = solver.chebyshev_filter(pr.apply_A, X, 5, a, b, a0)
    for rep in range(2):
        Xd = to_gpu(X)
        ctx.filter_batched([Xd], 5, a, b, a0, FILTER_BF16X3 | FILTER_LAST_FP64)
        assert colerr(Xd.cpu().numpy(), ref) < TOL_FILTER, rep
        ctx.release_workspace()
    Xd = to_gpu(X)
    Y = torch.empty_like(Xd)
    ctx.apply_h(0, Xd, Y)
    assert np.max(np.abs(Y.cpu().numpy() - pr.apply_H(X))) < 1e-12 * np.max(np.abs(pr.apply_H(X)))


# BF16x6: three bf16 parts per operand, six products: FP32-class (the vectors are FP32)
TOL6_DEGREE1 = 5e-6
TOL6_FILTER = 5e-5


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("nv", [5, 64, 70])
def test_bf16x6_single_degree(k, nv):
    from paper_2010_09701_gb300 import FILTER_BF16X3, STORE_BF16X6, STORE_F64
    prs, ctx, V, _ = paired(ks=[k], store=STORE_F64 | STORE_BF16X6)
    pr = prs[0]
    X = W.random_vectors(pr.n, nv, complex_=pr.complex, seed=nv + 60)
    ref = solver.chebyshev_filter(pr.apply_A, X, 1, 0.0, 500.0, -50.0)
    Xd = to_gpu(X, torch.complex64 if pr.complex else torch.float32)
    ctx.chebyshev_filter(0, Xd, 1, 0.0, 500.0, -50.0, flags=FILTER_BF16X3)
    out = Xd.cpu().numpy().astype(np.complex128 if pr.complex else np.float64)
    assert colerr(out, ref) < TOL6_DEGREE1


def test_bf16x6_batched_two_k():
    # the batched launch over two k-points with uneven vector counts
    from paper_2010_09701_gb300 import FILTER_BF16X3, FILTER_LAST_FP64, STORE_BF16X6, STORE_F64
    prs, ctx, V, _ = paired(ks=KS2, store=STORE_F64 | STORE_BF16X6)
    nvs = [20, 37]
    Xs = [W.random_vectors(pr.n, nv, complex_=True, seed=70 + i) for i, (pr, nv) in enumerate(zip(prs, nvs))]
    bnds = [bounds(pr) for pr in prs]
    refs = [solver.chebyshev_filter(pr.apply_A, X, 7, *bd) for pr, X, bd in zip(prs, Xs, bnds)]
    Xd = [to_gpu(X) for X in Xs]
    ctx.filter_batched(Xd, 7, [bd[0] for bd in bnds], [bd[1] for bd in bnds], [bd[2] for bd in bnds],
                       FILTER_BF16X3 | FILTER_LAST_FP64)
    for k in range(2):
        assert colerr(Xd[k].cpu().numpy(), refs[k]) < TOL6_FILTER, k
    ms = ctx.filter_autotune([to_gpu(X, torch.complex64) for X in Xs])
    # only the TMA kernel takes three parts; 128-vector tiles are for real data
    assert ms[3] > 0 and ms[4] > 0 and np.all(ms[:3] == 0) and ms[5] == 0


def test_bf16x6_four_m_tiles():
    from paper_2010_09701_gb300 import FILTER_BF16X3, STORE_BF16X6, STORE_F64
    pos = np.random.default_rng(5).uniform(0.0, 7.0, (9, 3))
    prs, ctx, V, _ = paired(a=7.0, n=2, p=6, Zs=(3,) * 9, pos=pos, quad=(7, 7, 1), r0=2.0, rc=3.0,
                            ks=[(0.2, 0.1, -0.3)], store=STORE_F64 | STORE_BF16X6)
    pr = prs[0]
    assert max(ctx.cell_info(e).size for e in range(8)) > 384
    X = W.random_vectors(pr.n, 16, complex_=True, seed=3)
    ref = solver.chebyshev_filter(pr.apply_A, X, 1, 0.0, 500.0, -50.0)
    Xd = to_gpu(X, torch.complex64)
    ctx.chebyshev_filter(0, Xd, 1, 0.0, 500.0, -50.0, flags=FILTER_BF16X3)
    assert colerr(Xd.cpu().numpy().astype(np.complex128), ref) < TOL6_DEGREE1


@pytest.mark.parametrize("store", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("nv", [70, 128, 200])
def test_real_128_vector_tiles(store, nv):
    # real data with 128 vectors per TMA tile (each cell matrix streams once per 128 vectors):
    # ragged last block, both splits; same products as 64-vector tiles up to FP32 summation order
    from paper_2010_09701_gb300 import FILTER_BF16X3, FILTER_LAST_FP64, STORE_BF16X3, STORE_BF16X6, STORE_F64
    prs, ctx, V, _ = paired(ks=[(0.0, 0.0, 0.0)],
                            store=STORE_F64 | (STORE_BF16X6 if store == "bf16x6" else STORE_BF16X3))
    pr = prs[0]
    a, b, a0 = bounds(pr)
    X = W.random_vectors(pr.n, nv, seed=nv + 1)
    ref = solver.chebyshev_filter(pr.apply_A, X, 6, a, b, a0)
    outs = {}
    for shape in (3, 5):
        ctx.set_filter_shape(shape)
        Xd = to_gpu(X)
        ctx.filter_batched([Xd], 6, [a], [b], [a0], FILTER_BF16X3 | FILTER_LAST_FP64)
        outs[shape] = Xd.cpu().numpy()
        assert colerr(outs[shape], ref) < (TOL6_FILTER if store == "bf16x6" else TOL_FILTER), shape
    ctx.set_filter_shape(-1)
    assert colerr(outs[5], outs[3]) < (1e-6 if store == "bf16x6" else 2e-5)


def test_real_128_vector_tiles_four_m_tiles():
    # n_aug > 384 (four M tiles, 512 accumulator columns of TMEM) with 128-vector tiles
    from paper_2010_09701_gb300 import FILTER_BF16X3
    pos = np.random.default_rng(5).uniform(0.0, 7.0, (9, 3))
    prs, ctx, V, _ = paired(a=7.0, n=2, p=6, Zs=(3,) * 9, pos=pos, quad=(7, 7, 1), r0=2.0, rc=3.0,
                            ks=[(0.0, 0.0, 0.0)])
    pr = prs[0]
    assert not pr.complex and max(ctx.cell_info(e).size for e in range(8)) > 384
    X = W.random_vectors(pr.n, 150, seed=9)
    ref = solver.chebyshev_filter(pr.apply_A, X, 1, 0.0, 500.0, -50.0)
    ctx.set_filter_shape(5)
    Xd = to_gpu(X, torch.float32)
    ctx.filter_batched([Xd], 1, [0.0], [500.0], [-50.0], FILTER_BF16X3)
    ctx.set_filter_shape(-1)
    assert colerr(Xd.cpu().numpy().astype(np.float64), ref) < TOL_DEGREE1


def test_filter_shape_argument_checked():
    from paper_2010_09701_gb300 import OefeError
    prs, ctx, V, _ = paired(ks=[(0.0, 0.0, 0.0)])
    for bad in (-2, 6):
        with pytest.raises(OefeError):
            ctx.set_filter_shape(bad)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("nv", [96, 120, 128])
def test_mixed_filter_wide_blocks(cplx, nv):
    # more than 64 vectors in one column group: the last (FP64) degree runs in column chunks that
    # fit the product buffer; vector counts above half the basis size included
    from paper_2010_09701_gb300 import FILTER_BF16X3, FILTER_LAST_FP64
    prs, ctx, V, _ = paired(ks=[KS[1] if cplx else KS[0]])
    pr = prs[0]
    assert 2 * nv > pr.n or nv == 96
    a, b, a0 = bounds(pr)
    X = W.random_vectors(pr.n, nv, complex_=cplx, seed=40 + nv)
    ref = solver.chebyshev_filter(pr.apply_A, X, 6, a, b, a0)
    Xd = to_gpu(X)
    ctx.filter_batched([Xd], 6, a, b, a0, FILTER_BF16X3 | FILTER_LAST_FP64)
    assert colerr(Xd.cpu().numpy(), ref) < TOL_FILTER
