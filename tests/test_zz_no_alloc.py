"""oefe_apply_a_noalloc: M^{-1}H X for callers that cannot allocate device
memory (a pool that owns the device, a request path that must not take
cudaMalloc's implicit synchronization). Its scratch is one fixed device array
shared by every call; the result must equal oefe_apply_a's, call after call,
with native FP64 products and with the FP32-pair products (whose first call
times its launch shapes through that same array).
This file is collected last so that a failure here stops a -x run only after
every other test has run."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_cases import paired, rel, to_gpu

pytestmark = pytest.mark.gpu


def _case(k, pairs):
    from paper_2010_09701_gb300 import F64_PAIRS, STORE_F64, STORE_F64PAIR
    # a 4^3 mesh: the cells away from the two nuclei have one quadrature leaf, so the pair mode
    # really runs the sum-factorized FP32-pair products
    prs, ctx, V, Vd = paired(ks=[k], n=4, a=8.0, rc=2.5)
    if pairs:
        ctx.set_f64_products(F64_PAIRS)
        ctx.build_hamiltonian(Vd, STORE_F64 | STORE_F64PAIR)
    return prs[0], ctx


@pytest.mark.parametrize("pairs", [False, True], ids=["native", "pairs"])
@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)])
def test_apply_a_noalloc_matches_workspace_path(k, pairs):
    pr, ctx = _case(k, pairs)
    # against the oracle, relative to the largest entry: FP64 sums of a few hundred terms in another
    # order, amplified on the enrichment rows by the condition of M^oo (the row-scaled bounds of the
    # products are tested in test_gpu_filter.py); the pair products only to a loose bound here
    tol_oracle = 1e-10 if pairs else 1e-12
    for call, nv in enumerate((9, 4)):   # two calls in a row; the array keeps the first call's contents
        X = to_gpu(W.random_vectors(pr.n, nv, complex_=pr.complex, seed=20 + call))
        Y = torch.full_like(X, float("nan"))
        ctx.apply_a_noalloc(0, X, Y)   # first: in pair mode its first product times the launch shapes
        Yref = torch.empty_like(X)
        ctx.apply_a(0, X, Yref)
        assert rel(Y.cpu().numpy(), Yref.cpu().numpy()) < 1e-13
        assert rel(Y.cpu().numpy(), pr.apply_A(X.cpu().numpy())) < tol_oracle


def test_apply_a_noalloc_refuses_beyond_the_fixed_size():
    from paper_2010_09701_gb300 import OefeError, binding
    from paper_2010_09701_gb300.binding import NOALLOC_SCRATCH_BYTES
    prs, ctx, V, _ = paired(ks=[(0.25, -0.4, 0.1)])
    pr = prs[0]
    # the fixed array holds ncells * npad * nv complex128 products (plus the enrichment sums);
    # npad is the largest augmented cell size rounded up to 128
    ncells = len(pr.cells)
    npad = -(-max(len(ctx.cell_info(e)) for e in range(ncells)) // 128) * 128
    nv = NOALLOC_SCRATCH_BYTES // (ncells * npad * 16) + 8
    assert ncells * npad * nv * 16 > NOALLOC_SCRATCH_BYTES
    X = torch.zeros(pr.n, nv, dtype=torch.complex128, device="cuda")
    Y = torch.empty_like(X)
    with pytest.raises(OefeError) as e:
        ctx.apply_a_noalloc(0, X, Y)
    assert e.value.code == binding.ERR_ARG
    assert "limit" in str(e.value)
