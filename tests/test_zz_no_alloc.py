"""oefe_apply_a_noalloc: M^{-1}H X for callers that cannot allocate device
memory (a pool that owns the device, a request path that must not take
cudaMalloc's implicit synchronization). Its scratch is one fixed device array
shared by every call; the result must equal oefe_apply_a's, call after call.
This file is collected last so that a failure here stops a -x run only after
every other test has run."""
import numpy as np
import pytest
import torch

import workloads as W
from gpu_cases import paired, rel, to_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k", [(0.0, 0.0, 0.0), (0.25, -0.4, 0.1)])
def test_apply_a_noalloc_matches_workspace_path(k):
    prs, ctx, V, _ = paired(ks=[k])
    pr = prs[0]
    for call, nv in enumerate((9, 4)):   # two calls in a row; the array keeps the first call's contents
        X = to_gpu(W.random_vectors(pr.n, nv, complex_=pr.complex, seed=20 + call))
        Yref = torch.empty_like(X)
        ctx.apply_a(0, X, Yref)
        Y = torch.full_like(X, float("nan"))
        ctx.apply_a_noalloc(0, X, Y)
        assert rel(Y.cpu().numpy(), Yref.cpu().numpy()) < 1e-13
        assert rel(Y.cpu().numpy(), pr.apply_A(X.cpu().numpy())) < 1e-13


def test_apply_a_noalloc_refuses_beyond_the_fixed_size():
    from paper_2010_09701_gb300 import OefeError, binding
    prs, ctx, V, _ = paired(ks=[(0.25, -0.4, 0.1)])
    pr = prs[0]
    # ncells * npad * nv * 16 bytes > 64 MiB: 8 cells x 128 rows -> nv = 4200
    X = torch.zeros(pr.n, 4200, dtype=torch.complex128, device="cuda")
    Y = torch.empty_like(X)
    with pytest.raises(OefeError) as e:
        ctx.apply_a_noalloc(0, X, Y)
    assert e.value.code == binding.ERR_ARG
    assert "limit" in str(e.value)
