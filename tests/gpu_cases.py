"""Paired oracle / library problems for the GPU parity tests (same seeded inputs)."""
import numpy as np

import workloads as W
from cases import oracle_problem, uniform_xb


def lib_context(a, xb, p, pos, Z, ks, quad, r0, rc, enrich=True, ngrid=2000, orbitals=W.ORBITALS_1S_2P):
    from paper_2010_09701_gb300 import Context
    ctx = Context(0)
    ctx.mesh(a, xb, p)
    pos = np.asarray(pos, float).reshape(-1, 3)
    if enrich and len(Z):
        R, dR = W.radial_tables(np.asarray(Z), orbitals, rc=rc, ngrid=ngrid)
        ctx.enrichment(pos, W.orbital_lm_codes(orbitals), R, dR, r0, rc)
    else:
        ctx.enrichment(np.zeros((0, 3)), np.zeros(0, np.int32), np.zeros(0), np.zeros(0), r0, rc)
    ctx.quadrature(*quad)
    ks = np.asarray(ks, float).reshape(-1, 3)
    ctx.kpoints(ks, np.full(len(ks), 1.0 / len(ks)))
    return ctx


def paired(a=6.0, n=2, p=3, Zs=(3, 4), ks=((0.0, 0.0, 0.0),), quad=(4, 5, 2), r0=1.5, rc=2.5, sigma=0.3,
           xb=None, pos=None, enrich=True, store=None):
    """Oracle problems (one per k) and a library context built from the same inputs and V."""
    import torch
    from paper_2010_09701_gb300 import STORE_BF16X3, STORE_F32, STORE_F64
    if pos is None:
        pos = np.array([[0.0, 0.0, 0.0], [a / 2, a / 2, a / 2]])[:len(Zs)]
    pos = np.asarray(pos, float)
    Z = np.array(Zs)
    xb = uniform_xb(a, n) if xb is None else xb
    prs = [oracle_problem(a, xb, p, pos, Z, k=k, quad=quad, r0=r0, rc=rc, enrich=enrich) for k in ks]
    V = W.veff(prs[0].quad.points, a, pos, Z, sigma=sigma) if len(Z) else np.zeros(prs[0].quad.nq)
    for pr in prs:
        pr.build(V)
    ctx = lib_context(a, xb, p, pos, Z, ks, quad, r0, rc, enrich=enrich)
    Vd = torch.tensor(V, dtype=torch.float64, device="cuda")
    ctx.build_hamiltonian(Vd, store if store is not None else (STORE_F64 | STORE_F32 | STORE_BF16X3))
    return prs, ctx, V, Vd


def c1_pair(store=None):
    w = W.config_c1()
    xb = W.mesh_breakpoints(w)
    return paired(a=w.a, p=w.p, Zs=tuple(w.Z), pos=w.pos, xb=xb, quad=w.quad_params(), r0=w.r0, rc=w.rc,
                  sigma=w.sigma, store=store)


def to_gpu(X, dtype=None):
    import torch
    t = torch.tensor(X, device="cuda")
    return t.to(dtype) if dtype is not None else t


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)
