"""Set up a library Context for a synthetic workload (mesh, enrichment,
quadrature, k-points) from the seeded inputs of ``workloads``."""
import numpy as np

import workloads as W

from .binding import Context


def setup_workload(w, device=0, stream=None, quad=None, kpoints=None):
    """Context with mesh, enrichment, quadrature and k-points of workload ``w``."""
    ctx = Context(device, stream)
    xb = W.mesh_breakpoints(w)
    ctx.mesh(w.a, xb, w.p)
    R, dR = W.radial_tables(w.Z, rc=w.rc, ngrid=w.ngrid)
    ctx.enrichment(w.pos, W.orbital_lm_codes(), R, dR, w.r0, w.rc)
    ctx.quadrature(*(quad or w.quad_params()))
    if kpoints is None:
        k, wk = W.monkhorst_pack(w.a, w.kgrid)
    else:
        k, wk = kpoints
    ctx.kpoints(k, wk)
    return ctx
