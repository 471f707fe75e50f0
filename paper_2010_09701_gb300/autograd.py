"""Adjoint of the cell-level H.X application as torch.autograd Functions.

H^O(V) is affine in the quadrature-point potential V through the
(|k|^2/2 + V) N_m^* N_n term of Eq. HOEFEelelements, so for the band trace
E = tr(X^+ H^O(V) X):
    dE/dV_q = w_q sum_v |u_v(x_q)|^2   (u the field of column v, Eq. UOEFE),
    dE/dX   = 2 H^O X                  (torch's convention for real and complex X).
Both are evaluated by the CUDA library; the backward pass recomputes the cell
gathers and the field interpolation instead of storing them.
"""
import torch


def _ensure_built(ctx, V):
    if ctx.built_from != (V.data_ptr(), V._version):
        ctx.build_hamiltonian(V.detach())


class BandTrace(torch.autograd.Function):
    """E = tr(X^+ H^O(V) X) for one k-point (FP64 path)."""

    @staticmethod
    def forward(fctx, V, X, octx, ik):
        _ensure_built(octx, V)
        HX = torch.empty_like(X)
        octx.apply_h(ik, X.detach(), HX)
        E = torch.sum(X.detach().conj() * HX).real
        fctx.save_for_backward(V, X)
        fctx.octx, fctx.ik = octx, ik
        return E

    @staticmethod
    def backward(fctx, g):
        V, X = fctx.saved_tensors
        octx, ik = fctx.octx, fctx.ik
        _ensure_built(octx, V)
        gV = gX = None
        if fctx.needs_input_grad[0]:
            gV = torch.empty_like(V)
            octx.band_trace_grad(ik, X.detach(), gV)
            gV = gV * g
        if fctx.needs_input_grad[1]:
            HX = torch.empty_like(X)
            octx.apply_h(ik, X.detach(), HX)
            gX = 2.0 * g * HX
        return gV, gX, None, None


class ApplyH(torch.autograd.Function):
    """Y = H^O(V) X. Vector-Jacobian products: grad_X = H^O G (H^O Hermitian);
    grad_V_q = w_q Re sum_v conj(u_G,v) u_X,v, obtained from the band-trace
    gradient by polarization: (f(X + G) - f(X - G)) / 4 with f(Z) = w_q sum |u_Z|^2."""

    @staticmethod
    def forward(fctx, V, X, octx, ik):
        _ensure_built(octx, V)
        Y = torch.empty_like(X)
        octx.apply_h(ik, X.detach(), Y)
        fctx.save_for_backward(V, X)
        fctx.octx, fctx.ik = octx, ik
        return Y

    @staticmethod
    def backward(fctx, G):
        V, X = fctx.saved_tensors
        octx, ik = fctx.octx, fctx.ik
        _ensure_built(octx, V)
        G = G.contiguous()
        gV = gX = None
        if fctx.needs_input_grad[0]:
            fp = torch.empty_like(V)
            fm = torch.empty_like(V)
            octx.band_trace_grad(ik, (X.detach() + G).contiguous(), fp)
            octx.band_trace_grad(ik, (X.detach() - G).contiguous(), fm)
            gV = 0.25 * (fp - fm)
        if fctx.needs_input_grad[1]:
            gX = torch.empty_like(X)
            octx.apply_h(ik, G, gX)
        return gV, gX, None, None


def band_trace(V, X, octx, ik=0):
    return BandTrace.apply(V, X, octx, ik)


def apply_h(V, X, octx, ik=0):
    return ApplyH.apply(V, X, octx, ik)
