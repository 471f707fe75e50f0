"""Thin ctypes binding of liboefe (include/oefe.h): argument marshalling only.

Every computation runs in the CUDA library; this module only passes pointers,
sizes and the current torch CUDA stream. It raises if the library is missing.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboefe.so")

OK, ERR_ARG, ERR_STATE, ERR_OOM, ERR_CUDA, ERR_CHOLESKY, ERR_NOTPD_MOO, ERR_TIMEOUT, ERR_NUMERIC = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
F64, F32, C128, C64 = 0, 1, 2, 3
STORE_F64, STORE_F32, STORE_BF16X3, STORE_BF16X6, STORE_F64PAIR, STORE_COMPACT = 1, 2, 4, 8, 16, 32
F64_NATIVE, F64_PAIRS = 0, 1
FILTER_LAST_FP64, FILTER_BF16X3 = 1, 2
NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024

# every symbol of include/oefe.h: (name, restype, argtypes)
_c = ctypes
_P = _c.c_void_p
_I = _c.c_int
_D = _c.c_double
_DP = _c.POINTER(_c.c_double)
_IP = _c.POINTER(_c.c_int)
_I64P = _c.POINTER(_c.c_int64)
SIGNATURES = [
    ("oefe_create", _I, [_c.POINTER(_P), _I, _P]),
    ("oefe_destroy", _I, [_P]),
    ("oefe_set_stream", _I, [_P, _P]),
    ("oefe_last_error", _I, [_P, _c.c_char_p, _c.c_size_t]),
    ("oefe_mesh", _I, [_P, _D, _IP, _DP, _I]),
    ("oefe_mesh_graded", _I, [_P, _D, _I, _I, _I, _DP, _D, _DP]),
    ("oefe_enrichment", _I, [_P, _I, _DP, _I, _IP, _I, _DP, _DP, _D, _D]),
    ("oefe_quadrature", _I, [_P, _I, _I, _I]),
    ("oefe_quadrature_count", _I, [_P, _I64P]),
    ("oefe_quadrature_points", _I, [_P, _DP, _DP]),
    ("oefe_kpoints", _I, [_P, _I, _DP, _DP]),
    ("oefe_ndof", _I, [_P, _I64P, _IP]),
    ("oefe_build_hamiltonian", _I, [_P, _P, _I]),
    ("oefe_cell_info", _I, [_P, _I, _IP, _IP]),
    ("oefe_cell_matrix", _I, [_P, _I, _I, _P]),
    ("oefe_overlap", _I, [_P, _I, _DP, _P]),
    ("oefe_apply_h", _I, [_P, _I, _P, _P, _I, _I, _I]),
    ("oefe_apply_a", _I, [_P, _I, _P, _P, _I, _I, _I]),
    ("oefe_apply_a_noalloc", _I, [_P, _I, _P, _P, _I, _I, _I]),
    ("oefe_chebyshev_filter", _I, [_P, _I, _P, _I, _I, _I, _I, _D, _D, _D, _I]),
    ("oefe_filter_batched", _I, [_P, _I, _c.POINTER(_P), _IP, _IP, _I, _I, _DP, _DP, _DP, _I]),
    ("oefe_filter_batched_defect", _I, [_P, _I, _c.POINTER(_P), _IP, _IP, _I, _I, _DP, _DP, _DP, _DP, _I]),
    ("oefe_filter_autotune", _I, [_P, _I, _c.POINTER(_P), _IP, _IP, _I, _DP]),
    ("oefe_orthonormalize", _I, [_P, _I, _P, _I, _I, _I, _DP]),
    ("oefe_rayleigh_ritz", _I, [_P, _I, _P, _I, _I, _I, _DP, _DP]),
    ("oefe_density", _I, [_P, _I, _c.POINTER(_P), _IP, _IP, _I, _DP, _P]),
    ("oefe_band_trace_grad", _I, [_P, _I, _P, _I, _I, _I, _P]),
    ("oefe_density_grad", _I, [_P, _I, _c.POINTER(_P), _IP, _IP, _I, _DP, _P, _I, _P]),
    ("oefe_band_trace", _I, [_P, _I, _P, _I, _I, _I, _DP, _P]),
    ("oefe_band_trace_vjp", _I, [_P, _I, _P, _I, _I, _I, _D, _P, _P]),
    ("oefe_apply_h_vjp", _I, [_P, _I, _P, _P, _P, _P, _I, _I, _I]),
    ("oefe_upper_bound", _I, [_P, _I, _P, _I, _I, _DP]),
    ("oefe_occupations", _I, [_I, _IP, _DP, _DP, _D, _D, _DP, _DP, _DP]),
    ("oefe_kernel_timing", _I, [_P, _I]),
    ("oefe_kernel_time", _I, [_P, _DP, _I64P]),
    ("oefe_release_workspace", _I, [_P]),
    ("oefe_product_flops", _I, [_P, _I, _I, _DP]),
    ("oefe_launch_count", _I, [_c.POINTER(_c.c_int64)]),
    ("oefe_set_f64_products", _I, [_P, _I]),
    ("oefe_set_product_shape", _I, [_P, _I]),
    ("oefe_set_filter_shape", _I, [_P, _I]),
]

_lib = None


def load():
    """Load liboefe.so (built by build_ext.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liboefe.so is not built: run __graft_entry__.build() or "
                               "python paper_2010_09701_gb300/build_ext.py")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def launch_count():
    """Kernel launches the library has issued in this process (graph replays count each kernel)."""
    n = ctypes.c_int64()
    if load().oefe_launch_count(ctypes.byref(n)) != 0:
        raise RuntimeError("oefe_launch_count failed")
    return int(n.value)


class OefeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("oefe error %d: %s" % (code, msg))
        self.code = code


def _dp(a):
    return a.ctypes.data_as(_DP)


def _ip(a):
    return a.ctypes.data_as(_IP)


def _dtype_code(t):
    import torch
    m = {torch.float64: F64, torch.float32: F32, torch.complex128: C128, torch.complex64: C64}
    if t.dtype not in m:
        raise TypeError("unsupported dtype %s" % t.dtype)
    return m[t.dtype]


def _block(X):
    """(pointer, nv, ld, dtype code) of a CUDA matrix with unit column stride."""
    if not X.is_cuda:
        raise ValueError("vector blocks must live on the GPU")
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("need a 2-D tensor with contiguous rows")
    return ctypes.c_void_p(X.data_ptr()), X.shape[1], X.stride(0), _dtype_code(X)


def occupations(eigs, w, n_electrons, temperature=500.0):
    """Fermi level, density weights 2 w_k f and band energy (oefe_occupations)."""
    lib = load()
    nv = np.array([len(e) for e in eigs], np.int32)
    eig = np.ascontiguousarray(np.concatenate([np.asarray(e, np.float64) for e in eigs]))
    w = np.ascontiguousarray(w, np.float64)
    occ = np.zeros(len(eig))
    mu = ctypes.c_double()
    eb = ctypes.c_double()
    code = lib.oefe_occupations(len(nv), _ip(nv), _dp(eig), _dp(w), float(n_electrons), float(temperature),
                                _dp(occ), ctypes.byref(mu), ctypes.byref(eb))
    if code != OK:
        raise OefeError(code, "occupations: bad arguments")
    out, o = [], 0
    for n in nv:
        out.append(occ[o:o + n])
        o += n
    return mu.value, out, eb.value


class Context:
    """One OEFE problem on one GPU; method names follow the C ABI (oefe_<name>)."""

    def __init__(self, device=0, stream=None):
        import torch
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.h = ctypes.c_void_p()
        self._check(self.lib.oefe_create(ctypes.byref(self.h), device, ctypes.c_void_p(stream)))
        self.nk = 0
        self._built_v, self._built_version, self.built_store = None, -1, STORE_F64

    def _check(self, code):
        if code != OK:
            buf = ctypes.create_string_buffer(512)
            if self.h:
                self.lib.oefe_last_error(self.h, buf, 512)
            raise OefeError(code, buf.value.decode())

    def close(self):
        if self.h:
            self.lib.oefe_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._check(self.lib.oefe_set_stream(self.h, ctypes.c_void_p(stream)))

    # -- geometry ---------------------------------------------------------------
    def mesh(self, a, xb, p):
        xb = [np.ascontiguousarray(b, np.float64) for b in xb]
        nc = np.array([len(b) - 1 for b in xb], np.int32)
        flat = np.ascontiguousarray(np.concatenate(xb))
        self._check(self.lib.oefe_mesh(self.h, float(a), _ip(nc), _dp(flat), int(p)))

    def mesh_graded(self, a, ncell, p, pos, ratio=1.5):
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        out = np.zeros(3 * (ncell + 1))
        self._check(self.lib.oefe_mesh_graded(self.h, float(a), int(ncell), int(p), len(pos), _dp(pos),
                                              float(ratio), _dp(out)))
        return out.reshape(3, ncell + 1)

    def enrichment(self, pos, lm, R, dR, r0, rc):
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        lm = np.ascontiguousarray(lm, np.int32)
        R = np.ascontiguousarray(R, np.float64)
        dR = np.ascontiguousarray(dR, np.float64)
        ngrid = R.shape[-1] if R.size else 4
        self._check(self.lib.oefe_enrichment(self.h, len(pos), _dp(pos), len(lm), _ip(lm), int(ngrid), _dp(R),
                                             _dp(dR), float(r0), float(rc)))

    def quadrature(self, nq_cell, nq_enr, depth):
        self._check(self.lib.oefe_quadrature(self.h, int(nq_cell), int(nq_enr), int(depth)))

    def quadrature_count(self):
        n = ctypes.c_int64()
        self._check(self.lib.oefe_quadrature_count(self.h, ctypes.byref(n)))
        return n.value

    def quadrature_points(self):
        n = self.quadrature_count()
        xyz = np.zeros((n, 3))
        w = np.zeros(n)
        self._check(self.lib.oefe_quadrature_points(self.h, _dp(xyz), _dp(w)))
        return xyz, w

    def kpoints(self, k, w):
        k = np.ascontiguousarray(k, np.float64).reshape(-1, 3)
        w = np.ascontiguousarray(w, np.float64)
        self._check(self.lib.oefe_kpoints(self.h, len(k), _dp(k), _dp(w)))
        self.nk = len(k)
        self.k = k.copy()

    def ndof(self):
        nh = ctypes.c_int64()
        nO = ctypes.c_int()
        self._check(self.lib.oefe_ndof(self.h, ctypes.byref(nh), ctypes.byref(nO)))
        return nh.value, nO.value

    # -- operators --------------------------------------------------------------
    def build_hamiltonian(self, veff, store=STORE_F64):
        import torch
        if not (veff.is_cuda and veff.dtype == torch.float64 and veff.is_contiguous()):
            raise ValueError("veff must be a contiguous float64 CUDA tensor")
        self._check(self.lib.oefe_build_hamiltonian(self.h, ctypes.c_void_p(veff.data_ptr()), int(store)))
        # the potential of the build is held (so no other tensor can take its memory and pass for it)
        # with its version counter, which changes on any in-place write
        self._built_v, self._built_version, self.built_store = veff, veff._version, int(store)

    def built_from(self, veff):
        """True when the stored operator was built from this potential's current values."""
        b = self._built_v
        return (b is not None and b.data_ptr() == veff.data_ptr() and b.shape == veff.shape and
                self._built_version == veff._version)

    def cell_info(self, cell):
        n = ctypes.c_int()
        self._check(self.lib.oefe_cell_info(self.h, int(cell), ctypes.byref(n), None))
        idx = np.zeros(n.value, np.int32)
        self._check(self.lib.oefe_cell_info(self.h, int(cell), ctypes.byref(n), _ip(idx)))
        return idx

    def cell_matrix(self, ik, cell, complex_=False):
        idx = self.cell_info(cell)
        H = np.zeros((len(idx), len(idx)), np.complex128 if complex_ else np.float64)
        self._check(self.lib.oefe_cell_matrix(self.h, int(ik), int(cell), ctypes.c_void_p(H.ctypes.data)))
        return H

    def overlap(self, ik, complex_=False):
        nh, nO = self.ndof()
        m = np.zeros(nh)
        Moo = np.zeros((nO, nO), np.complex128 if complex_ else np.float64)
        self._check(self.lib.oefe_overlap(self.h, int(ik), _dp(m), ctypes.c_void_p(Moo.ctypes.data)))
        return m, Moo

    def apply_h(self, ik, X, Y):
        px, nv, ld, dt = _block(X)
        py, nv2, ld2, dt2 = _block(Y)
        if (nv2, ld2, dt2) != (nv, ld, dt):
            raise ValueError("X and Y must have the same shape, strides and dtype")
        self._check(self.lib.oefe_apply_h(self.h, int(ik), px, py, nv, ld, dt))
        return Y

    def apply_a(self, ik, X, Y):
        px, nv, ld, dt = _block(X)
        py, nv2, ld2, dt2 = _block(Y)
        if (nv2, ld2, dt2) != (nv, ld, dt):
            raise ValueError("X and Y must have the same shape, strides and dtype")
        self._check(self.lib.oefe_apply_a(self.h, int(ik), px, py, nv, ld, dt))
        return Y

    def apply_a_noalloc(self, ik, X, Y):
        """Y = (M^O)^{-1} H^O X without any device allocation: the library's
        scratch is a fixed device array (NOALLOC_SCRATCH_BYTES), shared by every
        call, for callers that cannot allocate device memory."""
        px, nv, ld, dt = _block(X)
        py, nv2, ld2, dt2 = _block(Y)
        if (nv2, ld2, dt2) != (nv, ld, dt):
            raise ValueError("X and Y must have the same shape, strides and dtype")
        self._check(self.lib.oefe_apply_a_noalloc(self.h, int(ik), px, py, nv, ld, dt))
        return Y

    def chebyshev_filter(self, ik, X, degree, a, b, a0, flags=0):
        px, nv, ld, dt = _block(X)
        self._check(self.lib.oefe_chebyshev_filter(self.h, int(ik), px, nv, ld, dt, int(degree), float(a),
                                                   float(b), float(a0), int(flags)))
        return X

    def _blocks(self, Xs):
        ptrs, nvs, lds, dts = [], [], [], []
        for X in Xs:
            p, nv, ld, dt = _block(X)
            ptrs.append(p.value)
            nvs.append(nv)
            lds.append(ld)
            dts.append(dt)
        if len(set(dts)) != 1:
            raise ValueError("all vector blocks must have the same dtype")
        return (ctypes.c_void_p * len(ptrs))(*ptrs), np.array(nvs, np.int32), np.array(lds, np.int32), dts[0]

    def filter_batched(self, Xs, degree, a, b, a0, flags):
        arr, nvs, lds, dt = self._blocks(Xs)
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), (len(Xs),)))
        b = np.ascontiguousarray(np.broadcast_to(np.asarray(b, np.float64), (len(Xs),)))
        a0 = np.ascontiguousarray(np.broadcast_to(np.asarray(a0, np.float64), (len(Xs),)))
        self._check(self.lib.oefe_filter_batched(self.h, len(Xs), arr, _ip(nvs), _ip(lds), dt, int(degree), _dp(a),
                                                 _dp(b), _dp(a0), int(flags)))
        return Xs

    def filter_batched_defect(self, Xs, degree, a, b, a0, theta, flags):
        """X[k] <- p_m(A) X[k] for Ritz-like blocks X[k] with values theta[k] (oefe_filter_batched_defect)."""
        arr, nvs, lds, dt = self._blocks(Xs)
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), (len(Xs),)))
        b = np.ascontiguousarray(np.broadcast_to(np.asarray(b, np.float64), (len(Xs),)))
        a0 = np.ascontiguousarray(np.broadcast_to(np.asarray(a0, np.float64), (len(Xs),)))
        th = np.ascontiguousarray(np.concatenate([np.asarray(t, np.float64).ravel() for t in theta]))
        if len(theta) != len(Xs) or th.size != int(np.sum(nvs)):
            raise ValueError("one theta per vector of every block")
        self._check(self.lib.oefe_filter_batched_defect(self.h, len(Xs), arr, _ip(nvs), _ip(lds), dt, int(degree),
                                                        _dp(a), _dp(b), _dp(a0), _dp(th), int(flags)))
        return Xs

    def filter_autotune(self, Xs):
        arr, nvs, lds, dt = self._blocks(Xs)
        ms = np.zeros(6)
        self._check(self.lib.oefe_filter_autotune(self.h, len(Xs), arr, _ip(nvs), _ip(lds), dt, _dp(ms)))
        return ms

    def orthonormalize(self, ik, X):
        px, nv, ld, dt = _block(X)
        cond = ctypes.c_double()
        self._check(self.lib.oefe_orthonormalize(self.h, int(ik), px, nv, ld, dt, ctypes.byref(cond)))
        return cond.value

    def rayleigh_ritz(self, ik, X, resid=False):
        px, nv, ld, dt = _block(X)
        eig = np.zeros(nv)
        res = np.zeros(nv) if resid else None
        self._check(self.lib.oefe_rayleigh_ritz(self.h, int(ik), px, nv, ld, dt, _dp(eig),
                                                _dp(res) if resid else None))
        return (eig, res) if resid else eig

    @staticmethod
    def _density_args(Xs, occ):
        ptrs, nvs, lds, dts = [], [], [], []
        for X in Xs:
            p, nv, ld, dt = _block(X)
            ptrs.append(p.value)
            nvs.append(nv)
            lds.append(ld)
            dts.append(dt)
        arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
        nvs = np.array(nvs, np.int32)
        lds = np.array(lds, np.int32)
        occ = np.ascontiguousarray(np.concatenate([np.asarray(o, np.float64) for o in occ]))
        dtype = C128 if C128 in dts else F64
        return arr, nvs, lds, dtype, occ

    def density(self, Xs, occ, rho):
        arr, nvs, lds, dtype, occ = self._density_args(Xs, occ)
        self._check(self.lib.oefe_density(self.h, len(Xs), arr, _ip(nvs), _ip(lds), dtype, _dp(occ),
                                          ctypes.c_void_p(rho.data_ptr())))
        return rho

    def density_grad(self, Xs, occ, rho, ik, gV):
        """rho (as density) and gV = band_trace_grad(ik, Xs[ik]) from one pass over the fields."""
        arr, nvs, lds, dtype, occ = self._density_args(Xs, occ)
        self._check(self.lib.oefe_density_grad(self.h, len(Xs), arr, _ip(nvs), _ip(lds), dtype, _dp(occ),
                                               ctypes.c_void_p(rho.data_ptr()), int(ik),
                                               ctypes.c_void_p(gV.data_ptr())))
        return rho, gV

    def band_trace_grad(self, ik, X, gV):
        px, nv, ld, dt = _block(X)
        self._check(self.lib.oefe_band_trace_grad(self.h, int(ik), px, nv, ld, dt, ctypes.c_void_p(gV.data_ptr())))
        return gV

    @staticmethod
    def _same(X, Y, what):
        if Y.shape != X.shape or Y.stride() != X.stride() or Y.dtype != X.dtype or not Y.is_cuda:
            raise ValueError("%s must have the shape, strides and dtype of X" % what)

    def band_trace(self, ik, X, HX=None):
        """tr(X^+ H X) (a float); H X into HX when given."""
        px, nv, ld, dt = _block(X)
        if HX is not None:
            self._same(X, HX, "HX")
        e = ctypes.c_double()
        self._check(self.lib.oefe_band_trace(self.h, int(ik), px, nv, ld, dt, ctypes.byref(e),
                                             ctypes.c_void_p(HX.data_ptr()) if HX is not None else None))
        return e.value

    def band_trace_vjp(self, ik, X, alpha, gV=None, gX=None):
        """gV = alpha w_q sum |u|^2 and gX = 2 alpha H X, into the given tensors (either may be None)."""
        px, nv, ld, dt = _block(X)
        if gX is not None:
            self._same(X, gX, "gX")
        self._check(self.lib.oefe_band_trace_vjp(self.h, int(ik), px, nv, ld, dt, float(alpha),
                                                 ctypes.c_void_p(gV.data_ptr()) if gV is not None else None,
                                                 ctypes.c_void_p(gX.data_ptr()) if gX is not None else None))
        return gV, gX

    def apply_h_vjp(self, ik, X, Gy, gV=None, gX=None):
        """gV = w_q Re sum conj(u_Gy) u_X and gX = H Gy, into the given tensors (either may be None)."""
        px, nv, ld, dt = _block(X)
        self._same(X, Gy, "Gy")
        if gX is not None:
            self._same(X, gX, "gX")
        self._check(self.lib.oefe_apply_h_vjp(self.h, int(ik), px, ctypes.c_void_p(Gy.data_ptr()),
                                              ctypes.c_void_p(gV.data_ptr()) if gV is not None else None,
                                              ctypes.c_void_p(gX.data_ptr()) if gX is not None else None,
                                              nv, ld, dt))
        return gV, gX

    def product_flops(self, ik, nv):
        """FP64 operations of one FP64 operator application's cell products for nv vectors."""
        f = ctypes.c_double()
        self._check(self.lib.oefe_product_flops(self.h, int(ik), int(nv), ctypes.byref(f)))
        return f.value

    def set_f64_products(self, mode):
        """Arithmetic of the FP64 cell products: F64_NATIVE, or F64_PAIRS (FP32 pairs on the
        single-leaf cells; needs an operator built with STORE_F64PAIR)."""
        self._check(self.lib.oefe_set_f64_products(self.h, int(mode)))

    def set_filter_shape(self, shape):
        """Keep one of the autotuner's launch shapes (0..5) for the BF16X3 filters; -1: untuned."""
        self._check(self.lib.oefe_set_filter_shape(self.h, int(shape)))

    def set_product_shape(self, shape):
        """Launch shape of the FP32-pair cell products: -1 timed at first use (default), or 0, 1, 2."""
        self._check(self.lib.oefe_set_product_shape(self.h, int(shape)))

    def release_workspace(self):
        """Free the cached scratch arrays (the build's are several times the filter's)."""
        self._check(self.lib.oefe_release_workspace(self.h))

    def kernel_timing(self, dtypes=()):
        mask = 0
        for d in dtypes:
            mask |= 1 << d
        self._check(self.lib.oefe_kernel_timing(self.h, mask))

    def kernel_time(self):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self.lib.oefe_kernel_time(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def upper_bound(self, ik, v0, steps=20, flags=0):
        b = ctypes.c_double()
        self._check(self.lib.oefe_upper_bound(self.h, int(ik), ctypes.c_void_p(v0.data_ptr()), int(steps),
                                              int(flags), ctypes.byref(b)))
        return b.value
