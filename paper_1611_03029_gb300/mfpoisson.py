"""ctypes binding of the C ABI declared in include/mfpoisson.h.

Argument marshalling only: every step runs in the CUDA library.  Device
buffers are torch tensors (contiguous, on the context's device); streams are
torch CUDA streams.  The library must have been built (``build.build()``);
importing this module without it raises, there is no fallback.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmfpoisson.so")

MFP_OK, MFP_ERR_ARG, MFP_ERR_CUDA, MFP_ERR_OOM = 0, -1, -2, -3
MFP_ERR_NOT_CONVERGED, MFP_ERR_STATE = -4, -6
MFP_CG, MFP_SIPG = 0, 1
MFP_FP64, MFP_FP32, MFP_MIXED = 0, 1, 2
MFP_MAP_IDENTITY, MFP_MAP_SINE, MFP_MAP_NODES = 0, 1, 2
MFP_ARITH_DF, MFP_ARITH_NATIVE = 0, 1


class MfpDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("degree", ctypes.c_int),
                ("disc", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("mapping", ctypes.c_int), ("map_param", ctypes.c_double),
                ("kappa", ctypes.c_double),
                ("penalty_factor", ctypes.c_double),
                ("mg_precision", ctypes.c_int),
                ("cheb_degree", ctypes.c_int),
                ("eig_cg_iters", ctypes.c_int),
                ("fp64_arith", ctypes.c_int),
                ("neumann_sides", ctypes.c_int),
                ("box_lo", ctypes.c_double), ("box_hi", ctypes.c_double),
                ("map_nodes", ctypes.POINTER(ctypes.c_double))]


class MfpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("mfpoisson error %d: %s" % (status, msg))
        self.status = status


_lib = None


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libmfpoisson.so is missing; run "
                "paper_1611_03029_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
        dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        sig = {
            "mfp_desc_default": (None, [ctypes.POINTER(MfpDesc)]),
            "mfp_create": (ctypes.c_int, [ctypes.POINTER(MfpDesc), vp,
                                          ctypes.POINTER(vp)]),
            "mfp_destroy": (ctypes.c_int, [vp]),
            "mfp_n_levels": (ctypes.c_int, [vp]),
            "mfp_sizes": (ctypes.c_int, [vp, ctypes.c_int, i64p, i64p, i64p]),
            "mfp_set_coefficient": (ctypes.c_int, [vp, vp, vp, vp]),
            "mfp_rhs": (ctypes.c_int, [vp, ctypes.c_int, dp, ctypes.c_int, vp,
                                       ctypes.c_int64, vp]),
            "mfp_rhs_noalloc": (ctypes.c_int, [vp, ctypes.c_int, dp,
                                               ctypes.c_int, vp,
                                               ctypes.c_int64, vp]),
            "mfp_apply": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp,
                                         vp, ctypes.c_int, vp]),
            "mfp_hdg_apply": (ctypes.c_int, [vp, ctypes.c_double, vp, vp,
                                             vp]),
            "mfp_inverse_diagonal": (ctypes.c_int, [vp, ctypes.c_int,
                                                    ctypes.c_int, vp, vp]),
            "mfp_level_info": (ctypes.c_int, [vp, ctypes.c_int, dp, dp, dp,
                                              dp, ip]),
            "mfp_prolongate": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int,
                                              vp, vp, vp]),
            "mfp_restrict": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int,
                                            vp, vp, vp]),
            "mfp_smooth": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp,
                                          vp, ctypes.c_int, vp]),
            "mfp_vcycle": (ctypes.c_int, [vp, vp, vp, ctypes.c_int, vp]),
            "mfp_solve": (ctypes.c_int, [vp, vp, vp, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, ip,
                                         dp, vp]),
            "mfp_gradient": (ctypes.c_int, [vp, vp, vp, vp, vp, vp]),
            "mfp_counters": (ctypes.c_int, [vp, i64p, i64p, i64p]),
            "mfp_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ip, dp, vp]),
            "mfp_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != MFP_OK:
        raise MfpError(status, lib().mfp_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


_PREC = {"fp64": MFP_FP64, "fp32": MFP_FP32, "mixed": MFP_MIXED}


def neumann_mask(sides):
    """Bit mask of the Neumann sides: side 2e is x_e = lo, 2e+1 is x_e = hi."""
    m = 0
    for s in sides:
        if not 0 <= int(s) <= 5:
            raise ValueError("Neumann sides are 0..5")
        m |= 1 << int(s)
    return m
_DT = {MFP_FP64: torch.float64, MFP_FP32: torch.float32}


class Poisson:
    """A multigrid hierarchy of the matrix-free Poisson operator (one
    mfp_ctx).  Level -1 / None is the finest."""

    def __init__(self, nx, ny, nz, degree, disc="cg", n_levels=0,
                 mapping="identity", map_param=0.0, kappa=1.0,
                 penalty_factor=1.0, mg_precision="fp64", cheb_degree=5,
                 eig_cg_iters=15, fp64_arith="df", neumann_sides=(),
                 box=(0.0, 1.0), map_nodes=None, stream=None):
        L = lib()
        d = MfpDesc()
        L.mfp_desc_default(ctypes.byref(d))
        d.nx, d.ny, d.nz, d.degree = nx, ny, nz, degree
        d.disc = {"cg": MFP_CG, "dg": MFP_SIPG, "sipg": MFP_SIPG}[disc]
        d.n_levels = n_levels
        d.mapping = {"identity": MFP_MAP_IDENTITY, "sine": MFP_MAP_SINE,
                     "nodes": MFP_MAP_NODES}[mapping]
        nodes = None
        if mapping == "nodes":
            import numpy as np
            # host array [ncells][(k+1)^3][3], copied by mfp_create
            nodes = np.ascontiguousarray(map_nodes, dtype=np.float64)
            if nodes.size != nx * ny * nz * (degree + 1) ** 3 * 3:
                raise ValueError("map_nodes must be [ncells, (k+1)^3, 3]")
            d.map_nodes = nodes.ctypes.data_as(
                ctypes.POINTER(ctypes.c_double))
        d.map_param = map_param
        d.kappa = kappa
        d.penalty_factor = penalty_factor
        d.mg_precision = _PREC[mg_precision]
        d.cheb_degree = cheb_degree
        d.eig_cg_iters = eig_cg_iters
        d.fp64_arith = {"df": MFP_ARITH_DF, "native": MFP_ARITH_NATIVE}[
            fp64_arith]
        d.neumann_sides = neumann_mask(neumann_sides)
        d.box_lo, d.box_hi = float(box[0]), float(box[1])
        self.desc = d
        self.disc = disc
        self.degree = degree
        self.n = (nx, ny, nz)
        self.vprec = MFP_FP64 if mg_precision == "fp64" else MFP_FP32
        h = ctypes.c_void_p()
        _check(L.mfp_create(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().mfp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- sizes --------------------------------------------------------
    @property
    def n_levels(self):
        return lib().mfp_n_levels(self._h)

    def _lvl(self, level):
        return self.n_levels - 1 if level is None or level < 0 else level

    def sizes(self, level=None):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().mfp_sizes(self._h, self._lvl(level), ctypes.byref(a),
                               ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def n_dofs(self, level=None):
        return self.sizes(level)[0]

    # ---- operations ---------------------------------------------------
    def set_coefficient(self, a_cell, a_face=None, stream=None):
        _check(lib().mfp_set_coefficient(self._h, _ptr(a_cell), _ptr(a_face),
                                         _stream(stream)))
        # stamp of the coefficient the context now holds
        self.coef_stamp = getattr(self, "coef_stamp", 0) + 1

    def rhs(self, kind=0, params=None, out=None, stride=1, stream=None):
        n = self.n_dofs()
        if out is None:
            out = torch.empty(n * stride, dtype=torch.float64, device="cuda")
        arr, nterms = None, 0
        if params is not None:
            import numpy as np
            p = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 5)
            nterms = p.shape[0]
            arr = p.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            self._keep = p
        _check(lib().mfp_rhs(self._h, kind, arr, nterms, _ptr(out), stride,
                             _stream(stream)))
        return out

    def apply(self, src, dst=None, level=None, n_rhs=1, stream=None):
        prec = MFP_FP64 if src.dtype == torch.float64 else MFP_FP32
        if dst is None:
            dst = torch.empty_like(src)
        _check(lib().mfp_apply(self._h, self._lvl(level), prec, _ptr(src),
                               _ptr(dst), n_rhs, _stream(stream)))
        return dst

    def hdg_apply(self, x, y=None, tau_factor=5.0, stream=None):
        """HDG mixed operator on the cell unknowns (q_x, q_y, q_z, u),
        cell-major blocks of 4 (k+1)^3 values (SIPG contexts)."""
        if y is None:
            y = torch.empty_like(x)
        _check(lib().mfp_hdg_apply(self._h, tau_factor, _ptr(x), _ptr(y),
                                   _stream(stream)))
        return y

    def inverse_diagonal(self, level=None, dtype=torch.float64, stream=None):
        lv = self._lvl(level)
        out = torch.empty(self.n_dofs(lv), dtype=dtype, device="cuda")
        prec = MFP_FP64 if dtype == torch.float64 else MFP_FP32
        _check(lib().mfp_inverse_diagonal(self._h, lv, prec, _ptr(out),
                                          _stream(stream)))
        return out

    def level_info(self, level=None):
        v = [ctypes.c_double() for _ in range(4)]
        deg = ctypes.c_int()
        _check(lib().mfp_level_info(self._h, self._lvl(level),
                                    *[ctypes.byref(x) for x in v],
                                    ctypes.byref(deg)))
        return dict(lam_max=v[0].value, lam_min=v[1].value, lo=v[2].value,
                    hi=v[3].value, degree=deg.value)

    def prolongate(self, xc, level, stream=None):
        prec = MFP_FP64 if xc.dtype == torch.float64 else MFP_FP32
        xf = torch.empty(self.n_dofs(level), dtype=xc.dtype, device="cuda")
        _check(lib().mfp_prolongate(self._h, level, prec, _ptr(xc), _ptr(xf),
                                    _stream(stream)))
        return xf

    def restrict(self, xf, level, stream=None):
        prec = MFP_FP64 if xf.dtype == torch.float64 else MFP_FP32
        xc = torch.empty(self.n_dofs(level - 1), dtype=xf.dtype,
                         device="cuda")
        _check(lib().mfp_restrict(self._h, level, prec, _ptr(xf), _ptr(xc),
                                  _stream(stream)))
        return xc

    def smooth(self, b, x=None, level=None, stream=None):
        prec = MFP_FP64 if b.dtype == torch.float64 else MFP_FP32
        zero = x is None
        if x is None:
            x = torch.empty_like(b)
        _check(lib().mfp_smooth(self._h, self._lvl(level), prec, _ptr(b),
                                _ptr(x), int(zero), _stream(stream)))
        return x

    def vcycle(self, r, z=None, n_rhs=1, stream=None):
        if z is None:
            z = torch.empty_like(r)
        _check(lib().mfp_vcycle(self._h, _ptr(r), _ptr(z), n_rhs,
                                _stream(stream)))
        return z

    def solve(self, b, x=None, n_rhs=1, rtol=1e-10, max_it=200, stream=None,
              raise_on_fail=True):
        if x is None:
            x = torch.empty_like(b)
        its = (ctypes.c_int * n_rhs)()
        rel = (ctypes.c_double * n_rhs)()
        st = lib().mfp_solve(self._h, _ptr(b), _ptr(x), n_rhs, rtol, max_it,
                             its, rel, _stream(stream))
        if st != MFP_OK and (raise_on_fail or st != MFP_ERR_NOT_CONVERGED):
            _check(st)
        return x, list(its), list(rel)

    def gradient(self, u, lam, stream=None):
        _, ncq, nfq = self.sizes()
        p = self.degree + 1
        gc = torch.empty(ncq // p ** 3, p ** 3, dtype=torch.float64,
                         device="cuda")
        gf = None
        if self.disc != "cg":
            gf = torch.empty(nfq // p ** 2, p ** 2, dtype=torch.float64,
                             device="cuda")
        _check(lib().mfp_gradient(self._h, _ptr(u), _ptr(lam), _ptr(gc),
                                  _ptr(gf), _stream(stream)))
        return gc, gf

    def autotune(self, level=None, prec="fp64", n_rhs=1, stream=None):
        """Pick the fastest cells-per-block for this apply; returns
        (cells, ms per apply)."""
        cells, ms = ctypes.c_int(), ctypes.c_double()
        p = MFP_FP64 if prec in ("fp64", torch.float64) else MFP_FP32
        _check(lib().mfp_autotune(self._h, self._lvl(level), p, n_rhs,
                                  ctypes.byref(cells), ctypes.byref(ms),
                                  _stream(stream)))
        return cells.value, ms.value

    def counters(self):
        arr = (ctypes.c_int64 * self.n_levels)()
        v, k = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().mfp_counters(self._h, arr, ctypes.byref(v),
                                  ctypes.byref(k)))
        return list(arr), v.value, k.value


class MFPSolve(torch.autograd.Function):
    """u = A(a)^{-1} f as a differentiable function of the per-point
    coefficient (a_cell, a_face).  Backward solves A lambda = dL/du with the
    same symmetric operator and returns -lambda^T (dA/da) u from the
    library's gradient kernel.  The context holds one coefficient at a time:
    forward saves its own, and backward sets it again if another forward (or
    set_coefficient) has replaced it on the same context since."""

    @staticmethod
    def forward(ctx, a_cell, a_face, op, b, rtol, max_it):
        a_cell = a_cell.contiguous()
        a_face = None if a_face is None else a_face.contiguous()
        op.set_coefficient(a_cell, a_face)
        u, its, rel = op.solve(b, rtol=rtol, max_it=max_it)
        ctx.op, ctx.rtol, ctx.max_it = op, rtol, max_it
        ctx.stamp = op.coef_stamp
        ctx.has_face = a_face is not None
        if a_face is None:
            ctx.save_for_backward(u, a_cell)
        else:
            ctx.save_for_backward(u, a_cell, a_face)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        u, a_cell = ctx.saved_tensors[:2]
        if ctx.op.coef_stamp != ctx.stamp:
            a_face = ctx.saved_tensors[2] if ctx.has_face else None
            ctx.op.set_coefficient(a_cell.detach(), None if a_face is None
                                   else a_face.detach())
            ctx.stamp = ctx.op.coef_stamp
        lam, _, _ = ctx.op.solve(grad_u.contiguous(), rtol=ctx.rtol,
                                 max_it=ctx.max_it)
        gc, gf = ctx.op.gradient(u, lam)
        return gc, (gf if ctx.has_face else None), None, None, None, None
