"""ctypes binding of libovgb.so (include/overlap.h), argument marshalling only.

Every computation runs in the CUDA library; this module converts Python
arguments (numpy arrays for host buffers, torch CUDA tensors for device
buffers, torch streams) into the plain pointers and sizes of the C ABI and
raises on a non-zero status.  If the library has not been built the import
of the loader fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libovgb.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "overlap.h")

OV_F64, OV_F32, OV_F16S, OV_BF16S, OV_DF64 = 0, 1, 2, 3, 4
PREC = {"f64": OV_F64, "f32": OV_F32, "f16": OV_F16S, "bf16": OV_BF16S, "df64": OV_DF64}
STATUS = {0: "OV_OK", -1: "OV_EINVAL", -2: "OV_ENOMEM", -3: "OV_ECUDA", -4: "OV_ENOTCONV", -5: "OV_ESTALL",
          -6: "OV_ETIMEOUT", -7: "OV_ENAN", -8: "OV_ESTATE"}


class OverlapError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("fallback", ctypes.c_int),
                ("nrhs", ctypes.c_int), ("true_residual", ctypes.c_double * 64), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {"iterations": self.iterations, "reliable_updates": self.reliable_updates,
                "fallback": self.fallback, "true_residual": list(self.true_residual[: self.nrhs]),
                "seconds": self.seconds}


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "ov_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "ov_destroy": (_I, [_P]),
    "ov_last_error": (ctypes.c_char_p, [_P]),
    "ov_set_gauge": (_I, [_P, _P, _P]),
    "ov_apply_dslash": (_I, [_P, _P, _P, _D, _I, _I, _P]),
    "ov_apply_Hw": (_I, [_P, _P, _P, _D, _I, _I, _P]),
    "ov_set_sign_poly": (_I, [_P, _D, _D, _I, _D]),
    "ov_get_sign_poly": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "ov_apply_overlap": (_I, [_P, _P, _P, _D, _I, _I, _P]),
    "ov_set_sign_rational": (_I, [_P, _D, _D, _I, _D]),
    "ov_get_sign_rational": (_I, [_P, ctypes.POINTER(_I), _P, _P, ctypes.POINTER(_D)]),
    "ov_apply_normal": (_I, [_P, _P, _P, _D, _I, _I, _I, _P]),
    "ov_deflate": (_I, [_P, _I, _I, _D, _P]),
    "ov_set_eigenpairs": (_I, [_P, _I, _I, _P, _P, _P]),
    "ov_get_eigenpairs": (_I, [_P, _I, ctypes.POINTER(_I), _P, _P, _P]),
    "ov_cg_solve": (_I, [_P, _P, _P, _I, _D, _D, _I, _I, _I, ctypes.POINTER(SolveInfo), _P]),
    "ov_cg_solve_multimass": (_I, [_P, _P, _P, _I, _I, _P, _D, _I, _I, _I, ctypes.POINTER(SolveInfo), _P]),
    "ov_net_train": (_I, [_P, _I, _I, _D, _D, ctypes.POINTER(_D), _P]),
    "ov_net_set_weights": (_I, [_P, _P, _I]),
    "ov_net_get_weights": (_I, [_P, _P, _I]),
    "ov_net_apply": (_I, [_P, _P, _P, _I, _P]),
    "ov_net_loss_grad": (_I, [_P, _P, _P, _I, ctypes.POINTER(_D), _P, _P]),
    "ov_net_pairs": (_I, [_P]),
    "ov_net_loss_history": (_I, [_P, _P, _I]),
    "ov_field_create": (_I, [_P, _I, _I, ctypes.POINTER(_P)]),
    "ov_field_destroy": (_I, [_P]),
    "ov_field_import": (_I, [_P, _P, _P, _P]),
    "ov_field_export": (_I, [_P, _P, _P, _P]),
    "ov_dslash_field": (_I, [_P, _P, _P, _D, _I, _P]),
    "ov_overlap_field": (_I, [_P, _P, _P, _D, _P]),
    "ov_field_dot": (_I, [_P, _P, _P, _P, _P]),
    "ov_lowmode_update": (_I, [_P, _I, _P, _P, _I, _P, _P, _P]),
    "ov_project_lowmodes": (_I, [_P, _I, _P, _I, _P, _P]),
    "ov_field_dot_noalloc": (_I, [_P, _P, _P, _P]),
    "ov_device_bytes": (ctypes.c_longlong, [_P]),
    "ov_dslash_count": (ctypes.c_longlong, [_P]),
    "ov_set_graphs": (_I, [_P, _I]),
    "ov_graph_stats": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "ov_measure_fma_peak": (_I, [_I, ctypes.POINTER(_D), _P]),
    "ov_set_option": (_I, [_P, ctypes.c_char_p, _D]),
    "ov_get_option": (_I, [_P, ctypes.c_char_p, ctypes.POINTER(_D)]),
    "ov_set_dslash_shape": (_I, [_P, _I, _I, _I, _I, _I]),
    "ov_tune_dslash": (_I, [_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), _P]),
}


def declared_symbols(header: str = HEADER):
    """Names of the functions declared in include/overlap.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ov_[A-Za-z0-9_]+)\s*\(", text)))


def load(path: str = LIBPATH):
    """Load libovgb.so and set the prototypes.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def measure_fma_peak(prec="f64", stream=None):
    """GFLOP/s of fused multiply-add on the current GPU (ov_measure_fma_peak): f64 or f32."""
    lib = load()
    g = _D()
    st = lib.ov_measure_fma_peak(_prec(prec), ctypes.byref(g), _stream(stream))
    if st != 0:
        raise OverlapError(st, "ov_measure_fma_peak failed")
    return g.value


def _ptr(x):
    """Device pointer of a contiguous torch tensor or host pointer of a numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("numpy buffer must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


def _nbytes(x):
    if isinstance(x, np.ndarray):
        return x.nbytes
    return x.numel() * x.element_size()


class Field:
    """An internal-layout even/odd field (ov_field)."""

    def __init__(self, ctx: "Context", nrhs: int, prec):
        self.ctx = ctx
        self.nrhs = nrhs
        self.prec = _prec(prec)
        h = _P()
        ctx._check(ctx.lib.ov_field_create(ctx.h, nrhs, self.prec, ctypes.byref(h)))
        self.h = h

    def load(self, x, stream=None):
        self.ctx._check(self.ctx.lib.ov_field_import(self.ctx.h, self.h, _ptr(x), _stream(stream)))

    def store(self, x, stream=None):
        self.ctx._check(self.ctx.lib.ov_field_export(self.ctx.h, self.h, _ptr(x), _stream(stream)))

    def close(self):
        if self.h:
            self.ctx.lib.ov_field_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One lattice on the current CUDA device (ov_ctx)."""

    def __init__(self, dims, bc=(1.0, 1.0, 1.0, -1.0)):
        self.lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        h = _P()
        st = self.lib.ov_create(ctypes.byref(h), (_I * 4)(*self.dims), (_D * 4)(*[float(b) for b in bc]))
        if st != 0:
            raise OverlapError(st, f"ov_create({self.dims}) failed")
        self.h = h

    def _check(self, st):
        if st != 0:
            raise OverlapError(st, self.lib.ov_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.ov_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _nrhs(self, x):
        n = _nbytes(x) // (self.V * 12 * 16)
        if n * self.V * 12 * 16 != _nbytes(x):
            raise ValueError("buffer size is not a whole number of complex128 spinor fields")
        return n

    # -- calls of the ABI --------------------------------------------------------------
    def set_gauge(self, U, stream=None):
        if _nbytes(U) != self.V * 36 * 16:
            raise ValueError("gauge buffer must be complex128 [Lt,Lz,Ly,Lx,4,3,3]")
        self._check(self.lib.ov_set_gauge(self.h, _ptr(U), _stream(stream)))

    def apply_dslash(self, x, out, m, prec="f64", stream=None):
        self._check(self.lib.ov_apply_dslash(self.h, _ptr(x), _ptr(out), float(m), self._nrhs(x), _prec(prec),
                                             _stream(stream)))
        return out

    def apply_Hw(self, x, out, m, prec="f64", stream=None):
        self._check(self.lib.ov_apply_Hw(self.h, _ptr(x), _ptr(out), float(m), self._nrhs(x), _prec(prec),
                                         _stream(stream)))
        return out

    def set_sign_poly(self, rho, eps, degree, lambda_max=0.0):
        self._check(self.lib.ov_set_sign_poly(self.h, float(rho), float(eps), int(degree), float(lambda_max)))

    def get_sign_poly(self):
        r, e, lm = _D(), _D(), _D()
        n = _I()
        self._check(self.lib.ov_get_sign_poly(self.h, ctypes.byref(r), ctypes.byref(e), ctypes.byref(n),
                                              ctypes.byref(lm)))
        return {"rho": r.value, "eps": e.value, "degree": n.value, "lambda_max": lm.value}

    def set_sign_rational(self, rho, eps, npoles, lambda_max=0.0):
        self._check(self.lib.ov_set_sign_rational(self.h, float(rho), float(eps), int(npoles), float(lambda_max)))

    def get_sign_rational(self):
        n = _I()
        d = _D()
        self._check(self.lib.ov_get_sign_rational(self.h, ctypes.byref(n), None, None, ctypes.byref(d)))
        b, c = np.empty(n.value), np.empty(n.value)
        self._check(self.lib.ov_get_sign_rational(self.h, ctypes.byref(n), _ptr(b), _ptr(c), ctypes.byref(d)))
        return b, c, d.value

    def apply_overlap(self, x, out, mass=0.0, prec="f64", stream=None):
        self._check(self.lib.ov_apply_overlap(self.h, _ptr(x), _ptr(out), float(mass), self._nrhs(x), _prec(prec),
                                              _stream(stream)))
        return out

    def apply_normal(self, x, out, mass=0.0, prec="f64", chiral=0, stream=None):
        self._check(self.lib.ov_apply_normal(self.h, _ptr(x), _ptr(out), float(mass), self._nrhs(x), _prec(prec),
                                             int(chiral), _stream(stream)))
        return out

    def deflate(self, which, nev, tol, stream=None):
        self._check(self.lib.ov_deflate(self.h, int(which), int(nev), float(tol), _stream(stream)))

    def set_eigenpairs(self, which, vals, vecs, stream=None):
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        self._check(self.lib.ov_set_eigenpairs(self.h, int(which), len(vals), _ptr(vals),
                                               _ptr(vecs) if len(vals) else None, _stream(stream)))

    def get_eigenpairs(self, which, stream=None):
        n = _I()
        self._check(self.lib.ov_get_eigenpairs(self.h, int(which), ctypes.byref(n), None, None, _stream(stream)))
        vals = np.empty(n.value)
        vecs = np.empty((n.value, self.V * 12), dtype=np.complex128)
        if n.value:
            self._check(self.lib.ov_get_eigenpairs(self.h, int(which), ctypes.byref(n), _ptr(vals), _ptr(vecs),
                                                   _stream(stream)))
        return vals, vecs

    def cg_solve(self, b, x, mass=0.0, tol=1e-10, max_iter=1000, precond=0, inner_prec="f64", stream=None,
                 check=True):
        info = SolveInfo()
        st = self.lib.ov_cg_solve(self.h, _ptr(b), _ptr(x), self._nrhs(b), float(mass), float(tol), int(max_iter),
                                  int(precond), _prec(inner_prec), ctypes.byref(info), _stream(stream))
        if check:
            self._check(st)
        return info.as_dict() | {"status": st}

    def cg_solve_multimass(self, b, x, masses, tol=1e-10, max_iter=3000, inner_prec="f32", output=0, stream=None,
                           check=True):
        """ov_cg_solve_multimass: x holds len(masses) x nrhs fields ([mass][rhs]); output 0 the
        normal-equation solutions, 1 D(m)^-1 b, 2 the propagators (1 - D/2) D(m)^-1 b."""
        m = np.ascontiguousarray(masses, dtype=np.float64)
        nrhs = self._nrhs(b)
        if _nbytes(x) != len(m) * _nbytes(b):
            raise ValueError("x must hold len(masses) x nrhs fields")
        infos = (SolveInfo * len(m))()
        st = self.lib.ov_cg_solve_multimass(self.h, _ptr(b), _ptr(x), nrhs, len(m), _ptr(m), float(tol),
                                            int(max_iter), _prec(inner_prec), int(output), infos, _stream(stream))
        if check:
            self._check(st)
        return [infos[k].as_dict() | {"status": st, "mass": float(m[k])} for k in range(len(m))]

    # -- learned preconditioner ---------------------------------------------------------
    NET_DOUBLES = 9216

    def net_train(self, nsolves=4, steps=100, lr=1e-2, mass=0.0, stream=None):
        loss = _D()
        self._check(self.lib.ov_net_train(self.h, int(nsolves), int(steps), float(lr), float(mass),
                                          ctypes.byref(loss), _stream(stream)))
        return loss.value

    def net_weights(self):
        w = np.empty(self.NET_DOUBLES)
        self._check(self.lib.ov_net_get_weights(self.h, _ptr(w), self.NET_DOUBLES))
        return w.view(np.complex128)

    def net_set_weights(self, w):
        w = np.ascontiguousarray(np.asarray(w, dtype=np.complex128)).view(np.float64)
        self._check(self.lib.ov_net_set_weights(self.h, _ptr(w), self.NET_DOUBLES))

    def net_apply(self, x, out, stream=None):
        self._check(self.lib.ov_net_apply(self.h, _ptr(x), _ptr(out), self._nrhs(x), _stream(stream)))
        return out

    def net_loss_grad(self, r, e, stream=None):
        loss = _D()
        g = np.empty(self.NET_DOUBLES)
        self._check(self.lib.ov_net_loss_grad(self.h, _ptr(r), _ptr(e), self._nrhs(r), ctypes.byref(loss), _ptr(g),
                                              _stream(stream)))
        return loss.value, g.view(np.complex128)

    def net_pairs(self):
        return int(self.lib.ov_net_pairs(self.h))

    def net_loss_history(self):
        """Mean loss per pair before each Adam step of the last net_train, and after the last."""
        n = int(self.lib.ov_net_loss_history(self.h, None, 0))
        if n < 0:
            raise OverlapError(-n, "ov_net_loss_history")
        out = np.empty(n)
        if n:
            self.lib.ov_net_loss_history(self.h, _ptr(out), n)
        return out

    def field(self, nrhs, prec):
        return Field(self, nrhs, prec)

    def dslash_field(self, fin: Field, fout: Field, m, gamma5=False, stream=None):
        self._check(self.lib.ov_dslash_field(self.h, fin.h, fout.h, float(m), int(bool(gamma5)), _stream(stream)))

    def overlap_field(self, fin: Field, fout: Field, mass=0.0, stream=None):
        self._check(self.lib.ov_overlap_field(self.h, fin.h, fout.h, float(mass), _stream(stream)))

    def project_lowmodes(self, which, psi: Field, engine=0, stream=None):
        """c[i][r] = v_i^dag psi_r of the stored eigenvectors; engine 0 CUDA cores, 1 tensor cores."""
        n = _I()
        self._check(self.lib.ov_get_eigenpairs(self.h, int(which), ctypes.byref(n), None, None, _stream(stream)))
        out = np.empty(2 * n.value * psi.nrhs)
        self._check(self.lib.ov_project_lowmodes(self.h, int(which), psi.h, int(engine), _ptr(out), _stream(stream)))
        return out.view(np.complex128).reshape(n.value, psi.nrhs)

    def lowmode_update(self, which, psi: Field, coef, out1: Field, out2: Field = None, engine=0, stream=None):
        """ov_lowmode_update: out1 = psi - sum_i v_i c[i][r], out2 = gamma5 sum_i sign(val_i) c[i][r] v_i."""
        cf = np.ascontiguousarray(np.asarray(coef, dtype=np.complex128)).view(np.float64)
        self._check(self.lib.ov_lowmode_update(self.h, int(which), psi.h, _ptr(cf), int(engine), out1.h,
                                               out2.h if out2 is not None else None, _stream(stream)))

    def field_dot(self, x: Field, y: Field, stream=None):
        out = np.empty(2 * x.nrhs)
        self._check(self.lib.ov_field_dot(self.h, x.h, y.h, _ptr(out), _stream(stream)))
        return out.view(np.complex128)

    def field_dot_noalloc(self, x: Field, y: Field, out=None, stream=None):
        """ov_field_dot_noalloc: out is a host numpy array (default) or a device tensor of 2*nrhs doubles."""
        if out is None:
            out = np.empty(2 * x.nrhs)
        st = self.lib.ov_field_dot_noalloc(x.h, y.h, _ptr(out), _stream(stream))
        if st != 0:
            raise OverlapError(st, "ov_field_dot_noalloc failed")
        return out.view(np.complex128) if isinstance(out, np.ndarray) else out

    def device_bytes(self):
        return int(self.lib.ov_device_bytes(self.h))

    def dslash_count(self):
        return int(self.lib.ov_dslash_count(self.h))

    def set_graphs(self, enable):
        self._check(self.lib.ov_set_graphs(self.h, int(bool(enable))))

    def graph_stats(self):
        """(graphs captured, graph replays) so far on this context."""
        cap, rep = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self.lib.ov_graph_stats(self.h, ctypes.byref(cap), ctypes.byref(rep)))
        return cap.value, rep.value

    def set_option(self, name, value):
        self._check(self.lib.ov_set_option(self.h, name.encode(), float(value)))

    def get_option(self, name):
        v = _D()
        self._check(self.lib.ov_get_option(self.h, name.encode(), ctypes.byref(v)))
        return v.value

    def set_dslash_shape(self, prec, nrhs, bx, by, variant=0):
        self._check(self.lib.ov_set_dslash_shape(self.h, _prec(prec), int(nrhs), int(bx), int(by), int(variant)))

    def tune_dslash(self, prec, nrhs, stream=None):
        bx, by, var = _I(), _I(), _I()
        self._check(self.lib.ov_tune_dslash(self.h, _prec(prec), int(nrhs), ctypes.byref(bx), ctypes.byref(by),
                                            ctypes.byref(var), _stream(stream)))
        return bx.value, by.value, var.value
