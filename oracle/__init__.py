"""FP64 CPU oracle for the overlap-operator hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it, and it shares no code
with that path: ``oracle.c`` is a plain restatement of the paper's equations
in canonical layout with explicit 4x4 gamma matrices.

Functions and what pins each one (tests/test_oracle_*.py):

============================  =====================================================
``dslash`` / ``hw``           Eqs. (1)-(2).  Free-field plane-wave closed form,
                              gamma_5-hermiticity, gauge covariance, translation
                              covariance, dense D_w^dag = g5 D_w g5 on 2^4, L=2.
``cheb_coeffs`` / ``poly_*``  Eq. (4).  Interpolation at the nodes, numpy's
                              independent Chebyshev interpolant, the geometric
                              error rate (1+sqrt(eps))/(1-sqrt(eps)), Eq. (11).
``sign``                      Eqs. (5)-(7).  Dense eigendecomposition sign on
                              2^4 and 4^4, sign^2 = 1, free-field closed form.
``overlap``                   Eqs. (3), (8).  Free-field closed form, the
                              Ginsparg-Wilson relation, spectrum on the circle
                              |d - rho| = rho, D^dag D = rho (D + D^dag).
``overlap_normal`` / ``cg``   Eq. (9).  Dense linear solve on 2^4; true residual.
``multimass_cg``              Sec. II.  Dense solves of every mass; single-mass CG.
``lambda_max``                Eq. (5).  Dense eigendecomposition: a lower bound of
                              max |lambda| that reaches it when the Krylov space
                              is the whole space.
``lanczos_lowmodes``          Sec. V, Eq. (7).  Dense eigendecomposition on 2^4
                              (whole space) and 4^4; eigen-residuals.
``ellipk`` / ``jacobi``       scipy.special's independent K(m) and ellipj.
``zolotarev``                 Eq. (12).  Closed form at n = 1; equioscillation of
                              the error with 2n + 1 extremes of equal size.
``sign_rational``             Eqs. (7), (12).  Dense eigendecomposition sign on
                              2^4; sign^2 = 1; agreement with the polynomial sign.
``net_layer`` / ``_grad``     No paper counterpart.  Central finite differences
                              and gauge equivariance.
============================  =====================================================
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

c_int_p = ctypes.POINTER(ctypes.c_int)
c_dbl_p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no fast-math)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", _SO, src, "-lm"]
        )
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
    return _lib


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(lib().or_threads())


def set_threads(n: int) -> None:
    lib().or_set_threads(ctypes.c_int(int(n)))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(v) for v in dims])


def _bc(bc):
    return (ctypes.c_double * 4)(*[float(v) for v in bc])


def _field(x, V):
    x = np.ascontiguousarray(x, dtype=np.complex128)
    assert x.size == 12 * V, (x.shape, V)
    return x


def volume(dims):
    return int(np.prod([int(v) for v in dims]))


def gamma(mu: int) -> np.ndarray:
    """gamma_{mu+1} for mu = 0..3, gamma_5 for mu = 4 (4x4, chiral basis)."""
    out = np.zeros(16, dtype=np.complex128)
    lib().or_gamma(ctypes.c_int(mu), _ptr(out))
    return out.reshape(4, 4)


def _gauge(U, V):
    U = np.ascontiguousarray(U, dtype=np.complex128)
    assert U.size == 36 * V
    return U


def dslash(dims, bc, U, m, x):
    """D_w(m) x (Eq. 1) for one canonical spinor field."""
    V = volume(dims)
    x = _field(x, V)
    out = np.empty_like(x)
    lib().or_dslash(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(m), _ptr(x), _ptr(out))
    return out


def dslash_sites(dims, bc, U, m, x, sites):
    """(D_w(m) x) at the given canonical site indices, [nsites, 4, 3]."""
    V = volume(dims)
    x = _field(x, V)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    lib().or_dslash_sites(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(m), _ptr(x),
                          ctypes.c_long(len(sites)), _ptr(sites), _ptr(out))
    return out


def gamma5(x):
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    lib().or_gamma5(ctypes.c_long(x.size // 12), _ptr(x), _ptr(out))
    return out


def hw(dims, bc, U, m, x):
    """H_w = gamma_5 D_w(m) x."""
    V = volume(dims)
    x = _field(x, V)
    out = np.empty_like(x)
    lib().or_hw(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(m), _ptr(x), _ptr(out))
    return out


def cheb_coeffs(eps: float, n: int) -> np.ndarray:
    """Chebyshev-interpolant coefficients c_0..c_n of x^{-1/2} on [eps, 1] (c_0 halved)."""
    c = np.empty(n + 1)
    lib().or_cheb_coeffs(ctypes.c_double(eps), ctypes.c_int(n), _ptr(c))
    return c


def poly_eval(c, eps, x):
    c = np.ascontiguousarray(c, dtype=np.float64)
    f = lib().or_poly_eval
    f.restype = ctypes.c_double
    return np.array([f(_ptr(c), ctypes.c_int(len(c) - 1), ctypes.c_double(eps), ctypes.c_double(v))
                     for v in np.atleast_1d(x)])


def poly_delta(c, eps, npts=100000):
    """delta of Eq. (4) on a log-spaced grid of npts points."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    f = lib().or_poly_delta
    f.restype = ctypes.c_double
    return f(_ptr(c), ctypes.c_int(len(c) - 1), ctypes.c_double(eps), ctypes.c_int(npts))


def _defl(evals, evecs, V):
    if evals is None or len(evals) == 0:
        return 0, np.zeros(1), np.zeros(12, dtype=np.complex128)
    evals = np.ascontiguousarray(evals, dtype=np.float64)
    evecs = np.ascontiguousarray(evecs, dtype=np.complex128)
    assert evecs.size == len(evals) * 12 * V
    return len(evals), evals, evecs


def lambda_max(dims, bc, U, mw, steps=50, v0=None):
    """sqrt of the largest Ritz value of H_w^2 after `steps` Lanczos steps from v0 (Eq. 5 rescale)."""
    V = volume(dims)
    if v0 is None:
        v0 = np.ones(12 * V, dtype=np.complex128)
    v0 = _field(v0, V)
    f = lib().or_lambda_max
    f.restype = ctypes.c_double
    return f(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(mw), ctypes.c_int(steps), _ptr(v0))


def lanczos_lowmodes(dims, bc, U, mw, m, nev, v0=None):
    """The nev smallest-|lambda| eigenpairs of H_w from m Lanczos steps on H_w^2 and Rayleigh-Ritz with
    H_w (Eq. 7 needs the signs).  Returns (vals [nev], vecs [nev, 12V], max eigen-residual)."""
    V = volume(dims)
    if v0 is None:
        v0 = np.ones(12 * V, dtype=np.complex128)
    v0 = _field(v0, V)
    vals = np.empty(nev)
    vecs = np.empty((nev, 12 * V), dtype=np.complex128)
    f = lib().or_lanczos_lowmodes
    f.restype = ctypes.c_double
    r = f(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(mw), ctypes.c_int(m), ctypes.c_int(nev), _ptr(v0),
          _ptr(vals), _ptr(vecs))
    return vals, vecs, r


def ellipk(m: float) -> float:
    """Complete elliptic integral K(m), parameter m = k^2 (AGM)."""
    f = lib().or_ellipk
    f.restype = ctypes.c_double
    return f(ctypes.c_double(m))


def jacobi(u: float, m: float):
    """(sn, cn, dn)(u | m) by the descending AGM."""
    sn, cn, dn = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().or_jacobi(ctypes.c_double(u), ctypes.c_double(m), ctypes.byref(sn), ctypes.byref(cn), ctypes.byref(dn))
    return sn.value, cn.value, dn.value


def zolotarev(eps: float, n: int):
    """Zolotarev's optimal P(x) = sum_i b_i / (x + c_i) ~ x^{-1/2} on [eps, 1] (Eq. 12).
    Returns (b, c, delta)."""
    b, c = np.empty(n), np.empty(n)
    f = lib().or_zolotarev
    f.restype = ctypes.c_double
    d = f(ctypes.c_double(eps), ctypes.c_int(n), _ptr(b), _ptr(c))
    return b, c, d


def rational_eval(b, c, x):
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    f = lib().or_rational_eval
    f.restype = ctypes.c_double
    return np.array([f(_ptr(b), _ptr(c), ctypes.c_int(len(b)), ctypes.c_double(v)) for v in np.atleast_1d(x)])


def sign_rational(dims, bc, U, mw, lmax, b, c, x, tol=1e-14, evals=None, evecs=None):
    """sign(H_w(mw)) x by Eq. (7) with the rational P of Eq. (12), shifted inverses by multi-shift CG."""
    V = volume(dims)
    x = _field(x, V)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    nev, lam, eta = _defl(evals, evecs, V)
    out = np.empty_like(x)
    lib().or_sign_rational(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(mw), ctypes.c_double(lmax),
                           ctypes.c_int(len(b)), _ptr(b), _ptr(c), ctypes.c_double(tol), ctypes.c_int(nev), _ptr(lam),
                           _ptr(eta), _ptr(x), _ptr(out))
    return out


def overlap_rational(dims, bc, U, rho, mass, lmax, b, c, x, tol=1e-14, evals=None, evecs=None):
    """D(m) x with the rational sign (Eqs. 3, 8, 12)."""
    V = volume(dims)
    x = _field(x, V)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    nev, lam, eta = _defl(evals, evecs, V)
    out = np.empty_like(x)
    lib().or_overlap_rational(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(rho), ctypes.c_double(mass),
                              ctypes.c_double(lmax), ctypes.c_int(len(b)), _ptr(b), _ptr(c), ctypes.c_double(tol),
                              ctypes.c_int(nev), _ptr(lam), _ptr(eta), _ptr(x), _ptr(out))
    return out


def sign(dims, bc, U, mw, lmax, eps, coeffs, x, evals=None, evecs=None):
    """sign(H_w(mw)) x by Eq. (7): exact on the given eigenpairs of H_w, Q P(Q^2) elsewhere."""
    V = volume(dims)
    x = _field(x, V)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    nev, lam, eta = _defl(evals, evecs, V)
    out = np.empty_like(x)
    lib().or_sign(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(mw), ctypes.c_double(lmax),
                  ctypes.c_double(eps), ctypes.c_int(len(coeffs) - 1), _ptr(coeffs), ctypes.c_int(nev),
                  _ptr(lam), _ptr(eta), _ptr(x), _ptr(out))
    return out


def overlap(dims, bc, U, rho, mass, lmax, eps, coeffs, x, evals=None, evecs=None):
    """D(m) x = rho D x + m (1 - D/2) x with D = 1 + gamma_5 sign(H_w(-rho)) (Eqs. 3, 8)."""
    V = volume(dims)
    x = _field(x, V)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    nev, lam, eta = _defl(evals, evecs, V)
    out = np.empty_like(x)
    lib().or_overlap(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(rho), ctypes.c_double(mass),
                     ctypes.c_double(lmax), ctypes.c_double(eps), ctypes.c_int(len(coeffs) - 1), _ptr(coeffs),
                     ctypes.c_int(nev), _ptr(lam), _ptr(eta), _ptr(x), _ptr(out))
    return out


def overlap_normal(dims, bc, U, rho, mass, lmax, eps, coeffs, x, evals=None, evecs=None):
    """D(m)^dag D(m) x."""
    V = volume(dims)
    x = _field(x, V)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    nev, lam, eta = _defl(evals, evecs, V)
    out = np.empty_like(x)
    lib().or_overlap_normal(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(rho),
                            ctypes.c_double(mass), ctypes.c_double(lmax), ctypes.c_double(eps),
                            ctypes.c_int(len(coeffs) - 1), _ptr(coeffs), ctypes.c_int(nev), _ptr(lam),
                            _ptr(eta), _ptr(x), _ptr(out))
    return out


def cg(dims, bc, U, rho, mass, lmax, eps, coeffs, b, tol=1e-10, max_iter=1000, evals=None,
       evecs=None, mu=None, xi=None, zero_tol=1e-10):
    """Deflated CG on D(m)^dag D(m) x = b.  Returns (x, iterations, true relative residual)."""
    V = volume(dims)
    b = _field(b, V)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    nev, lam, eta = _defl(evals, evecs, V)
    nev2, mu_, xi_ = _defl(mu, xi, V)
    x = np.empty_like(b)
    res = ctypes.c_double(0)
    it = lib().or_cg(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(rho), ctypes.c_double(mass),
                     ctypes.c_double(lmax), ctypes.c_double(eps), ctypes.c_int(len(coeffs) - 1), _ptr(coeffs),
                     ctypes.c_int(nev), _ptr(lam), _ptr(eta), ctypes.c_int(nev2), _ptr(mu_), _ptr(xi_),
                     ctypes.c_double(zero_tol), _ptr(b), _ptr(x), ctypes.c_double(tol), ctypes.c_int(max_iter),
                     ctypes.byref(res))
    return x, it, res.value


def multimass_cg(dims, bc, U, rho, lmax, eps, coeffs, b, masses, tol=1e-10, max_iter=1000, evals=None,
                 evecs=None, mu=None, xi=None):
    """One multi-shifted CG for D(m)^dag D(m) x_m = b at every mass m (Sec. II), the low modes
    (mu, xi) of the massless D^dag D deflated.  Returns (x [nmass, V, 4, 3], iterations,
    true relative residuals per mass with the two-sign operator)."""
    V = volume(dims)
    b = _field(b, V)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    masses = np.ascontiguousarray(masses, dtype=np.float64)
    nev, lam, eta = _defl(evals, evecs, V)
    nev2, mu_, xi_ = _defl(mu, xi, V)
    x = np.empty((len(masses),) + b.shape, dtype=np.complex128)
    res = np.empty(len(masses))
    it = lib().or_multimass_cg(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_double(rho),
                               ctypes.c_double(lmax), ctypes.c_double(eps), ctypes.c_int(len(coeffs) - 1),
                               _ptr(coeffs), ctypes.c_int(nev), _ptr(lam), _ptr(eta), ctypes.c_int(nev2), _ptr(mu_),
                               _ptr(xi_), ctypes.c_int(len(masses)), _ptr(masses), _ptr(b), _ptr(x),
                               ctypes.c_double(tol), ctypes.c_int(max_iter), _ptr(res))
    return x, it, res


def net_layer(dims, bc, U, W, x):
    """One gauge-covariant layer: W [9, cout, cin, 4, 4], x [cin, V, 4, 3] -> y [cout, V, 4, 3]."""
    V = volume(dims)
    W = np.ascontiguousarray(W, dtype=np.complex128)
    _, cout, cin = W.shape[:3]
    x = np.ascontiguousarray(x, dtype=np.complex128).reshape(cin, V, 4, 3)
    y = np.empty((cout, V, 4, 3), dtype=np.complex128)
    lib().or_net_layer(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_int(cin), ctypes.c_int(cout),
                       _ptr(W), _ptr(x), _ptr(y))
    return y


def net_layer_grad(dims, bc, U, W, x, gy):
    """Backward of net_layer: returns (gx, gW) for upstream gradient gy (Re + i Im convention)."""
    V = volume(dims)
    W = np.ascontiguousarray(W, dtype=np.complex128)
    _, cout, cin = W.shape[:3]
    x = np.ascontiguousarray(x, dtype=np.complex128).reshape(cin, V, 4, 3)
    gy = np.ascontiguousarray(gy, dtype=np.complex128).reshape(cout, V, 4, 3)
    gx = np.empty((cin, V, 4, 3), dtype=np.complex128)
    gW = np.empty_like(W)
    lib().or_net_layer_grad(_dims(dims), _bc(bc), _ptr(_gauge(U, V)), ctypes.c_int(cin), ctypes.c_int(cout),
                            _ptr(W), _ptr(x), _ptr(gy), _ptr(gx), _ptr(gW))
    return gx, gW


def net_apply(dims, bc, U, W1, W2, x):
    """The 2-layer preconditioner M(x) = L2(L1(x)) (linear, gauge covariant)."""
    h = net_layer(dims, bc, U, W1, x)
    return net_layer(dims, bc, U, W2, h)[0]
