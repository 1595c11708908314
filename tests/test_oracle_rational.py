"""Pins of the oracle's rational sign function (Eq. 12: P(x) = sum_i b_i / (x + c_i),
Zolotarev's optimal coefficients, the shifted inverses by one multi-shift CG):

* its elliptic functions against scipy.special's independent K(m) and ellipj;
* the coefficients at n = 1 against their closed form, and for larger n by the
  property that characterises the optimal approximation: the error
  1 - sqrt(x) P(x) equioscillates with 2n + 1 extremes of equal size delta;
* the rational sign of H_w against a dense eigendecomposition on 2^4, with and
  without low-mode deflation (Eq. 7), sign^2 = 1, and agreement with the
  polynomial sign where both are accurate."""
import numpy as np
import pytest

import oracle
import synth
from _util import rel
from test_oracle_sign import ABC, RHO, small_case  # noqa: F401  (fixture)

scipy_special = pytest.importorskip("scipy.special")


@pytest.mark.parametrize("m", [1e-6, 0.1, 0.5, 0.9, 0.99, 1 - 1e-6])
def test_elliptic_functions_match_scipy(m):
    assert abs(oracle.ellipk(m) / scipy_special.ellipk(m) - 1) < 1e-14
    for u in (0.0, 0.1, 0.7, 1.3, 0.9 * scipy_special.ellipk(m)):
        sn, cn, dn, _ = scipy_special.ellipj(u, m)
        got = oracle.jacobi(u, m)
        assert np.allclose(got, (sn, cn, dn), rtol=0, atol=2e-14), (u, m, got, (sn, cn, dn))


@pytest.mark.parametrize("eps", [0.01, 0.2])
def test_zolotarev_one_pole_closed_form(eps):
    """n = 1: sign(q) ~ D q / (q^2 + k), k = sqrt(eps); q / (q^2 + k) takes 1/(1+k) at both
    ends of [k, 1] and 1/(2 sqrt k) at q = sqrt(k), so D = 2 / (1/(1+k) + 1/(2 sqrt k))."""
    k = np.sqrt(eps)
    b, c, d = oracle.zolotarev(eps, 1)
    D = 2.0 / (1.0 / (1.0 + k) + 1.0 / (2.0 * np.sqrt(k)))
    assert abs(c[0] - k) < 1e-14 and abs(b[0] - D) < 1e-14
    assert abs(d - (1.0 / (2 * np.sqrt(k)) - 1.0 / (1 + k)) / (1.0 / (2 * np.sqrt(k)) + 1.0 / (1 + k))) < 1e-14


def _alternation(err, lo, hi, G=20001, S=2001):
    """Signed extreme values of err on [lo, hi]: the sign changes of err split the interval into
    segments (robust against rounding: |err| is ~delta away from its zeros), and the extreme of
    each segment is taken on a fine sample of it."""
    q = np.exp(np.linspace(np.log(lo), np.log(hi), G))
    e = err(q)
    zc = np.where(np.sign(e[1:]) != np.sign(e[:-1]))[0]
    edges = [lo] + [np.sqrt(q[i] * q[i + 1]) for i in zc] + [hi]
    out = []
    for a, b in zip(edges[:-1], edges[1:]):
        v = err(np.exp(np.linspace(np.log(a), np.log(b), S)))
        out.append(v[np.argmax(np.abs(v))])
    return np.array(out)


@pytest.mark.parametrize("eps,n", [(0.01, 4), (0.01, 8), (1e-3, 12), (1e-4, 16)])
def test_zolotarev_equioscillation(eps, n):
    b, c, d = oracle.zolotarev(eps, n)
    assert np.all(c > 0) and np.all(b > 0)

    def err(q):
        x = q * q
        return 1.0 - q * (b[None, :] / (x[:, None] + c[None, :])).sum(axis=1)

    e = _alternation(err, np.sqrt(eps), 1.0)
    assert len(e) == 2 * n + 1
    assert np.all(np.sign(e[1:]) == -np.sign(e[:-1]))  # alternating
    # equal size (the optimal, Chebyshev approximation), to the sampling and rounding resolution
    tol = 1e-5 + 200 * np.finfo(float).eps / d
    assert np.allclose(np.abs(e), d, rtol=tol, atol=0), (np.abs(e) / d - 1)
    # that size is delta of Eq. 4 on [eps, 1] (sqrt(x) P(x) evaluated by the oracle)
    x = np.exp(np.linspace(np.log(eps), 0.0, 4001))
    assert abs(np.max(np.abs(1 - np.sqrt(x) * oracle.rational_eval(b, c, x))) / d - 1) < 1e-3 + tol


def test_rational_sign_dense(small_case):  # noqa: F811
    dims, U, H, lam, vec = small_case
    lmax = 1.01 * np.abs(lam).max()
    psi = synth.gaussian_spinor(dims, 2)[0].reshape(-1)
    exact = vec @ (np.sign(lam) * (vec.conj().T @ psi))
    # whole spectrum inside [eps, 1]: no deflation
    eps = 0.99 * (np.abs(lam).min() / lmax) ** 2
    b, c, d = oracle.zolotarev(eps, 20)
    out = oracle.sign_rational(dims, ABC, U, -RHO, lmax, b, c, psi)
    assert rel(out, exact) < d + 1e-12
    out2 = oracle.sign_rational(dims, ABC, U, -RHO, lmax, b, c, out)
    assert rel(out2, psi) < 2 * d + 1e-12
    # deflation (Eq. 7) of the 12 lowest modes, interval above them
    order = np.argsort(np.abs(lam))
    nev = 12
    eps = 0.999 * (np.abs(lam[order[nev]]) / lmax) ** 2
    b, c, d = oracle.zolotarev(eps, 10)
    ev, eta = lam[order[:nev]], vec[:, order[:nev]].T.copy()
    out = oracle.sign_rational(dims, ABC, U, -RHO, lmax, b, c, psi, evals=ev, evecs=eta)
    assert rel(out, exact) < d + 1e-12
    # the polynomial and the rational sign agree where both are accurate
    n = int(np.ceil(np.log(1e-13 / 0.41) / (-2.0 * np.sqrt(eps)))) + 20
    poly = oracle.sign(dims, ABC, U, -RHO, lmax, eps, oracle.cheb_coeffs(eps, n), psi, ev, eta)
    assert rel(out, poly) < d + 1e-11


def test_rational_overlap_matches_dense(small_case):  # noqa: F811
    """D(m) with the rational sign against rho(1 + g5 sign) + m(1 - D/2) from the dense sign."""
    dims, U, H, lam, vec = small_case
    lmax = 1.01 * np.abs(lam).max()
    eps = 0.99 * (np.abs(lam).min() / lmax) ** 2
    b, c, d = oracle.zolotarev(eps, 20)
    V = oracle.volume(dims)
    S = vec @ np.diag(np.sign(lam)) @ vec.conj().T
    g5 = np.kron(np.eye(V), np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3)))
    Dn = np.eye(12 * V) + g5 @ S
    psi = synth.gaussian_spinor(dims, 5)[0].reshape(-1)
    for m in (0.0, 0.1):
        ref = RHO * (Dn @ psi) + m * (psi - 0.5 * (Dn @ psi))
        got = oracle.overlap_rational(dims, ABC, U, RHO, m, lmax, b, c, psi).reshape(-1)
        assert rel(got, ref) < 2 * d + 1e-12
