"""Pins of the oracle's polynomial (Eq. 4, Eq. 11), deflated sign function
(Eqs. 5-7) and overlap operator (Eqs. 3, 8): numpy's independent Chebyshev
interpolant, the paper's printed order/accuracy numbers, the geometric
convergence rate fixed by the singularity of x^{-1/2}, a dense
eigendecomposition sign, the free-field closed form, sign^2 = 1, the
Ginsparg-Wilson relation and the circle spectrum."""
import os

import numpy as np
import pytest

import oracle
import synth
from _util import dense, g5_dense, rel, grid, free_momenta

RHO = 1.5
ABC = (1.0, 1.0, 1.0, -1.0)
GOLD = os.path.join(os.path.dirname(__file__), "golden", "eq11_triples.txt")


def load_triples():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        d, n, se = line.split()[:3]
        rows.append((float(d), float(n), float(se)))
    return rows


# ---------------------------------------------------------------- polynomial
def test_interpolates_at_chebyshev_nodes():
    eps, n = 0.05, 40
    c = oracle.cheb_coeffs(eps, n)
    th = np.pi * (np.arange(n + 1) + 0.5) / (n + 1)
    x = 0.5 * (1 + eps) + 0.5 * (1 - eps) * np.cos(th)
    assert np.abs(oracle.poly_eval(c, eps, x) * np.sqrt(x) - 1).max() < 1e-13


def test_matches_numpy_chebyshev_interpolant():
    for eps, n in ((0.05, 30), (0.01, 100)):
        c = oracle.cheb_coeffs(eps, n)
        f = np.polynomial.chebyshev.Chebyshev.interpolate(lambda x: x ** -0.5, n, domain=[eps, 1])
        assert np.abs(f.coef - c).max() < 1e-12


def test_geometric_rate_from_singularity():
    """x^{-1/2} is singular at x = 0, i.e. y = -(1+eps)/(1-eps): the interpolation
    error decays like rho^-n with rho = (1 + sqrt eps)/(1 - sqrt eps)."""
    eps = 0.01
    ns = np.arange(60, 121, 10)
    d = [oracle.poly_delta(oracle.cheb_coeffs(eps, int(n)), eps, 20000) for n in ns]
    slope = np.polyfit(ns, np.log(d), 1)[0]
    theory = -np.log((1 + np.sqrt(eps)) / (1 - np.sqrt(eps)))
    assert abs(slope / theory - 1) < 0.05


def test_paper_triples_follow_eq11():
    """The orders printed in Sec. II (given as "n ~ ...") follow the paper's own rule
    (Eq. 11): n = ln(A / delta) / (b sqrt(eps)) to within 25 %."""
    for delta, n, se in load_triples():
        n_pred = np.log(0.41 / delta) / (2.1 * se)
        assert abs(n_pred / n - 1) < 0.25, (delta, n, se, n_pred)


@pytest.mark.parametrize("eps", [0.04, 0.01, 0.0025])
def test_interpolant_close_to_eq11(eps):
    """Eq. 11 describes the optimal polynomial; the Chebyshev interpolant used here is
    within a small factor of it wherever delta is above the FP64 rounding floor."""
    se = np.sqrt(eps)
    for n in (20, 40, 60, 80, 120):
        d = oracle.poly_delta(oracle.cheb_coeffs(eps, n), eps, 20000)
        pred = 0.41 * np.exp(-2.1 * n * se)
        if pred < 1e-11:
            continue
        assert 0.5 < d / pred < 3.0, (eps, n, d, pred)


# ---------------------------------------------------------------- sign function
def dense_hw(dims, U):
    V = oracle.volume(dims)
    return dense(lambda v: oracle.hw(dims, ABC, U, -RHO, v), V)


@pytest.fixture(scope="module")
def small_case():
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 31, 0.9)
    H = dense_hw(dims, U)
    lam, vec = np.linalg.eigh(H)
    return dims, U, H, lam, vec


def test_sign_dense_eig_with_deflation(small_case):
    dims, U, H, lam, vec = small_case
    V = oracle.volume(dims)
    order = np.argsort(np.abs(lam))
    nev = 12
    lmax = 1.01 * np.abs(lam).max()
    eps = 0.999 * (np.abs(lam[order[nev]]) / lmax) ** 2
    n = int(np.ceil(np.log(1e-13 / 0.41) / (-2.0 * np.sqrt(eps)))) + 20
    c = oracle.cheb_coeffs(eps, n)
    ev = lam[order[:nev]]
    eta = vec[:, order[:nev]].T.copy()
    psi = synth.gaussian_spinor(dims, 2)[0].reshape(-1)
    out = oracle.sign(dims, ABC, U, -RHO, lmax, eps, c, psi, ev, eta)
    exact = vec @ (np.sign(lam) * (vec.conj().T @ psi))
    assert rel(out, exact) < 1e-11
    # sign^2 = 1
    out2 = oracle.sign(dims, ABC, U, -RHO, lmax, eps, c, out, ev, eta)
    assert rel(out2, psi) < 1e-11
    # without deflation the low modes are approximated poorly (Sec. II, Fig. 2)
    bad = oracle.sign(dims, ABC, U, -RHO, lmax, eps, c, psi)
    assert rel(bad, exact) > 1e-6


def test_sign_dense_eig_no_deflation(small_case):
    dims, U, H, lam, vec = small_case
    lmax = 1.01 * np.abs(lam).max()
    eps = 0.99 * (np.abs(lam).min() / lmax) ** 2
    n = int(np.ceil(np.log(1e-13 / 0.41) / (-2.0 * np.sqrt(eps)))) + 20
    c = oracle.cheb_coeffs(eps, n)
    psi = synth.gaussian_spinor(dims, 3)[0].reshape(-1)
    out = oracle.sign(dims, ABC, U, -RHO, lmax, eps, c, psi)
    exact = vec @ (np.sign(lam) * (vec.conj().T @ psi))
    assert rel(out, exact) < 1e-11


def free_spectrum(dims, bc, m):
    g = [oracle.gamma(k) for k in range(4)]
    ps = free_momenta(dims, bc)
    P = np.meshgrid(*ps, indexing="ij")
    A = m + sum(1 - np.cos(p) for p in P)
    s2 = sum(np.sin(p) ** 2 for p in P)
    return A, s2


def test_sign_free_field_closed_form():
    """U = 1: H_w^2 = A^2 + s^2, so gamma_5 sign(H_w) = D_w(p) / sqrt(A^2 + s^2)."""
    dims = (4, 4, 4, 4)
    U = synth.unit_gauge(dims)
    A, s2 = free_spectrum(dims, ABC, -RHO)
    lmax = 1.01 * np.sqrt((A ** 2 + s2).max())
    eps, n = 0.01, 200
    assert (A ** 2 + s2).min() / lmax ** 2 > eps
    c = oracle.cheb_coeffs(eps, n)
    g = [oracle.gamma(k) for k in range(4)]
    x, y, z, t = grid(dims)
    rng = np.random.default_rng(3)
    for _ in range(3):
        k = [rng.integers(0, 4) for _ in range(4)]
        p = [(2 * np.pi * k[mu] + (np.pi if ABC[mu] < 0 else 0)) / 4 for mu in range(4)]
        ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = ph[..., None, None] * chi
        Ap = -RHO + sum(1 - np.cos(q) for q in p)
        Dp = Ap * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        norm = np.sqrt(Ap ** 2 + sum(np.sin(q) ** 2 for q in p))
        out = oracle.gamma5(oracle.sign(dims, ABC, U, -RHO, lmax, eps, c, psi)).reshape(psi.shape)
        assert np.abs(out - ph[..., None, None] * (Dp @ chi) / norm).max() < 1e-12
        # overlap, Eq. 3 scaled by rho: rho (1 + D_w(p)/|D_w(p)|)
        ov = oracle.overlap(dims, ABC, U, RHO, 0.0, lmax, eps, c, psi).reshape(psi.shape)
        exp = ph[..., None, None] * (RHO * (chi + (Dp @ chi) / norm))
        assert np.abs(ov - exp).max() < 1e-12


# ---------------------------------------------------------------- overlap
@pytest.fixture(scope="module")
def dense_overlap(small_case):
    dims, U, H, lam, vec = small_case
    V = oracle.volume(dims)
    order = np.argsort(np.abs(lam))
    nev = 12
    lmax = 1.01 * np.abs(lam).max()
    eps = 0.999 * (np.abs(lam[order[nev]]) / lmax) ** 2
    n = int(np.ceil(np.log(1e-13 / 0.41) / (-2.0 * np.sqrt(eps)))) + 20
    c = oracle.cheb_coeffs(eps, n)
    ev = lam[order[:nev]]
    eta = vec[:, order[:nev]].T.copy()
    D = dense(lambda v: oracle.overlap(dims, ABC, U, RHO, 0.0, lmax, eps, c, v, ev, eta), V)
    return dims, U, D, (lmax, eps, c, ev, eta)


def test_ginsparg_wilson(dense_overlap):
    dims, U, D, _ = dense_overlap
    g5 = g5_dense(oracle.volume(dims))
    lhs = g5 @ D + D @ g5
    rhs = D @ g5 @ D / RHO
    assert np.abs(lhs - rhs).max() < 1e-10


def test_spectrum_on_circle(dense_overlap):
    dims, U, D, _ = dense_overlap
    d = np.linalg.eigvals(D)
    assert np.abs(np.abs(d - RHO) - RHO).max() < 1e-10


def test_normal_operator_identity(dense_overlap):
    """D^dag D = rho (D + D^dag) for the exact sign; gamma_5 commutes with D^dag D."""
    dims, U, D, _ = dense_overlap
    g5 = g5_dense(oracle.volume(dims))
    DD = D.conj().T @ D
    assert np.abs(DD - RHO * (D + D.conj().T)).max() < 1e-10
    assert np.abs(g5 @ DD - DD @ g5).max() < 1e-10
    # gamma_5-hermiticity of the overlap
    assert np.abs(D.conj().T - g5 @ D @ g5).max() < 1e-10


@pytest.mark.parametrize("m", [0.0, 0.07])
def test_chiral_sector_normal_operator(dense_overlap, m):
    """On a chiral sector (gamma5 = chi) the normal operator needs one sign application:
    P D(m)^dag D(m) P = m^2 P + (rho^2 - m^2/4)/rho (1 + chi gamma5) D(0) P, P = (1 + chi gamma5)/2,
    a consequence of sign^2 = 1 (the chiral basis of Sec. V).  The oracle's two-sign D^dag D
    and its one-sign D(0) are compared on random vectors of each sector."""
    dims, U, D, (lmax, eps, c, ev, eta) = dense_overlap
    psi = synth.gaussian_spinor(dims, 8)[0]
    for chi in (+1, -1):
        ph = psi.copy()
        ph[..., (2, 3) if chi > 0 else (0, 1), :] = 0  # project onto the sector
        ph = ph.reshape(-1)
        lhs = oracle.overlap_normal(dims, ABC, U, RHO, m, lmax, eps, c, ph, ev, eta)
        u = oracle.overlap(dims, ABC, U, RHO, 0.0, lmax, eps, c, ph, ev, eta)
        cm = (RHO ** 2 - m * m / 4) / RHO
        rhs = m * m * ph + cm * (u + chi * oracle.gamma5(u).reshape(-1))
        assert rel(rhs, lhs) < 1e-12


def test_massive_overlap_eq8(dense_overlap):
    """D(m) = rho D + m (1 - D/2): affine in m with the massless operator (D = D(0)/rho)."""
    dims, U, D, (lmax, eps, c, ev, eta) = dense_overlap
    psi = synth.gaussian_spinor(dims, 5)[0].reshape(-1)
    m = 0.07
    out = oracle.overlap(dims, ABC, U, RHO, m, lmax, eps, c, psi, ev, eta)
    D0 = D / RHO
    assert rel(out, RHO * D0 @ psi + m * (psi - 0.5 * D0 @ psi)) < 1e-12


def test_cg_dense_solve(dense_overlap):
    """Deflated CG on D(m)^dag D(m) against a dense linear solve."""
    dims, U, D, (lmax, eps, c, ev, eta) = dense_overlap
    V = oracle.volume(dims)
    m = 0.05
    Dm = (RHO - m / 2) * (D / RHO) + m * np.eye(12 * V)
    A = Dm.conj().T @ Dm
    b = synth.gaussian_spinor(dims, 6)[0].reshape(-1)
    xref = np.linalg.solve(A, b)
    # deflation basis: 10 lowest eigenpairs of A from a dense Hermitian eig
    mu, xi = np.linalg.eigh(0.5 * (A + A.conj().T))
    for nev2 in (0, 10):
        x, it, res = oracle.cg(dims, ABC, U, RHO, m, lmax, eps, c, b, tol=1e-12, max_iter=500,
                               evals=ev, evecs=eta, mu=mu[:nev2] if nev2 else None,
                               xi=xi[:, :nev2].T.copy() if nev2 else None)
        assert it > 0 and res <= 1e-12
        assert rel(x, xref) < 1e-9
        if nev2:
            assert it < it_plain
        else:
            it_plain = it


def test_cg_deflated_guess_is_exact_in_span(dense_overlap):
    """A right-hand side inside span(xi) is solved exactly by the deflated guess (0 iterations)."""
    dims, U, D, (lmax, eps, c, ev, eta) = dense_overlap
    A = D.conj().T @ D
    mu, xi = np.linalg.eigh(0.5 * (A + A.conj().T))
    b = xi[:, :4] @ np.array([1.0, -2.0, 0.5j, 1 + 1j])
    x, it, res = oracle.cg(dims, ABC, U, RHO, 0.0, lmax, eps, c, b, tol=1e-10, max_iter=50,
                           evals=ev, evecs=eta, mu=mu[:8], xi=xi[:, :8].T.copy())
    assert it == 0 and res < 1e-10


def test_cg_with_approximate_eigenvectors(dense_overlap):
    """Deflation with eigenvectors perturbed at 1e-5 still reaches the dense solution: the
    low part is re-solved on every cycle's true residual (Eq. 9 applied to the residual)."""
    dims, U, D, (lmax, eps, c, ev, eta) = dense_overlap
    V = oracle.volume(dims)
    m = 0.05
    Dm = (RHO - m / 2) * (D / RHO) + m * np.eye(12 * V)
    A = Dm.conj().T @ Dm
    b = synth.gaussian_spinor(dims, 8)[0].reshape(-1)
    mu, xi = np.linalg.eigh(0.5 * (A + A.conj().T))
    rng = np.random.default_rng(5)
    xp = xi[:, :10] + 1e-5 * (rng.standard_normal((12 * V, 10)) + 1j * rng.standard_normal((12 * V, 10)))
    xp, _ = np.linalg.qr(xp)
    mup = np.real(np.einsum("ki,kl,li->i", xp.conj(), A, xp))
    x, it, res = oracle.cg(dims, ABC, U, RHO, m, lmax, eps, c, b, tol=1e-12, max_iter=800, evals=ev, evecs=eta,
                           mu=mup, xi=xp.T.copy())
    assert it > 0 and res <= 1e-12
    assert rel(x, np.linalg.solve(A, b)) < 1e-9


def test_chiral_sector_cg_needs_the_sector_projection(dense_overlap):
    """The reliable-update recursion with the one-sign chiral-sector operator (reading of Sec. V's
    chiral structure): with the inner residual projected onto the source's sector at every true
    residual it reaches the full operator's 1e-10; without the projection, rounding-level
    components in the other sector (where the one-sign form acts as m^2 and couples back) grow
    every cycle.  Dense oracle operators, inner arithmetic in single precision."""
    dims, U, D, (lmax, eps, c, ev, eta) = dense_overlap
    V = oracle.volume(dims)
    m = 0.05
    D0 = D  # rho (1 + gamma5 sign), the massless overlap
    Dm = (RHO - m / 2) * (D0 / RHO) + m * np.eye(12 * V)
    N = Dm.conj().T @ Dm
    g5 = np.diag(g5_dense(V)).real
    b = synth.point_sources(dims)[4].reshape(-1)  # spin 1: gamma5 = +1
    cm = (RHO ** 2 - m * m / 4) / RHO
    A = m * m * np.eye(12 * V) + cm * (D0 + g5[:, None] * D0)

    def solve(project):
        x = np.zeros_like(b)
        bn = np.linalg.norm(b)
        r = b.copy()
        rs = r.astype(np.complex64)
        xs = np.zeros_like(rs)
        p = rs.copy()
        rr = np.vdot(rs, rs).real
        rmax = np.sqrt(rr)
        for _ in range(200):
            q = (A @ p.astype(np.complex128)).astype(np.complex64)
            a = rr / np.vdot(p, q).real
            xs += a * p
            rs -= a * q
            rn = np.vdot(rs, rs).real
            if np.sqrt(rn) < 0.1 * rmax:
                x = x + xs.astype(np.complex128)
                xs[:] = 0
                r = b - N @ x
                if np.linalg.norm(r) <= 1e-10 * bn:
                    return np.linalg.norm(r) / bn
                rs = r.astype(np.complex64)
                if project:
                    rs[g5 < 0] = 0
                rn = np.vdot(rs, rs).real
                rmax = np.sqrt(rn)
            p = rs + (rn / rr) * p
            rr = rn
        return np.linalg.norm(b - N @ (x + xs.astype(np.complex128))) / bn

    assert solve(True) <= 1e-10


@pytest.mark.parametrize("ndefl", [0, 8])
def test_multimass_cg_dense(dense_overlap, ndefl):
    """One multi-shifted CG for several masses (Sec. II) against dense solves of each
    D(m)^dag D(m) x = b, with and without the massless low modes deflated (Eq. 9); the
    shared Krylov space rests on D(m)^dag D(m) = a_m (D^dag D + m^2 / a_m), a_m = 1 - m^2/(4 rho^2)."""
    dims, U, D, (lmax, eps, c, ev, eta) = dense_overlap
    V = oracle.volume(dims)
    b = synth.gaussian_spinor(dims, 11)[0].reshape(-1)
    masses = np.array([0.02, 0.1, 0.5])
    mu = xi = None
    if ndefl:
        DD = D.conj().T @ D
        w, v = np.linalg.eigh(0.5 * (DD + DD.conj().T))
        mu, xi = w[:ndefl], np.ascontiguousarray(v[:, :ndefl].T)
    x, it, res = oracle.multimass_cg(dims, ABC, U, RHO, lmax, eps, c, b, masses, tol=1e-11, max_iter=2000,
                                     evals=ev, evecs=eta, mu=mu, xi=xi)
    assert it > 0
    for k, m in enumerate(masses):
        Dm = (RHO - m / 2) * (D / RHO) + m * np.eye(12 * V)
        ref = np.linalg.solve(Dm.conj().T @ Dm, b)
        assert res[k] <= 1e-10
        assert rel(x[k].reshape(-1), ref) < 1e-8


def test_multimass_matches_single_mass_cg(dense_overlap):
    """Each mass of the multi-shifted solve agrees with the single-mass deflated CG of Eq. 9."""
    dims, U, D, (lmax, eps, c, ev, eta) = dense_overlap
    b = synth.gaussian_spinor(dims, 12)[0]
    masses = [0.05, 0.2]
    x, it, res = oracle.multimass_cg(dims, ABC, U, RHO, lmax, eps, c, b, masses, tol=1e-12, max_iter=3000,
                                     evals=ev, evecs=eta)
    for k, m in enumerate(masses):
        xs, its, rs = oracle.cg(dims, ABC, U, RHO, m, lmax, eps, c, b, tol=1e-12, max_iter=3000, evals=ev,
                                evecs=eta)
        assert rs <= 1e-12 and res[k] <= 1e-11
        assert rel(x[k], xs) < 1e-9
        if k == 0:
            assert it <= its + 5  # the lightest mass sets the iteration count of the shared recursion
