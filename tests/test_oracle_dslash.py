"""Pins of the oracle's Wilson operator (Eqs. 1-2) against facts fixed by the
mathematics, not by the oracle itself: the Clifford algebra of the chiral
basis, the free-field plane-wave spectrum, gamma_5-hermiticity (Sec. II),
gauge and translation covariance, and the dense adjoint relation."""
import numpy as np
import pytest

import oracle
import synth

RHO = 1.5
ABC = (1.0, 1.0, 1.0, -1.0)  # antiperiodic in time


def grid(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return x, y, z, t


def test_gamma_algebra():
    g = [oracle.gamma(m) for m in range(5)]
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2.0 * np.eye(4) * (a == b))
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]))
    assert np.allclose(g[4], g[0] @ g[1] @ g[2] @ g[3])


@pytest.mark.parametrize("dims,bc", [((4, 4, 6, 8), ABC), ((2, 2, 2, 2), ABC), ((6, 4, 4, 4), (1, 1, 1, 1))])
def test_free_field_plane_waves(dims, bc):
    """U = 1: D_w(p) = m + sum(1 - cos p_mu) + i sum gamma_mu sin p_mu, with
    p_mu = (2 pi k + theta_mu) / L_mu, theta = pi for an antiperiodic direction."""
    U = synth.unit_gauge(dims)
    g = [oracle.gamma(m) for m in range(4)]
    x, y, z, t = grid(dims)
    rng = np.random.default_rng(7)
    m = -RHO
    for trial in range(4):
        k = [rng.integers(0, L) for L in dims]
        p = [(2 * np.pi * k[mu] + (np.pi if bc[mu] < 0 else 0.0)) / dims[mu] for mu in range(4)]
        ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = ph[..., None, None] * chi
        out = oracle.dslash(dims, bc, U, m, psi).reshape(psi.shape)
        Dp = (m + sum(1 - np.cos(q) for q in p)) * np.eye(4) + 1j * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        assert np.abs(out - ph[..., None, None] * (Dp @ chi)).max() < 1e-13


def test_gamma5_hermiticity():
    dims = (4, 4, 4, 6)
    U = synth.gauge_field(dims, 1, 0.5)
    a = synth.gaussian_spinor(dims, 2)[0]
    b = synth.gaussian_spinor(dims, 3)[0]
    ha = oracle.hw(dims, ABC, U, -RHO, a)
    hb = oracle.hw(dims, ABC, U, -RHO, b)
    lhs, rhs = np.vdot(b, ha), np.vdot(hb, a)
    assert abs(lhs - rhs) < 1e-12 * np.linalg.norm(a) * np.linalg.norm(hb)


def test_gauge_covariance():
    """D[U^g](g psi) = g D[U] psi with U^g_mu(n) = g(n) U_mu(n) g(n+mu)^dagger."""
    dims = (4, 2, 4, 6)
    U = synth.gauge_field(dims, 11, 0.8)
    g = synth.gauge_transform(dims, 5)
    psi = synth.gaussian_spinor(dims, 4)[0]
    ax = {0: 3, 1: 2, 2: 1, 3: 0}
    Ug = np.empty_like(U)
    for mu in range(4):
        gn = np.roll(g, -1, axis=ax[mu])
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gn, -1, -2))
    gpsi = np.einsum("...ab,...sb->...sa", g, psi)
    lhs = oracle.dslash(dims, ABC, Ug, -RHO, gpsi).reshape(psi.shape)
    rhs = np.einsum("...ab,...sb->...sa", g, oracle.dslash(dims, ABC, U, -RHO, psi).reshape(psi.shape))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_translation_covariance():
    dims = (4, 4, 2, 6)
    bc = (1, 1, 1, 1)
    U = synth.gauge_field(dims, 12, 0.6)
    psi = synth.gaussian_spinor(dims, 8)[0]
    ref = oracle.dslash(dims, bc, U, -RHO, psi).reshape(psi.shape)
    for axis in range(4):
        Us = np.roll(U, 1, axis=axis)
        ps = np.roll(psi, 1, axis=axis)
        out = oracle.dslash(dims, bc, Us, -RHO, ps).reshape(psi.shape)
        assert np.abs(out - np.roll(ref, 1, axis=axis)).max() < 1e-13


def dense(op, dims):
    V = oracle.volume(dims)
    N = 12 * V
    M = np.empty((N, N), dtype=np.complex128)
    e = np.zeros(N, dtype=np.complex128)
    for j in range(N):
        e[:] = 0
        e[j] = 1
        M[:, j] = op(e)
    return M


def test_dense_adjoint_2x2x2x2():
    """D_w^dagger = g5 D_w g5 on 2^4, where n + mu and n - mu are the same site."""
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, 21, 1.0)
    D = dense(lambda v: oracle.dslash(dims, ABC, U, -RHO, v), dims)
    g5 = np.kron(np.eye(16), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.abs(D.conj().T - g5 @ D @ g5).max() < 1e-14
    H = g5 @ D
    assert np.abs(H - H.conj().T).max() < 1e-14


def test_two_site_direction_sums_both_hops():
    """On L_mu = 2 the forward and backward hop reach the same neighbour; with U = 1,
    periodic bc and a field constant in space-time, D_w psi = m psi (sum of (1-g)+(1+g) = 2)."""
    dims = (2, 2, 2, 2)
    U = synth.unit_gauge(dims)
    chi = np.arange(12).reshape(4, 3) + 1j
    psi = np.broadcast_to(chi, (2, 2, 2, 2, 4, 3)).copy()
    out = oracle.dslash(dims, (1, 1, 1, 1), U, 0.3, psi).reshape(psi.shape)
    assert np.abs(out - 0.3 * psi).max() < 1e-14


def test_sampled_sites_match_full():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 1, 0.3)
    psi = synth.gaussian_spinor(dims, 2)[0]
    full = oracle.dslash(dims, ABC, U, -RHO, psi).reshape(-1, 4, 3)
    sites = np.array([0, 5, 63, 128, 255])
    assert np.abs(oracle.dslash_sites(dims, ABC, U, -RHO, psi, sites) - full[sites]).max() == 0.0
