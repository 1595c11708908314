"""Pins of the oracle's gauge-covariant network layer (the learned
preconditioner; the paper has no counterpart): the gradient against central
finite differences of the loss, and equivariance under a random SU(3) gauge
transform."""
import numpy as np

import oracle
import synth

ABC = (1.0, 1.0, 1.0, -1.0)
AX = {0: 3, 1: 2, 2: 1, 3: 0}


def rand_w(rng, cout, cin, scale=0.3):
    return scale * (rng.standard_normal((9, cout, cin, 4, 4)) + 1j * rng.standard_normal((9, cout, cin, 4, 4)))


def loss(dims, U, W1, W2, r, e):
    y = oracle.net_apply(dims, ABC, U, W1, W2, r).reshape(-1)
    return np.vdot(y - e, y - e).real / np.vdot(e, e).real


def grads(dims, U, W1, W2, r, e):
    V = oracle.volume(dims)
    h = oracle.net_layer(dims, ABC, U, W1, r.reshape(1, V, 4, 3))
    y = oracle.net_layer(dims, ABC, U, W2, h)
    gy = 2.0 * (y - e.reshape(1, V, 4, 3)) / np.vdot(e, e).real
    gh, gW2 = oracle.net_layer_grad(dims, ABC, U, W2, h, gy)
    _, gW1 = oracle.net_layer_grad(dims, ABC, U, W1, r.reshape(1, V, 4, 3), gh)
    return gW1, gW2, gh


def test_gradient_matches_finite_differences():
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 41, 0.7)
    rng = np.random.default_rng(0)
    W1 = rand_w(rng, 3, 1)
    W2 = rand_w(rng, 1, 3)
    r = synth.gaussian_spinor(dims, 1)[0].reshape(-1)
    e = synth.gaussian_spinor(dims, 2)[0].reshape(-1)
    gW1, gW2, _ = grads(dims, U, W1, W2, r, e)
    h = 1e-6
    for (W, gW, which) in ((W1, gW1, 1), (W2, gW2, 2)):
        for _ in range(12):
            idx = tuple(rng.integers(0, s) for s in W.shape)
            for d, part in ((1.0, np.real), (1j, np.imag)):
                Wp, Wm = W.copy(), W.copy()
                Wp[idx] += h * d
                Wm[idx] -= h * d
                if which == 1:
                    fd = (loss(dims, U, Wp, W2, r, e) - loss(dims, U, Wm, W2, r, e)) / (2 * h)
                else:
                    fd = (loss(dims, U, W1, Wp, r, e) - loss(dims, U, W1, Wm, r, e)) / (2 * h)
                an = part(gW[idx])
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (which, idx, fd, an)


def test_input_gradient_is_adjoint():
    """<gy, L x> = <L^dag gy, x>: the input gradient is the adjoint layer."""
    dims = (2, 2, 4, 2)
    U = synth.gauge_field(dims, 42, 0.7)
    rng = np.random.default_rng(1)
    W = rand_w(rng, 2, 3)
    V = oracle.volume(dims)
    x = rng.standard_normal((3, V, 4, 3)) + 1j * rng.standard_normal((3, V, 4, 3))
    gy = rng.standard_normal((2, V, 4, 3)) + 1j * rng.standard_normal((2, V, 4, 3))
    y = oracle.net_layer(dims, ABC, U, W, x)
    gx, _ = oracle.net_layer_grad(dims, ABC, U, W, x, gy)
    assert abs(np.vdot(gy, y) - np.vdot(gx, x)) < 1e-12 * np.linalg.norm(gy) * np.linalg.norm(y) * 10


def test_gauge_equivariance():
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, 43, 0.8)
    g = synth.gauge_transform(dims, 9)
    rng = np.random.default_rng(2)
    W1 = rand_w(rng, 4, 1)
    W2 = rand_w(rng, 1, 4)
    Ug = np.empty_like(U)
    for mu in range(4):
        gn = np.roll(g, -1, axis=AX[mu])
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gn, -1, -2))
    r = synth.gaussian_spinor(dims, 3)[0]
    gr = np.einsum("...ab,...sb->...sa", g, r)
    lhs = oracle.net_apply(dims, ABC, Ug, W1, W2, gr).reshape(r.shape)
    rhs = np.einsum("...ab,...sb->...sa", g, oracle.net_apply(dims, ABC, U, W1, W2, r).reshape(r.shape))
    assert np.abs(lhs - rhs).max() < 1e-12


def _hop(field, dims, bc, mu, step):
    """field(n + step mu_hat) on the canonical [t, z, y, x, ...] block, with the boundary
    phase bc[mu] on every value that crossed the lattice edge."""
    ax = AX[mu]
    out = np.roll(field, -step, axis=ax)
    L = dims[mu]
    edge = [slice(None)] * field.ndim
    edge[ax] = L - 1 if step > 0 else 0  # sites whose neighbour wrapped around
    out[tuple(edge)] *= bc[mu]
    return out


def test_one_hot_paths_give_single_transports():
    """W = identity spin matrix on one path and zero elsewhere makes the layer a single
    parallel transport: path 1+2mu gives U_mu(n) x(n+mu), path 2+2mu gives
    U_mu(n-mu)^dag x(n-mu), path 0 gives x.  A transposed spin matrix, swapped paths or
    a missing boundary phase all fail this (the gradient and equivariance pins do not
    see them); a non-diagonal spin matrix checks the spin index order."""
    dims = (4, 2, 2, 4)
    U = synth.gauge_field(dims, 17, 0.8)
    x = synth.gaussian_spinor(dims, 4)[0]  # [t, z, y, x, 4, 3]
    V = oracle.volume(dims)
    rng = np.random.default_rng(3)
    S = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))  # spin matrix, not symmetric
    for p in range(9):
        W = np.zeros((9, 1, 1, 4, 4), dtype=np.complex128)
        W[p, 0, 0] = S
        y = oracle.net_layer(dims, ABC, U, W, x.reshape(1, V, 4, 3))[0].reshape(x.shape)
        if p == 0:
            t = x
        else:
            mu, fwd = (p - 1) // 2, (p - 1) % 2 == 0
            if fwd:  # U_mu(n) x(n + mu)
                t = np.einsum("...ab,...sb->...sa", U[..., mu, :, :], _hop(x, dims, ABC, mu, +1))
            else:    # U_mu(n - mu)^dag x(n - mu)
                um = _hop(U[..., mu, :, :], dims, (1.0,) * 4, mu, -1)
                t = np.einsum("...ba,...sb->...sa", um.conj(), _hop(x, dims, ABC, mu, -1))
        expect = np.einsum("st,...ta->...sa", S, t)
        assert np.abs(y - expect).max() < 1e-13, p
