"""Pins of the oracle's Lanczos on H_w^2 (the lambda_max rescale of Eq. 5 and the low modes of
H_w that Eq. 7 deflates, Sec. V's eigensolver in its plainest form) against dense
eigendecompositions of the oracle's own H_w: exact when the Krylov space is the whole space
(2x2x2x4, dimension 384), and by values and eigen-residuals on 4^4."""
import numpy as np

import oracle
import synth
from _util import dense, rel

ABC = (1.0, 1.0, 1.0, -1.0)
RHO = 1.5


def _dense_spectrum(dims, U):
    V = oracle.volume(dims)
    H = dense(lambda v: oracle.hw(dims, ABC, U, -RHO, v), V)
    return np.linalg.eigh(H)


def test_lambda_max_whole_space_and_bound():
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 31, 0.9)
    lam, _ = _dense_spectrum(dims, U)
    top = np.abs(lam).max()
    v0 = synth.gaussian_spinor(dims, 7)[0].reshape(-1)
    full = oracle.lambda_max(dims, ABC, U, -RHO, steps=384, v0=v0)
    assert abs(full / top - 1) < 1e-10
    for steps in (10, 30, 50):
        est = oracle.lambda_max(dims, ABC, U, -RHO, steps=steps, v0=v0)
        assert est <= top * (1 + 1e-12)  # Ritz values bound the top eigenvalue from below
    assert oracle.lambda_max(dims, ABC, U, -RHO, steps=50, v0=v0) > 0.99 * top


def test_lowmodes_whole_space_exact():
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 31, 0.9)
    lam, vec = _dense_spectrum(dims, U)
    order = np.argsort(np.abs(lam))
    nev = 10
    v0 = synth.gaussian_spinor(dims, 8)[0].reshape(-1)
    vals, vecs, res = oracle.lanczos_lowmodes(dims, ABC, U, -RHO, m=384, nev=nev, v0=v0)
    assert np.allclose(vals, lam[order[:nev]], rtol=0, atol=1e-10)  # signed, sorted by |lambda|
    assert res < 1e-10
    assert np.abs(vecs.conj() @ vecs.T - np.eye(nev)).max() < 1e-12


def test_lowmodes_partial_krylov_4c4():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 1, 0.3)
    lam, _ = _dense_spectrum(dims, U)
    nev = 6
    v0 = synth.gaussian_spinor(dims, 9)[0].reshape(-1)
    vals, vecs, res = oracle.lanczos_lowmodes(dims, ABC, U, -RHO, m=600, nev=nev, v0=v0)
    exact = np.sort(np.abs(lam))[:nev]
    assert np.allclose(np.sort(np.abs(vals)), exact, rtol=1e-8, atol=0)
    for i in range(nev):
        r = oracle.hw(dims, ABC, U, -RHO, vecs[i]).reshape(-1) - vals[i] * vecs[i]
        assert np.linalg.norm(r) <= 1e-6
