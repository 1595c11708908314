"""The GPU's lambda_max estimate (Eq. 5 rescale) and low H_w modes (Eq. 7, Sec. V eigensolver)
against the oracle's own Lanczos on H_w^2 (pinned by dense eigendecompositions) on a lattice
too large for a dense eigendecomposition in the test."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import ABC, RHO, dev, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def lat():
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, seed=3, s=0.5, ape_steps=3)
    return dims, U


def test_lambda_max_matches_oracle_lanczos(lat):
    from paper_1106_4964_gb300 import Context

    dims, U = lat
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    ctx.set_sign_poly(RHO, 0.05, 10, 0.0)
    gpu = ctx.get_sign_poly()["lambda_max"] / 1.01
    v0 = synth.gaussian_spinor(dims, 11)[0].reshape(-1)
    ora = oracle.lambda_max(dims, ABC, U, -RHO, steps=50, v0=v0)
    top = oracle.lambda_max(dims, ABC, U, -RHO, steps=300, v0=v0)  # converged top of the spectrum
    print(f"lambda_max: GPU {gpu:.6f}, oracle 50 steps {ora:.6f}, oracle 300 steps {top:.6f}")
    assert gpu <= top * (1 + 1e-9) and ora <= top * (1 + 1e-9)
    assert abs(gpu / top - 1) < 2e-3 and abs(ora / top - 1) < 2e-3


def test_low_modes_match_oracle_lanczos(lat):
    from paper_1106_4964_gb300 import Context

    dims, U = lat
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    ctx.set_sign_poly(RHO, 0.05, 10, 0.0)
    lmax = ctx.get_sign_poly()["lambda_max"]
    nev = 8
    ctx.deflate(0, nev, 1e-10)
    vals, vecs = ctx.get_eigenpairs(0)
    v0 = synth.gaussian_spinor(dims, 12)[0].reshape(-1)
    ov, oe, ores = oracle.lanczos_lowmodes(dims, ABC, U, -RHO, m=700, nev=nev + 4, v0=v0)
    print(f"low modes: GPU {vals}, oracle {ov[:nev]}, oracle residual {ores:.2e}")
    # the oracle's own pairs: eigen-residual r <= 1e-6 lambda_max, so its eigenvalues are exact to
    # r^2 / gap (Hermitian) and its vectors to r / gap
    assert ores < 1e-6 * lmax
    # the same |lambda| spectrum, and every signed GPU eigenvalue is one of the oracle's (a +-lambda pair
    # at the edge of the nev modes may contribute either member)
    assert np.allclose(np.sort(np.abs(vals)), np.sort(np.abs(ov))[:nev], rtol=0, atol=1e-9 * lmax)
    for v in vals:
        assert np.min(np.abs(ov - v)) < 1e-9 * lmax
    # each GPU vector lies in the oracle's eigenspace of its eigenvalue
    for i in range(nev):
        same = np.abs(ov - vals[i]) < 1e-7 * lmax
        P = oe[same]
        proj = P.conj() @ vecs[i]
        assert abs(np.linalg.norm(proj) - 1) < 1e-6
