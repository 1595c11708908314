"""Low-mode projection c = v^dag psi (Eqs. 6-7, 9) on the tensor cores
(tcgen05, bf16 operands, FP32 accumulation) against numpy in FP64 and
against the CUDA-core engine, and the 16-bit overlap with the tensor-core
projection against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import ABC, RHO, dev, host, need_gpu, rel, torch
from test_gpu_overlap import OTOL, setup

pytestmark = pytest.mark.gpu

# bf16 operands (unit roundoff 2^-9 each) in FP32 sums: ~4e-3 per coefficient vector
TC_TOL = 2e-2


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def orthonormal(V, n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((12 * V, n)) + 1j * rng.standard_normal((12 * V, n))
    q, _ = np.linalg.qr(a)
    return np.ascontiguousarray(q.T)


@pytest.mark.parametrize("dims,nev,nrhs", [((8, 8, 8, 8), 20, 3), ((4, 4, 4, 4), 128, 1), ((8, 4, 4, 8), 37, 12)])
def test_tensor_core_projection(dims, nev, nrhs):
    from paper_1106_4964_gb300 import Context

    V = oracle.volume(dims)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(synth.unit_gauge(dims)))
    vecs = orthonormal(V, nev, 1)
    ctx.set_eigenpairs(1, np.linspace(0.1, 1.0, nev), dev(vecs))
    psi = synth.gaussian_spinor(dims, 2, nrhs=nrhs)
    exact = vecs.conj() @ psi.reshape(nrhs, -1).T  # [nev][nrhs]
    f64 = ctx.field(nrhs, "f64")
    f64.load(dev(psi))
    c0 = ctx.project_lowmodes(1, f64, engine=0)
    assert rel(c0, exact) < 1e-12
    for prec in ("f32", "f16"):
        f = ctx.field(nrhs, prec)
        f.load(dev(psi))
        c1 = ctx.project_lowmodes(1, f, engine=1)
        for r in range(nrhs):
            assert rel(c1[:, r], exact[:, r]) < TC_TOL, (prec, r, rel(c1[:, r], exact[:, r]))
        # repeated calls give identical results (fixed-order FP64 reduction of the partials)
        assert np.array_equal(c1, ctx.project_lowmodes(1, f, engine=1))


def test_overlap_16bit_with_tensor_core_projection():
    cf = setup((4, 4, 4, 4), 0.3, 1, 0.05, 100)
    # keep the 100 smallest |lambda| modes (<= 128) and put eps just below the next one
    lam = cf["lam"]
    order = np.argsort(np.abs(lam))
    nev = 100
    eps = 0.999 * (np.abs(lam[order[nev]]) / cf["lmax"]) ** 2
    n = 160
    ev = lam[order[:nev]].copy()
    eta = np.ascontiguousarray(cf["vec"][:, order[:nev]].T)
    c = oracle.cheb_coeffs(eps, n)
    psi = synth.gaussian_spinor(cf["dims"], 4)
    ref = oracle.overlap(cf["dims"], ABC, cf["U"], RHO, 0.0, cf["lmax"], eps, c, psi, ev, eta)
    from paper_1106_4964_gb300 import Context

    ctx = Context(cf["dims"], ABC)
    ctx.set_gauge(dev(cf["U"]))
    ctx.set_sign_poly(RHO, eps, n, cf["lmax"])
    ctx.set_eigenpairs(0, ev, dev(eta))
    errs = {}
    for tc in (1, 0):
        ctx.set_option("proj_tc", tc)
        for prec in ("f16", "bf16"):
            out = torch.empty_like(dev(psi))
            ctx.apply_overlap(dev(psi), out, 0.0, prec=prec)
            errs[(tc, prec)] = rel(host(out), ref)
    print("16-bit overlap errors (tensor-core projection, prec):", errs)
    for (tc, prec), e in errs.items():
        assert e <= OTOL[prec], (tc, prec, e)
