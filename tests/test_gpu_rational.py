"""Rational sign function on the GPU (Sec. V, Eq. 12: P(Q^2) = sum_i b_i (Q^2 + c_i)^-1
with Zolotarev's coefficients, the shifted inverses by one multi-shift CG, single- and
double-pass) against the FP64 oracle's rational overlap (pinned by dense
eigendecompositions and the equioscillation of its coefficients)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import ABC, RHO, dev, host, need_gpu, rel, torch
from test_gpu_overlap import setup

pytestmark = pytest.mark.gpu

NPOLES = 6  # delta ~ 1e-8 on [0.05, 1]: large enough to compare the two coefficient generators' delta
RTOL = {"f64": 1e-10, "df64": 1e-10, "f32": 1e-5, "f16": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def cfg1():
    return setup((4, 4, 4, 4), 0.3, 1, 0.05, 100)


def _ctx(cf, npass, npoles=NPOLES):
    from paper_1106_4964_gb300 import Context

    ctx = Context(cf["dims"], ABC)
    ctx.set_gauge(dev(cf["U"]))
    ctx.set_sign_rational(RHO, cf["eps"], npoles, cf["lmax"])
    ctx.set_eigenpairs(0, cf["ev"], dev(cf["eta"]))
    ctx.set_option("rational_pass", npass)
    ctx.set_option("rational_tol", 1e-13)
    return ctx


def test_coefficients_match_oracle(cfg1):
    ctx = _ctx(cfg1, 2)
    b, c, d = ctx.get_sign_rational()
    bo, co, do = oracle.zolotarev(cfg1["eps"], NPOLES)
    assert rel(c, co) < 1e-12 and rel(b, bo) < 1e-10 and abs(d / do - 1) < 1e-6
    assert 1e-12 < d < 1e-6


@pytest.mark.parametrize("npass", [1, 2])
@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16"])
def test_rational_overlap_parity(cfg1, npass, prec):
    cf = cfg1
    bo, co, do = oracle.zolotarev(cf["eps"], NPOLES)
    psi = synth.gaussian_spinor(cf["dims"], 2, nrhs=2)
    ctx = _ctx(cf, npass)
    out = torch.empty_like(dev(psi))
    n0 = ctx.dslash_count()
    ctx.apply_overlap(dev(psi), out, 0.1, prec=prec)
    launches = ctx.dslash_count() - n0
    iters = ctx.get_option("rational_iterations")
    got = host(out)
    for r in range(2):
        ref = oracle.overlap_rational(cf["dims"], ABC, cf["U"], RHO, 0.1, cf["lmax"], bo, co, psi[r], tol=1e-14,
                                      evals=cf["ev"], evecs=cf["eta"])
        err = rel(got[r], ref)
        assert err <= RTOL[prec], (npass, prec, r, err)
    # one H_w^2 (two launches) per CG iteration, twice over for the double pass, plus the final D_w
    assert launches == 2 * npass * iters + 1
    print(f"rational overlap {prec} pass {npass}: {int(iters)} CG iterations, {launches} dslash launches")


def test_rational_matches_polynomial_sign(cfg1):
    """Where both approximations are accurate (delta ~ 1e-14 each: 12 poles, degree 100) the rational
    and the polynomial overlap operators agree on the GPU."""
    cf = cfg1
    psi = synth.gaussian_spinor(cf["dims"], 3)
    ctx = _ctx(cf, 2, npoles=12)
    out_r = torch.empty_like(dev(psi))
    ctx.apply_overlap(dev(psi), out_r, 0.0, prec="f64")
    ctx.set_sign_poly(RHO, cf["eps"], cf["n"], cf["lmax"])
    out_p = torch.empty_like(dev(psi))
    ctx.apply_overlap(dev(psi), out_p, 0.0, prec="f64")
    assert rel(host(out_r), host(out_p)) < 1e-10


def test_cg_with_rational_sign(cfg1):
    """The deflated mixed-precision CG runs unchanged on the rational operator and meets the
    oracle's true residual of the rational D(m)^dag D(m)."""
    cf = cfg1
    bo, co, do = oracle.zolotarev(cf["eps"], NPOLES)
    ctx = _ctx(cf, 2)
    b = synth.point_sources(cf["dims"])[[0, 8]]
    x = torch.empty_like(dev(b))
    ctx.cg_solve(dev(b), x, mass=0.1, tol=1e-10, max_iter=2000, inner_prec="f32")
    xs = host(x)
    for r in range(2):
        t = oracle.overlap_rational(cf["dims"], ABC, cf["U"], RHO, 0.1, cf["lmax"], bo, co, xs[r], tol=1e-14,
                                    evals=cf["ev"], evecs=cf["eta"])
        g5 = oracle.gamma5(t)
        Ax = oracle.gamma5(oracle.overlap_rational(cf["dims"], ABC, cf["U"], RHO, 0.1, cf["lmax"], bo, co, g5,
                                                   tol=1e-14, evals=cf["ev"], evecs=cf["eta"]))
        assert rel(Ax, b[r]) <= 1e-10
