"""GPU multi-mass solve (Sec. II, the paragraph after Eq. 8: one multi-shifted
CG for the propagators of several quark masses, deflated by the massless low
modes, Eq. 9) against the FP64 oracle:

* each mass's solution of D(m)^dag D(m) x = b meets the FP64 true residual
  1e-10 of the oracle's two-sign operator and agrees with the oracle's own
  multi-shifted CG (or_multimass_cg, pinned by dense solves) to the accuracy
  that the condition number allows;
* output 1 satisfies D(m) x = b and output 2, the propagator
  (1 - D/2) D(m)^-1 b, satisfies D(m) x = (1 - D/2) b (both functions of D
  commute), each checked with the oracle's D(m)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import ABC, RHO, dev, host, need_gpu, rel, torch
from test_gpu_overlap import make_ctx, setup

pytestmark = pytest.mark.gpu

MASSES = [0.02, 0.1, 0.5]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def cfg1():
    return setup((4, 4, 4, 4), 0.3, 1, 0.05, 100)


def _normal(cf, m, v):
    return oracle.overlap_normal(cf["dims"], ABC, cf["U"], RHO, m, cf["lmax"], cf["eps"], cf["c"], v, cf["ev"],
                                 cf["eta"])


def _D(cf, m, v):
    return oracle.overlap(cf["dims"], ABC, cf["U"], RHO, m, cf["lmax"], cf["eps"], cf["c"], v, cf["ev"], cf["eta"])


@pytest.mark.parametrize("inner,chiral", [("f32", 0), ("f32", 1), ("f16", 1), ("f64", 0)])
def test_multimass_normal_equations(cfg1, inner, chiral):
    cf = cfg1
    ctx = make_ctx(cf)
    ctx.set_option("chiral", chiral)
    ctx.deflate(1, 8, 1e-10)
    b = synth.point_sources(cf["dims"])[[0, 4, 8, 11]]  # both chiralities
    x = torch.empty((len(MASSES),) + b.shape, dtype=torch.complex128, device="cuda")
    infos = ctx.cg_solve_multimass(dev(b), x, MASSES, tol=1e-10, max_iter=3000, inner_prec=inner)
    xs = host(x)
    for k, m in enumerate(MASSES):
        for r in range(len(b)):
            res = rel(_normal(cf, m, xs[k, r]), b[r])
            assert res <= 1e-10, (m, r, res)
            assert infos[k]["true_residual"][r] <= 1e-10
    # the oracle's multi-shifted CG on one source (no massless deflation): same solutions up to
    # kappa x the residuals (kappa of D(m)^dag D(m) is at most (2 rho / m)^2)
    xo, it, reso = oracle.multimass_cg(cf["dims"], ABC, cf["U"], RHO, cf["lmax"], cf["eps"], cf["c"], b[0], MASSES,
                                       tol=1e-11, max_iter=3000, evals=cf["ev"], evecs=cf["eta"])
    for k, m in enumerate(MASSES):
        assert reso[k] <= 1e-10
        assert rel(xs[k, 0], xo[k]) <= (2 * RHO / m) ** 2 * 2e-10
    print(f"multimass inner={inner} chiral={chiral}: iterations {[i['iterations'] for i in infos]}, "
          f"oracle shared recursion {it}")


@pytest.mark.parametrize("output", [1, 2])
def test_multimass_inverse_and_propagator(cfg1, output):
    cf = cfg1
    ctx = make_ctx(cf)
    ctx.set_option("chiral", 1)
    ctx.deflate(1, 8, 1e-10)
    b = synth.point_sources(cf["dims"])[[1, 6]]
    x = torch.empty((len(MASSES),) + b.shape, dtype=torch.complex128, device="cuda")
    ctx.cg_solve_multimass(dev(b), x, MASSES, tol=1e-12, max_iter=4000, inner_prec="f32", output=output)
    xs = host(x)
    for k, m in enumerate(MASSES):
        for r in range(len(b)):
            lhs = _D(cf, m, xs[k, r])
            rhs = b[r] if output == 1 else b[r] - _D(cf, 0.0, b[r]) / (2 * RHO)
            err = rel(lhs, rhs)
            assert err <= 1e-9, (output, m, r, err)


def test_multimass_twelve_sources_8c4():
    """All 12 point sources and two masses in one call on 8^4 (the chiral one-sign
    recursion, 16 massless D^dag D modes deflated); every (mass, source) meets the FP64
    true residual of the oracle's operator."""
    from paper_1106_4964_gb300 import Context

    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, seed=1, s=0.5, ape_steps=3)
    eps, n, lmax = 0.005, 150, 6.6  # [eps, 1] covers this field's H_w spectrum (no H_w deflation)
    c = oracle.cheb_coeffs(eps, n)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    ctx.set_sign_poly(RHO, eps, n, lmax)
    ctx.set_option("chiral", 1)
    ctx.tune_dslash("f32", 12)
    ctx.deflate(1, 16, 1e-5)
    b = synth.point_sources(dims)
    masses = [0.05, 0.2]
    x = torch.empty((2,) + b.shape, dtype=torch.complex128, device="cuda")
    infos = ctx.cg_solve_multimass(dev(b), x, masses, tol=1e-10, max_iter=3000, inner_prec="f32")
    xs = host(x)
    worst = 0.0
    for k, m in enumerate(masses):
        for r in range(12):
            Ax = oracle.overlap_normal(dims, ABC, U, RHO, m, lmax, eps, c, xs[k, r])
            worst = max(worst, rel(Ax, b[r]))
    print(f"multimass 8^4 12 sources: iterations {[i['iterations'] for i in infos]}, worst {worst:.2e}")
    assert worst <= 1e-10
