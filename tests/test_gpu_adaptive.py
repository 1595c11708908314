"""Adaptive-precision CG (Sec. V, propagator paragraph: the adaptive CG that the
paper finds 60 % faster): the inner operator of the mixed-precision CG uses a
lower-degree sign polynomial whose delta (Eq. 4) meets a looser target, while
every true residual and reliable update keeps the full polynomial.

* the inner degree the library selects is the lowest one whose delta, by the
  oracle's own evaluation of Eq. 4, meets the target;
* the adaptive solve meets the FP64 true residual 1e-10 of the oracle's
  full-degree D(m)^dag D(m), single- and multi-mass, and needs far fewer
  dslash applications than the non-adaptive solve."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import ABC, RHO, dev, host, need_gpu, rel, torch
from test_gpu_overlap import make_ctx, setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.fixture(scope="module")
def cfg1():
    return setup((4, 4, 4, 4), 0.3, 1, 0.05, 100)


@pytest.mark.parametrize("target", [1e-2, 1e-4, 1e-7])
def test_inner_degree_is_lowest_meeting_delta(cfg1, target):
    ctx = make_ctx(cfg1)
    assert ctx.get_option("adaptive_degree") == cfg1["n"]  # off: the full degree
    ctx.set_option("adaptive_delta", target)
    n_in = int(ctx.get_option("adaptive_degree"))
    eps = cfg1["eps"]
    assert 1 <= n_in < cfg1["n"]
    d_in = oracle.poly_delta(oracle.cheb_coeffs(eps, n_in), eps)
    d_below = oracle.poly_delta(oracle.cheb_coeffs(eps, n_in - 1), eps)
    print(f"target {target:g}: inner degree {n_in}, delta {d_in:.3e} (degree {n_in - 1}: {d_below:.3e})")
    assert d_in <= 1.05 * target
    assert d_below > 0.95 * target


@pytest.mark.parametrize("chiral", [0, 1])
def test_adaptive_cg_meets_full_residual(cfg1, chiral):
    cf = cfg1
    b = synth.point_sources(cf["dims"])[[0, 2, 7, 10]]
    runs = {}
    for adaptive in (0.0, 1e-4):
        ctx = make_ctx(cf)
        ctx.set_option("chiral", chiral)
        ctx.set_option("adaptive_delta", adaptive)
        ctx.deflate(1, 8, 1e-10)
        x = torch.empty_like(dev(b))
        n0 = ctx.dslash_count()
        info = ctx.cg_solve(dev(b), x, mass=0.05, tol=1e-10, max_iter=3000, inner_prec="f32")
        runs[adaptive] = (host(x), info, ctx.dslash_count() - n0)
    xs, info, launches = runs[1e-4]
    for r in range(len(b)):
        Ax = oracle.overlap_normal(cf["dims"], ABC, cf["U"], RHO, 0.05, cf["lmax"], cf["eps"], cf["c"], xs[r],
                                   cf["ev"], cf["eta"])
        assert rel(Ax, b[r]) <= 1e-10
    print(f"adaptive cg chiral={chiral}: iterations {info['iterations']} vs {runs[0.0][1]['iterations']}, "
          f"dslash launches {launches} vs {runs[0.0][2]}")
    assert launches < 0.6 * runs[0.0][2]


def test_adaptive_multimass(cfg1):
    cf = cfg1
    ctx = make_ctx(cf)
    ctx.set_option("chiral", 1)
    ctx.set_option("adaptive_delta", 1e-4)
    ctx.deflate(1, 8, 1e-10)
    b = synth.point_sources(cf["dims"])[[3, 9]]
    masses = [0.03, 0.3]
    x = torch.empty((2,) + b.shape, dtype=torch.complex128, device="cuda")
    ctx.cg_solve_multimass(dev(b), x, masses, tol=1e-10, max_iter=3000, inner_prec="f32")
    xs = host(x)
    for k, m in enumerate(masses):
        for r in range(2):
            Ax = oracle.overlap_normal(cf["dims"], ABC, cf["U"], RHO, m, cf["lmax"], cf["eps"], cf["c"], xs[k, r],
                                       cf["ev"], cf["eta"])
            assert rel(Ax, b[r]) <= 1e-10
