"""Failure paths of the solver and of the bounded device waits, made on the
host side or by shortening a wait's limit (no GPU fault, trap or hang):

* a NaN in a source gives OV_ENAN;
* an iteration limit too small for the tolerance gives OV_ENOTCONV with the
  solve report filled in;
* a learned preconditioner with deliberately bad weights trips the stall rule,
  the solve falls back to plain deflated CG and still meets the FP64 residual;
* the first bounded mbarrier wait of the bulk-copy dslash, given a limit of
  zero polls, runs out: the kernel records the timeout, drains its copies with
  a wait of the full limit and writes nothing, the call returns OV_ETIMEOUT,
  and the context keeps working."""
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


def test_nan_source_gives_enan(cfg1):
    from paper_1106_4964_gb300 import OverlapError

    ctx = make_ctx(cfg1)
    b = synth.gaussian_spinor(cfg1["dims"], 2, nrhs=2)
    b[1, 0, 0, 0, 1, 2, 1] = np.nan
    with pytest.raises(OverlapError) as e:
        ctx.cg_solve(dev(b), torch.empty_like(dev(b)), mass=0.05, tol=1e-10, max_iter=100, inner_prec="f32")
    assert e.value.status == -7  # OV_ENAN


def test_iteration_limit_gives_enotconv_with_report(cfg1):
    ctx = make_ctx(cfg1)
    b = synth.gaussian_spinor(cfg1["dims"], 3, nrhs=3)
    x = torch.empty_like(dev(b))
    info = ctx.cg_solve(dev(b), x, mass=0.05, tol=1e-10, max_iter=2, inner_prec="f32", check=False)
    assert info["status"] == -4  # OV_ENOTCONV
    assert info["iterations"] == 2
    assert len(info["true_residual"]) == 3
    assert all(1e-10 < r < 1.0 for r in info["true_residual"])
    # the report is the true residual of the returned iterate, by the oracle's operator
    xs = host(x)
    cf = cfg1
    for r in range(3):
        Ax = oracle.overlap_normal(cf["dims"], ABC, cf["U"], RHO, 0.05, cf["lmax"], cf["eps"], cf["c"], xs[r],
                                   cf["ev"], cf["eta"])
        assert abs(rel(Ax, b[r]) - info["true_residual"][r]) <= 1e-8 * info["true_residual"][r] + 1e-14


def test_bad_preconditioner_falls_back(cfg1):
    cf = cfg1
    ctx = make_ctx(cf)
    rng = np.random.default_rng(5)
    w = 3.0 * (rng.standard_normal(4608) + 1j * rng.standard_normal(4608))  # a network that scrambles r
    ctx.net_set_weights(w)
    b = synth.point_sources(cf["dims"])[[0, 9]]
    x = torch.empty_like(dev(b))
    info = ctx.cg_solve(dev(b), x, mass=0.05, tol=1e-10, max_iter=2000, precond=1, inner_prec="f32")
    assert info["fallback"] == 1
    xs = host(x)
    for r in range(2):
        Ax = oracle.overlap_normal(cf["dims"], ABC, cf["U"], RHO, 0.05, cf["lmax"], cf["eps"], cf["c"], xs[r],
                                   cf["ev"], cf["eta"])
        assert rel(Ax, b[r]) <= 1e-10


@pytest.mark.parametrize("variant", [4, 5])
def test_bulk_copy_wait_timeout_is_reported(variant):
    from paper_1106_4964_gb300 import Context, OverlapError

    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 4, 0.5)
    psi = synth.gaussian_spinor(dims, 6)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    ctx.set_dslash_shape("f32", 1, 128, 1, variant)
    ctx.set_option("wait_polls", 0)
    out = torch.empty_like(dev(psi))
    with pytest.raises(OverlapError) as e:
        ctx.apply_dslash(dev(psi), out, -RHO, prec="f32")
    assert e.value.status == -6  # OV_ETIMEOUT
    ctx.set_option("wait_polls", 1 << 22)
    ctx.apply_dslash(dev(psi), out, -RHO, prec="f32")
    ref = oracle.dslash(dims, ABC, U, -RHO, psi[0])
    assert rel(host(out), ref) <= 1e-5
