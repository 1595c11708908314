"""GPU parity of the even/odd dslash and H_w (Eqs. 1-2) against the FP64 oracle,
through the C ABI: several lattices (including a ragged last block and
L = 2 directions), all storage precisions, multi-RHS, host and device
buffers, the internal-field path, and sampled sites of the full 24^3 x 64
workload in the benchmark's launch configuration."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import ABC, RHO, TOL, dev, host, need_gpu, rel, torch

pytestmark = pytest.mark.gpu

DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 4, 6, 8), (6, 4, 4, 6), (8, 8, 8, 8), (2, 6, 4, 10)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16", "df64"])
def test_dslash_parity(dims, prec):
    from paper_1106_4964_gb300 import Context

    U = synth.gauge_field(dims, 1, 0.5)
    psi = synth.gaussian_spinor(dims, 2)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    out = torch.empty_like(dev(psi))
    ctx.apply_dslash(dev(psi), out, -RHO, prec=prec)
    ref = oracle.dslash(dims, ABC, U, -RHO, psi)
    err = rel(host(out), ref)
    print(f"dslash {dims} {prec}: rel err {err:.3e}")
    assert err <= TOL[prec]
    ctx.apply_Hw(dev(psi), out, -RHO, prec=prec)
    err = rel(host(out), oracle.hw(dims, ABC, U, -RHO, psi))
    assert err <= TOL[prec]


@pytest.mark.parametrize("prec,nrhs", [("f64", 3), ("f32", 12), ("f16", 5), ("f64", 12), ("df64", 7)])
def test_multi_rhs(prec, nrhs):
    from paper_1106_4964_gb300 import Context

    dims = (4, 4, 4, 6)
    U = synth.gauge_field(dims, 3, 0.5)
    psi = synth.gaussian_spinor(dims, 4, nrhs=nrhs)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    out = torch.empty_like(dev(psi))
    ctx.apply_dslash(dev(psi), out, 0.1, prec=prec)
    got = host(out)
    for r in range(nrhs):
        assert rel(got[r], oracle.dslash(dims, ABC, U, 0.1, psi[r])) <= TOL[prec]


def test_host_buffers_and_periodic_bc():
    from paper_1106_4964_gb300 import Context

    dims, bc = (4, 2, 4, 4), (1.0, 1.0, 1.0, 1.0)
    U = synth.gauge_field(dims, 5, 0.5)
    psi = synth.gaussian_spinor(dims, 6)
    ctx = Context(dims, bc)
    ctx.set_gauge(U)  # host numpy buffer
    out = np.empty_like(psi)
    ctx.apply_dslash(psi, out, -RHO, prec="f64")
    assert rel(out, oracle.dslash(dims, bc, U, -RHO, psi)) <= 1e-12


def test_field_path_matches_canonical():
    from paper_1106_4964_gb300 import Context

    dims = (6, 4, 4, 6)
    U = synth.gauge_field(dims, 7, 0.5)
    psi = synth.gaussian_spinor(dims, 8, nrhs=2)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    for prec in ("f64", "f32", "f16"):
        fi, fo = ctx.field(2, prec), ctx.field(2, prec)
        fi.load(dev(psi))
        ctx.dslash_field(fi, fo, -RHO, gamma5=True)
        out = torch.empty_like(dev(psi))
        fo.store(out)
        ref = np.stack([oracle.hw(dims, ABC, U, -RHO, psi[r]) for r in range(2)])
        assert rel(host(out), ref) <= TOL[prec]


def test_rejects_non_su3_gauge():
    from paper_1106_4964_gb300 import Context, OverlapError

    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 1, 0.3)
    U[1, 2, 3, 0, 2] *= 1.001
    ctx = Context(dims, ABC)
    with pytest.raises(OverlapError) as e:
        ctx.set_gauge(dev(U))
    assert "SU(3)" in str(e.value)


def test_bad_arguments():
    from paper_1106_4964_gb300 import Context, OverlapError

    with pytest.raises(OverlapError):
        Context((3, 4, 4, 4))
    ctx = Context((4, 4, 4, 4))
    x = torch.zeros((1, 4, 4, 4, 4, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(OverlapError):  # no gauge yet
        ctx.apply_dslash(x, torch.empty_like(x), 0.0)
    with pytest.raises(OverlapError):  # overlap needs set_sign_poly
        ctx.set_gauge(dev(synth.unit_gauge((4, 4, 4, 4))))
        ctx.apply_overlap(x, torch.empty_like(x))


@pytest.fixture(scope="module")
def big():
    dims = (24, 24, 24, 64)
    U = synth.gauge_field(dims, 1, 0.5, ape_steps=3)
    psi = synth.gaussian_spinor(dims, 2)
    return dims, U, psi


@pytest.mark.parametrize("prec", ["f32", "f64", "f16", "df64"])
def test_full_size_sampled_sites(big, prec):
    """24^3 x 64 (the benchmark workload), internal-field launch as timed by bench.py;
    256 sampled output sites against the oracle computed site by site."""
    from paper_1106_4964_gb300 import Context

    dims, U, psi = big
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    ctx.tune_dslash(prec, 1)  # the launch shape bench.py times
    fi, fo = ctx.field(1, prec), ctx.field(1, prec)
    fi.load(dev(psi))
    ctx.dslash_field(fi, fo, -RHO)
    out = torch.empty_like(dev(psi))
    fo.store(out)
    got = host(out).reshape(-1, 4, 3)
    rng = np.random.default_rng(0)
    V = oracle.volume(dims)
    sites = np.concatenate([[0, V - 1, V // 2], rng.integers(0, V, 253)])
    ref = oracle.dslash_sites(dims, ABC, U, -RHO, psi, sites)
    assert rel(got[sites], ref) <= TOL[prec]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-14), ("f32", 1e-6), ("f16", 2e-3), ("df64", 1e-13)])
def test_field_dot(prec, tol):
    """FP64-accumulated scalar products of internal fields (Sec. III) against numpy."""
    from paper_1106_4964_gb300 import Context

    dims = (6, 4, 4, 6)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(synth.unit_gauge(dims)))
    x = synth.gaussian_spinor(dims, 31, nrhs=3)
    y = synth.gaussian_spinor(dims, 32, nrhs=3)
    fx, fy = ctx.field(3, prec), ctx.field(3, prec)
    fx.load(dev(x))
    fy.load(dev(y))
    got = ctx.field_dot(fx, fy)
    for r in range(3):
        ref = np.vdot(x[r], y[r])
        assert abs(got[r] - ref) <= tol * np.linalg.norm(x[r]) * np.linalg.norm(y[r])
    # bitwise reproducible
    assert np.array_equal(got, ctx.field_dot(fx, fy))


# every launch variant the autotuner may pick: (bx, by, variant)
VARIANTS = [(128, 1, 0), (64, 2, 0), (64, 1, 1), (32, 2, 2), (64, 1, 3), (128, 1, 4), (128, 1, 5), (64, 1, 6),
            (32, 2, 6), (64, 1, 7), (64, 1, 8), (128, 1, 9), (64, 1, 10), (32, 2, 10), (64, 1, 11), (32, 1, 11)]


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 6), (2, 6, 4, 10), (16, 16, 16, 32)])
@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_dslash_variants(dims, prec):
    """Each register-budget and staging variant (including the bulk-copy staged one, whose
    neighbour ranges are clipped at the array ends and wrap around the lattice) against the
    oracle, for one and three right-hand sides."""
    from paper_1106_4964_gb300 import Context

    U = synth.gauge_field(dims, 5, 0.5)
    psi = synth.gaussian_spinor(dims, 6, nrhs=3)
    ref = [oracle.dslash(dims, ABC, U, -RHO, psi[r]) for r in range(3)]
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    for bx, by, var in VARIANTS:
        for nrhs in (1, 3):
            ctx.set_dslash_shape(prec, nrhs, bx, by, var)
            src = dev(psi[:nrhs])
            out = torch.empty_like(src)
            ctx.apply_dslash(src, out, -RHO, prec=prec)
            got = host(out)
            for r in range(nrhs):
                err = rel(got[r], ref[r])
                assert err <= TOL[prec], (bx, by, var, nrhs, r, err)


@pytest.mark.parametrize("prec", ["f32", "f16", "df64"])
def test_autotuned_shape_parity(prec):
    from paper_1106_4964_gb300 import Context

    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 7, 0.5)
    psi = synth.gaussian_spinor(dims, 8, nrhs=2)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    for nrhs in (1, 2):
        shape = ctx.tune_dslash(prec, nrhs)
        out = torch.empty_like(dev(psi[:nrhs]))
        ctx.apply_dslash(dev(psi[:nrhs]), out, 0.2, prec=prec)
        got = host(out)
        for r in range(nrhs):
            assert rel(got[r], oracle.dslash(dims, ABC, U, 0.2, psi[r])) <= TOL[prec], shape


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_twelve_rhs_autotuned_parity(prec):
    """The 12-source launch the multi-RHS solves take (autotuned: typically the packed-pair
    variants, several sources per thread) against the oracle for every source, and each
    pair variant forced explicitly with an odd source count (a half-empty last pair)."""
    from paper_1106_4964_gb300 import Context

    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 9, 0.5)
    psi = synth.gaussian_spinor(dims, 10, nrhs=12)
    ref = [oracle.dslash(dims, ABC, U, -RHO, psi[r]) for r in range(12)]
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    shape = ctx.tune_dslash(prec, 12)
    out = torch.empty_like(dev(psi))
    ctx.apply_dslash(dev(psi), out, -RHO, prec=prec)
    got = host(out)
    for r in range(12):
        assert rel(got[r], ref[r]) <= TOL[prec], (shape, r)
    for bx, by, var in [(64, 2, 10), (32, 3, 10), (64, 1, 11), (32, 2, 11)]:
        ctx.set_dslash_shape(prec, 11, bx, by, var)
        out = torch.empty_like(dev(psi[:11]))
        ctx.apply_dslash(dev(psi[:11]), out, -RHO, prec=prec)
        got = host(out)
        for r in range(11):
            assert rel(got[r], ref[r]) <= TOL[prec], (bx, by, var, r)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("df64", 1e-12), ("f32", 1e-6)])
def test_full_size_hw_hermiticity(big, prec, tol):
    """A property that holds at any size, checked on the whole 24^3 x 64 lattice: H_w is
    Hermitian, <u, H_w v> = <H_w u, v> (gamma5-hermiticity of D_w, Sec. II)."""
    from paper_1106_4964_gb300 import Context

    dims, U, _ = big
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(U))
    u = dev(synth.gaussian_spinor(dims, 41))
    v = dev(synth.gaussian_spinor(dims, 42))
    hu, hv = torch.empty_like(u), torch.empty_like(v)
    ctx.apply_Hw(u, hu, -RHO, prec=prec)
    ctx.apply_Hw(v, hv, -RHO, prec=prec)
    lhs = torch.vdot(u.reshape(-1), hv.reshape(-1)).item()
    rhs = torch.vdot(hu.reshape(-1), v.reshape(-1)).item()
    scale = (torch.linalg.vector_norm(u) * torch.linalg.vector_norm(hv)).item()
    assert abs(lhs - rhs) <= tol * scale
