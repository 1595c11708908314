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
    # engine 2: bf16 rows and bf16 psi plus their remainders, FP32-class against the exact FP64 values of
    # the FP32 field (the FP32 rounding of psi and of the rows stays: 1e-6 per coefficient vector)
    f = ctx.field(nrhs, "f32")
    f.load(dev(psi))
    c2 = ctx.project_lowmodes(1, f, engine=2)
    c0f = ctx.project_lowmodes(1, f, engine=0)
    for r in range(nrhs):
        assert rel(c2[:, r], exact[:, r]) < 2e-5, (r, rel(c2[:, r], exact[:, r]))
        assert rel(c2[:, r], c0f[:, r]) < 2e-5


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


# V c update on the tensor cores: bf16 rows (16-bit fields) lose ~2^-9 of |sum v c| per element;
# FP32 fields add the bf16 remainder rows and keep ~2^-17 (coefficients are split the same way)
UPD_TOL = {"f32": 5e-5, "f16": 1e-2, "bf16": 1.5e-2}


@pytest.mark.parametrize("dims,nev,nrhs", [((8, 8, 8, 8), 20, 3), ((4, 4, 4, 4), 128, 1), ((8, 4, 4, 8), 37, 12),
                                           ((16, 16, 16, 32), 100, 1)])
def test_tensor_core_update(dims, nev, nrhs):
    """out1 = psi - sum_i v_i c_i and out2 = gamma5 sum_i sign(val_i) c_i v_i (Eq. 7) by tcgen05 against
    numpy in FP64 and against the CUDA-core engine, with coefficients as large as the field."""
    from paper_1106_4964_gb300 import Context

    V = oracle.volume(dims)
    ctx = Context(dims, ABC)
    ctx.set_gauge(dev(synth.unit_gauge(dims)))
    vecs = synth.orthonormal_fields(dims, nev, seed=31).reshape(nev, -1)
    rng = np.random.default_rng(32)
    vals = rng.uniform(0.1, 1.0, nev) * rng.choice([-1.0, 1.0], nev)
    ctx.set_eigenpairs(0, vals, dev(vecs))
    psi = synth.gaussian_spinor(dims, 33, nrhs=nrhs).reshape(nrhs, -1)
    scale = np.linalg.norm(psi[0]) / np.sqrt(nev)
    coef = scale * (rng.standard_normal((nev, nrhs)) + 1j * rng.standard_normal((nev, nrhs)))
    low = (vecs.T @ coef).T                                   # [nrhs, 12V]: sum_i v_i c_ir
    g5 = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)
    exp1 = psi - low
    exp2 = g5 * (vecs.T @ (np.sign(vals)[:, None] * coef)).T
    for prec in ("f32", "f16", "bf16"):
        f, o1, o2 = ctx.field(nrhs, prec), ctx.field(nrhs, prec), ctx.field(nrhs, prec)
        f.load(dev(psi.reshape((nrhs,) + synth.gaussian_spinor(dims, 1)[0].shape)))
        got = {}
        for engine in (1, 0):
            ctx.lowmode_update(0, f, coef, o1, o2, engine=engine)
            a, b = torch.empty_like(dev(psi)), torch.empty_like(dev(psi))
            o1.store(a)
            o2.store(b)
            got[engine] = (host(a), host(b))
        for r in range(nrhs):
            e1 = rel(got[1][0][r], exp1[r])
            e2 = rel(got[1][1][r], exp2[r])
            assert e1 < UPD_TOL[prec] and e2 < UPD_TOL[prec], (prec, r, e1, e2)
            # the CUDA-core engine in the same storage precision is no more accurate than that
            assert rel(got[0][0][r], exp1[r]) < UPD_TOL[prec]
        print(f"tensor-core update {dims} nev={nev} nrhs={nrhs} {prec}: worst rel err "
              f"{max(rel(got[1][0][r], exp1[r]) for r in range(nrhs)):.2e} / "
              f"{max(rel(got[1][1][r], exp2[r]) for r in range(nrhs)):.2e}")
        for x in (f, o1, o2):
            x.close()
