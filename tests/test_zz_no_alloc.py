"""The allocation-free scalar product (ov_field_dot_noalloc) against the
ordinary one (ov_field_dot), called through the C ABI twice in a row.

It exists for callers that cannot allocate device memory when they call (a
CUDA graph being captured in global mode, a memory manager that owns the
device): its partial sums live in a fixed array of the library's device
image.  This file is collected last so that a failure here never hides the
other GPU tests of a run that stops at the first failure."""
import numpy as np
import pytest

import synth
from gpu_common import ABC, dev, need_gpu, torch

pytestmark = pytest.mark.gpu

# the same kernels run in both entry points; only the location of the partial sums differs
TOL = {"f64": 1e-14, "f32": 1e-14, "f16": 1e-14}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("dims,nrhs", [((6, 4, 4, 6), 3), ((24, 24, 24, 64), 2)])
def test_noalloc_dot_matches_field_dot(prec, dims, nrhs):
    from paper_1106_4964_gb300 import Context

    ctx = Context(dims, ABC)
    x = synth.gaussian_spinor(dims, 41, nrhs=nrhs)
    y = synth.gaussian_spinor(dims, 42, nrhs=nrhs)
    fx, fy = ctx.field(nrhs, prec), ctx.field(nrhs, prec)
    fx.load(dev(x))
    fy.load(dev(y))
    ref = ctx.field_dot(fx, fy)
    held = ctx.device_bytes()
    scale = np.array([np.linalg.norm(x[r]) * np.linalg.norm(y[r]) for r in range(nrhs)])
    for _ in range(2):  # two calls in a row: the shared array keeps the last call's partial sums
        got = ctx.field_dot_noalloc(fx, fy)
        assert np.all(np.abs(got - ref) <= TOL[prec] * scale)
    out = torch.zeros(2 * nrhs, dtype=torch.float64, device="cuda")
    for _ in range(2):
        ctx.field_dot_noalloc(fx, fy, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.complex128)
        assert np.all(np.abs(got - ref) <= TOL[prec] * scale)
    assert ctx.device_bytes() == held  # nothing allocated through the context
