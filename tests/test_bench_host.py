"""Host-side logic of bench.py that needs no GPU:

* the degree search of `sign_for_delta` (the lowest multiple of 10 whose sign accuracy delta of
  Eq. 4 meets a target), driven through a stand-in context whose delta is the oracle's Chebyshev
  interpolant measured on [eps, 1], against a brute-force scan of every multiple of 10;
* the launch-variant bookkeeping: every dslash variant the library declares has a kernel name and
  a source unit that exists (the DRAM-traffic figures are keyed by the hash of that unit);
* the algorithmic byte counts per site, against the counts written out by hand from the storage
  formats (24 reals per spinor, 12 reals per reconstruct-12 link, a 4-byte scale per 16-bit
  spinor)."""
import os
import re

import numpy as np
import pytest

import bench
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _delta(eps, n):
    c = oracle.cheb_coeffs(eps, n)
    sx = np.linspace(np.sqrt(eps), 1.0, 4001)
    x = sx * sx
    y = (2 * x - (1 + eps)) / (1 - eps)
    return float(np.max(np.abs(1 - sx * np.polynomial.chebyshev.chebval(y, c))))


class _FakeCtx:
    """The two calls sign_for_delta makes, with delta from the oracle's interpolant."""

    def __init__(self):
        self.cache = {}
        self.installed = None

    def set_sign_poly(self, rho, eps, n, lmax):
        self.installed = (eps, n)

    def get_option(self, name):
        assert name == "sign_delta"
        key = self.installed
        if key not in self.cache:
            self.cache[key] = _delta(*key)
        return self.cache[key]


@pytest.mark.parametrize("eps,target", [(0.05, 1e-10), (0.01, 1e-8), (0.0064, 1e-10)])
def test_sign_for_delta_is_lowest_degree(eps, target):
    ctx = _FakeCtx()
    n, d = bench.sign_for_delta(ctx, eps, 6.6, target, 0)
    assert d <= target and ctx.installed == (eps, n)
    # brute force over the multiples of 10 below the answer: none meets the target
    for m in range(10, n, 10):
        assert _delta(eps, m) > target, (m, n)


def test_sign_for_delta_fixed_degree():
    ctx = _FakeCtx()
    n, d = bench.sign_for_delta(ctx, 0.05, 6.6, 0.0, 37)
    assert n == 37 and ctx.installed == (0.05, 37) and d == pytest.approx(_delta(0.05, 37))


def test_every_variant_has_a_kernel_and_a_unit():
    with open(os.path.join(ROOT, "paper_1106_4964_gb300", "csrc", "ov_kernels.h")) as f:
        nvar = int(re.search(r"DSLASH_VARIANTS\s*=\s*(\d+)", f.read()).group(1))
    assert sorted(bench.VARIANT_UNIT) == list(range(nvar))
    for v in range(nvar):
        assert os.path.exists(os.path.join(ROOT, "paper_1106_4964_gb300", "csrc", bench.VARIANT_UNIT[v]))
        name = bench.kernel_name("f32", v)
        with open(os.path.join(ROOT, "paper_1106_4964_gb300", "csrc", bench.VARIANT_UNIT[v])) as f:
            src = f.read()
        kernel = name.split("<")[0]
        # the named kernel is defined in its unit, or in the shared header for the basic variants
        if kernel not in src:
            with open(os.path.join(ROOT, "paper_1106_4964_gb300", "csrc", "dslash_common.cuh")) as f:
                assert kernel in f.read(), (v, name)
    assert len(bench.kernel_sources_sha(1)) == 16


def test_algorithmic_bytes_per_site():
    # one RHS: 4 links x 12 reals + spinor in + spinor out (24 reals each)
    assert bench.site_bytes("f64") == 4 * 12 * 8 + 2 * 24 * 8
    assert bench.site_bytes("f32") == 4 * 12 * 4 + 2 * 24 * 4
    assert bench.site_bytes("f16") == 4 * 12 * 2 + 2 * (24 * 2 + 4)
    # 12 RHS share the links
    assert bench.site_bytes("f32", 12) == pytest.approx(4 * 12 * 4 / 12 + 2 * 24 * 4)
    # Clenshaw step: two D_w launches plus psi_h, b_{k+1}, b_{k+2}
    assert bench.clenshaw_step_bytes("f32", 1, True) == 2 * (4 * 12 * 4 + 2 * 96) + 3 * 96
    # 16-bit storage with FP32 recurrence fields: 16-bit links, FP32 spinors
    assert bench.clenshaw_step_bytes("f16", 1, True) == 2 * (4 * 12 * 2 + 2 * 96) + 3 * 96
    assert bench.clenshaw_step_bytes("f16", 1, False) == 2 * (4 * 12 * 2 + 2 * 52) + 3 * 52
