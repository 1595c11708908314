"""Seeded synthetic inputs for the overlap-operator hot path.

This module is the only code shared by the FP64 oracle tests, the CUDA-path
tests and the benchmark.  It generates *data* and holds none of the method's
arithmetic (no Wilson operator, no sign function, no solver):

* ``gauge_field``: SU(3) links U_mu(n) = exp(i s H), H = sum_a h_a lambda_a / 2
  with h_a ~ N(0, 1) per link (Gell-Mann basis), optionally followed by APE
  smearing U' = Proj[(1 - alpha) U + alpha/6 * sum of the six staples] and
  Gram-Schmidt re-unitarisation (rows 1, 2 orthonormalised, row 3 =
  conj(row1 x row2)), which makes every link exactly representable by its
  first two rows (reconstruct-12).
* ``gaussian_spinor``: complex spinors with Re, Im ~ N(0, 1).
* ``point_sources``: the 12 spin-colour delta sources of one propagator.
* ``gauge_transform``: a random SU(3) matrix per site (covariance tests).
* ``orthonormal_fields``: n seeded orthonormal spinor fields (stand-ins for a
  set of eigenvectors where a formula holds for any orthonormal set).

Canonical layout (shared by every consumer):

* dims are given as (Lx, Ly, Lz, Lt); arrays are indexed [t][z][y][x] with x
  fastest;
* gauge field: complex128 [Lt, Lz, Ly, Lx, 4 (mu = x, y, z, t), 3, 3];
* spinor field: complex128 [nrhs, Lt, Lz, Ly, Lx, 4 (spin), 3 (colour)].

Random numbers come from numpy ``Generator(PCG64(seed))`` drawn in canonical
order, so a seed fixes the field on every machine up to the last bits of the
floating-point smearing arithmetic.
"""
from __future__ import annotations

import numpy as np
import torch

__all__ = [
    "gauge_field",
    "unit_gauge",
    "gaussian_spinor",
    "point_sources",
    "gauge_transform",
    "orthonormal_fields",
    "gell_mann",
]

# axis of the [t][z][y][x] site block that direction mu (0=x .. 3=t) runs along
_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_1..lambda_8 as a [8, 3, 3] array."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1], l[1, 1, 0] = -1j, 1j
    l[2, 0, 0], l[2, 1, 1] = 1, -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2], l[4, 2, 0] = -1j, 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2], l[6, 2, 1] = -1j, 1j
    l[7, 0, 0] = l[7, 1, 1] = 1 / np.sqrt(3)
    l[7, 2, 2] = -2 / np.sqrt(3)
    return l


def _shape(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def _expm_i(h: torch.Tensor) -> torch.Tensor:
    """exp(i h) for a batch of Hermitian 3x3 matrices (scaling and squaring of
    a 16-term Taylor series, accurate to rounding for |h| < 10)."""
    x = 1j * h
    norm = torch.linalg.matrix_norm(x, ord="fro").amax().item()
    k = max(0, int(np.ceil(np.log2(max(norm, 1e-300) / 0.25))))
    x = x / (2.0 ** k)
    eye = torch.eye(3, dtype=x.dtype).expand_as(x)
    term = eye.clone()
    out = eye.clone()
    for j in range(1, 17):
        term = term @ x / j
        out = out + term
    for _ in range(k):
        out = out @ out
    return out


def _reunitarise(u: torch.Tensor) -> torch.Tensor:
    """Project onto SU(3): Gram-Schmidt on rows 1 and 2, row 3 = conj(r1 x r2)."""
    r1 = u[..., 0, :]
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    r2 = u[..., 1, :]
    r2 = r2 - (r1.conj() * r2).sum(-1, keepdim=True) * r1
    r2 = r2 / torch.linalg.vector_norm(r2, dim=-1, keepdim=True)
    r3 = torch.linalg.cross(r1, r2, dim=-1).conj()
    return torch.stack([r1, r2, r3], dim=-2)


def _shift(f: torch.Tensor, mu: int, step: int) -> torch.Tensor:
    """f(n + step * mu_hat) on the periodic site block (leading 4 axes)."""
    return torch.roll(f, shifts=-step, dims=_AXIS[mu])


def _ape_step(u: torch.Tensor, alpha: float) -> torch.Tensor:
    """One APE smearing step of all four directions from the same old field."""
    out = []
    for mu in range(4):
        umu = u[..., mu, :, :]
        staple = torch.zeros_like(umu)
        for nu in range(4):
            if nu == mu:
                continue
            unu = u[..., nu, :, :]
            # forward: U_nu(n) U_mu(n+nu) U_nu(n+mu)^dag
            staple += unu @ _shift(umu, nu, 1) @ _shift(unu, mu, 1).mH
            # backward: U_nu(n-nu)^dag U_mu(n-nu) U_nu(n-nu+mu)
            unu_b = _shift(unu, nu, -1)
            staple += unu_b.mH @ _shift(umu, nu, -1) @ _shift(unu_b, mu, 1)
        out.append(_reunitarise((1.0 - alpha) * umu + (alpha / 6.0) * staple))
    return torch.stack(out, dim=-3)


def gauge_field(dims, seed: int = 1, s: float = 0.5, ape_steps: int = 0,
                alpha: float = 0.6, threads: int | None = None) -> np.ndarray:
    """Random SU(3) gauge field, complex128 [Lt, Lz, Ly, Lx, 4, 3, 3].

    U_mu(n) = exp(i s H), H = sum_a h_a lambda_a/2, h_a ~ N(0,1) drawn from
    PCG64(seed) in canonical order [t][z][y][x][mu][a]; then ``ape_steps``
    APE smearing steps with weight ``alpha``.  The result is always
    re-unitarised so that row 3 == conj(row1 x row2) to rounding.
    """
    if threads:
        torch.set_num_threads(int(threads))
    shp = _shape(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    h = rng.standard_normal(shp + (4, 8))
    lam = gell_mann()
    herm = np.einsum("...a,aij->...ij", h, lam / 2.0)
    u = _expm_i(torch.from_numpy(herm) * float(s))
    u = _reunitarise(u)
    for _ in range(int(ape_steps)):
        u = _ape_step(u, float(alpha))
    return np.ascontiguousarray(u.numpy())


def unit_gauge(dims) -> np.ndarray:
    """The free field U_mu(n) = 1."""
    shp = _shape(dims)
    u = np.zeros(shp + (4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def gaussian_spinor(dims, seed: int = 2, nrhs: int = 1) -> np.ndarray:
    """Gaussian complex spinors, complex128 [nrhs, Lt, Lz, Ly, Lx, 4, 3]."""
    shp = (int(nrhs),) + _shape(dims) + (4, 3)
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal(shp)
    im = rng.standard_normal(shp)
    return re + 1j * im


def point_sources(dims, site=(0, 0, 0, 0)) -> np.ndarray:
    """The 12 spin-colour point sources delta_{n,site} delta_{s,s0} delta_{c,c0}
    (source index = 3*s0 + c0), complex128 [12, Lt, Lz, Ly, Lx, 4, 3].
    ``site`` is (x, y, z, t)."""
    x, y, z, t = site
    out = np.zeros((12,) + _shape(dims) + (4, 3), dtype=np.complex128)
    for s0 in range(4):
        for c0 in range(3):
            out[3 * s0 + c0, t, z, y, x, s0, c0] = 1.0
    return out


def gauge_transform(dims, seed: int = 3) -> np.ndarray:
    """A random SU(3) matrix g(n) per site, complex128 [Lt, Lz, Ly, Lx, 3, 3]."""
    shp = _shape(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    h = rng.standard_normal(shp + (8,))
    herm = np.einsum("...a,aij->...ij", h, gell_mann() / 2.0)
    g = _reunitarise(_expm_i(torch.from_numpy(herm) * 2.0))
    return np.ascontiguousarray(g.numpy())


def orthonormal_fields(dims, n: int, seed: int = 5) -> np.ndarray:
    """n orthonormal complex spinor fields, complex128 [n, Lt, Lz, Ly, Lx, 4, 3]:
    Gaussian fields orthonormalised by two passes of Cholesky QR (X <- X R^-1
    with R^dag R = X^dag X), which leaves |X^dag X - 1| at rounding level."""
    x = gaussian_spinor(dims, seed=seed, nrhs=n).reshape(n, -1).T.copy()
    for _ in range(2):
        g = x.conj().T @ x
        r = np.linalg.cholesky(g).conj().T  # g = r^dag r, r upper triangular
        x = np.linalg.solve(r.T, x.T).T     # x r^-1, as (r^T)^-1 x^T transposed
    return np.ascontiguousarray(x.T).reshape((n,) + _shape(dims) + (4, 3))
