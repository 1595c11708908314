"""Small helpers shared by the tests (no method arithmetic)."""
import numpy as np


def dense(op, V):
    """Dense matrix of a linear map on 12*V-component fields, column by column."""
    N = 12 * V
    M = np.empty((N, N), dtype=np.complex128)
    e = np.zeros(N, dtype=np.complex128)
    for j in range(N):
        e[:] = 0
        e[j] = 1
        M[:, j] = np.asarray(op(e)).reshape(-1)
    return M


def g5_dense(V):
    return np.kron(np.eye(V), np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3)))


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def grid(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return x, y, z, t


def free_momenta(dims, bc):
    """All lattice momenta p_mu = (2 pi k + theta_mu)/L_mu, theta = pi if antiperiodic."""
    ps = [(2 * np.pi * np.arange(L) + (np.pi if b < 0 else 0.0)) / L for L, b in zip(dims, bc)]
    return ps
