"""Independent brute-force statements used to pin the oracle (tests only).

The global Q1 matrix is assembled here the textbook way, from 1D element matrices
summed into global 1D stiffness/mass matrices and combined by Kronecker products,
and Gauss-Seidel / Jacobi run on that dense matrix.  Nothing here calls the oracle,
so agreement between the two is evidence for both.
"""
import math

import numpy as np


def global_1d(n: int, h: float):
    """Global 1D stiffness and mass matrices on n cells (n+1 vertices)."""
    A = np.zeros((n + 1, n + 1))
    M = np.zeros((n + 1, n + 1))
    ae = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
    me = np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0
    for c in range(n):
        A[c:c + 2, c:c + 2] += ae
        M[c:c + 2, c:c + 2] += me
    return A, M


def global_matrix(dim: int, n, h: float) -> np.ndarray:
    """Dense A = K / h^d on all vertices, x fastest (kron(z, kron(y, x)))."""
    if isinstance(n, int):
        n = (n,) * dim
    mats = [global_1d(n[a], h) for a in range(dim)]  # axis 0 = x
    K = 0.0
    for axis in range(dim):
        term = None
        # build kron over axes from slowest (last) to fastest (x)
        for b in reversed(range(dim)):
            Ab, Mb = mats[b]
            factor = Ab if b == axis else Mb
            term = factor if term is None else np.kron(term, factor)
        K = K + term
    return K / h ** dim


def interior_mask(shape) -> np.ndarray:
    m = np.zeros(shape, dtype=bool)
    sl = tuple(slice(1, s - 1) for s in shape)
    m[sl] = True
    return m


def colour_array(shape) -> np.ndarray:
    """Vertex colour (i&1) + 2(j&1) + 4(k&1) for arrays (z, y, x) or (y, x)."""
    idx = np.indices(shape)
    if len(shape) == 3:
        k, j, i = idx
        return (i & 1) + 2 * (j & 1) + 4 * (k & 1)
    j, i = idx
    return (i & 1) + 2 * (j & 1)


def dense_apply(u: np.ndarray, h: float) -> np.ndarray:
    dim = u.ndim
    n = tuple(s - 1 for s in reversed(u.shape))
    A = global_matrix(dim, n, h)
    y = (A @ u.ravel()).reshape(u.shape)
    y[~interior_mask(u.shape)] = 0.0
    return y


def dense_gs(u0: np.ndarray, f: np.ndarray, h: float, sweeps: int, order_seed=None):
    """Coloured Gauss-Seidel on the dense matrix: colours ascending, lexicographic
    inside a colour (or a random order inside each colour when order_seed is set)."""
    dim = u0.ndim
    n = tuple(s - 1 for s in reversed(u0.shape))
    A = global_matrix(dim, n, h)
    u = u0.ravel().copy()
    ff = f.ravel()
    col = colour_array(u0.shape).ravel()
    inner = interior_mask(u0.shape).ravel()
    g = np.random.default_rng(order_seed) if order_seed is not None else None
    for _ in range(sweeps):
        for c in range(1 << dim):
            ids = np.nonzero(inner & (col == c))[0]
            if g is not None:
                ids = g.permutation(ids)
            for i in ids:
                row = A[i]
                off = row @ u - row[i] * u[i]
                u[i] = (ff[i] - off) / row[i]
    return u.reshape(u0.shape)


def dense_jacobi(u0, f, h, omega, sweeps):
    dim = u0.ndim
    n = tuple(s - 1 for s in reversed(u0.shape))
    A = global_matrix(dim, n, h)
    inner = interior_mask(u0.shape).ravel()
    u = u0.ravel().copy()
    for _ in range(sweeps):
        r = f.ravel() - A @ u
        d = np.diag(A)
        un = u + omega * r / d
        u = np.where(inner, un, u)
    return u.reshape(u0.shape)


def symbol(dim: int, thetas) -> float:
    """lambda_S(theta) = sum over axes of a(theta_axis) * prod_others m(theta_other),
    a(t) = 2 - 2cos t (1D stiffness symbol), m(t) = (2 + cos t)/3 (1D mass symbol)."""
    a = [2.0 - 2.0 * math.cos(t) for t in thetas[:dim]]
    m = [(2.0 + math.cos(t)) / 3.0 for t in thetas[:dim]]
    tot = 0.0
    for ax in range(dim):
        p = a[ax]
        for b in range(dim):
            if b != ax:
                p *= m[b]
        tot += p
    return tot


def sine_mode(dim: int, n: int, modes) -> np.ndarray:
    x = np.arange(n + 1) / n
    if dim == 3:
        return (np.sin(modes[2] * math.pi * x)[:, None, None] *
                np.sin(modes[1] * math.pi * x)[None, :, None] *
                np.sin(modes[0] * math.pi * x)[None, None, :])
    return np.sin(modes[1] * math.pi * x)[:, None] * np.sin(modes[0] * math.pi * x)[None, :]
