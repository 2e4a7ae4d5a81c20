"""Superoperator form of the Lindblad equation and its exact solutions.

TEST INFRASTRUCTURE ONLY (small N; the superoperator has N^4 entries).

Vectorisation is column stacking, vec(X) = X.flatten(order="F"), for which
vec(A X B) = (B^T kron A) vec(X). With that convention Eq. 2 / Eq. S8 reads

    Lsup = -(1-omega) i (I kron H - H^T kron I)
           + omega sum_k ( L_k^* kron L_k
                           - 1/2 (I kron L_k^dag L_k + L_k^T L_k^* kron I) ).

The paper prints the first dissipator factor as L_k^dag kron L_k; the
column-stacking identity above (which the paper's other three terms obey)
gives L_k^* kron L_k, and that is the reading used here.

The jump operators are the N^2 matrices L_ij = sqrt(G_ij)|i><j| (Eq. S7 and
the paragraph after it). Every Kronecker product is formed element by element
with the index formula of Eq. 3 / Eq. S9.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def kron_eq3(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Kronecker product of two n x n matrices by Eq. 3 (0-based indices):
    C[i, j] = A[i div n, j div n] * B[i mod n, j mod n]."""
    n = a.shape[0]
    assert a.shape == (n, n) and b.shape == (n, n)
    i = np.arange(n * n)[:, None]
    j = np.arange(n * n)[None, :]
    return a[i // n, j // n] * b[i % n, j % n]


def vec(x: np.ndarray) -> np.ndarray:
    return np.asarray(x).flatten(order="F")


def unvec(v: np.ndarray, n: int) -> np.ndarray:
    return np.asarray(v).reshape((n, n), order="F")


def jump_operators(G: np.ndarray):
    """Nonzero L_ij = sqrt(G_ij)|i><j| for all i, j with G_ij != 0."""
    n = G.shape[0]
    ops = []
    for i in range(n):
        for j in range(n):
            if G[i, j] != 0.0:
                L = np.zeros((n, n), dtype=np.complex128)
                L[i, j] = np.sqrt(G[i, j])
                ops.append(L)
    return ops


def superoperator(H: np.ndarray, G: np.ndarray, omega: float) -> np.ndarray:
    """N^2 x N^2 generator of Eq. 2 / Eq. S8 (column-stacking convention)."""
    n = H.shape[0]
    eye = np.eye(n, dtype=np.complex128)
    Hc = H.astype(np.complex128)
    lsup = -(1.0 - omega) * 1j * (kron_eq3(eye, Hc) - kron_eq3(Hc.T, eye))
    diss = np.zeros((n * n, n * n), dtype=np.complex128)
    for L in jump_operators(G):
        LdL = L.conj().T @ L
        diss += kron_eq3(L.conj(), L)
        diss -= 0.5 * (kron_eq3(eye, LdL) + kron_eq3(L.T @ L.conj(), eye))
    return lsup + omega * diss


def rk4_amplification(z):
    """Stability polynomial of classical RK4: R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24."""
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0


def rk4_by_eigendecomposition(lsup: np.ndarray, rho0: np.ndarray, dt: float, steps: int):
    """y_n = R(dt Lsup)^n y_0 through Lsup = V diag(lam) V^-1.

    For a linear ODE, n classical RK4 steps are exactly the n-th power of the
    amplification matrix R(dt Lsup). Returns (rho_n, cond(V))."""
    n = rho0.shape[0]
    lam, V = np.linalg.eig(lsup)
    coef = np.linalg.solve(V, vec(rho0))
    amp = rk4_amplification(dt * lam) ** steps
    y = V @ (amp * coef)
    return unvec(y, n), float(np.linalg.cond(V))


def rk4_by_matrix_power(lsup: np.ndarray, rho0: np.ndarray, dt: float, steps: int):
    """y_n = R(dt Lsup)^n y_0 by repeated squaring of the amplification matrix
    (no eigendecomposition, so no conditioning issue)."""
    n = rho0.shape[0]
    z = dt * lsup
    eye = np.eye(z.shape[0], dtype=np.complex128)
    z2 = z @ z
    R = eye + z + z2 / 2.0 + (z2 @ z) / 6.0 + (z2 @ z2) / 24.0
    P = np.linalg.matrix_power(R, steps)
    return unvec(P @ vec(rho0), n)


def exact_solution(lsup: np.ndarray, rho0: np.ndarray, t: float) -> np.ndarray:
    """rho(t) = exp(Lsup t) rho(0) (the matrix-exponential solution of the
    main text), by scipy's expm."""
    n = rho0.shape[0]
    return unvec(scipy.linalg.expm(lsup * t) @ vec(rho0), n)


def null_state(lsup: np.ndarray) -> tuple[np.ndarray, float, float]:
    """Steady state as the null vector of Lsup (right singular vector of the
    smallest singular value), made Hermitian and trace-normalised.
    Returns (rho_ss, smallest singular value, second smallest)."""
    nn = lsup.shape[0]
    n = int(round(np.sqrt(nn)))
    _, s, vh = np.linalg.svd(lsup)
    v = vh[-1].conj()
    rho = unvec(v, n)
    rho = rho / np.trace(rho)
    rho = 0.5 * (rho + rho.conj().T)
    return rho, float(s[-1]), float(s[-2])


def stationary_by_power_iteration(G: np.ndarray, tol: float = 1e-15, max_iter: int = 200000):
    """Stationary vector of the column-stochastic G: p <- G p until the
    1-norm change is below tol."""
    n = G.shape[0]
    p = np.full(n, 1.0 / n)
    for _ in range(max_iter):
        q = G @ p
        q /= q.sum()
        if np.abs(q - p).sum() < tol:
            return q
        p = q
    return p
