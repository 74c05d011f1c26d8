"""Brute-force references for pinning the oracle (test-only; no FFTs).

Everything here is written from definitions with explicit loops or dense
matrices, independently of ``oracle/``:
  * direct circular 2D convolution,
  * the circulant (Toeplitz on the torus) matrix of a filter, the operator
    T(.) of Sec. III-D eq. (csc2sc),
  * an explicit DFT matrix built from exp(-2 pi i k n / N).
"""
import numpy as np


def circ_conv2(d: np.ndarray, z: np.ndarray) -> np.ndarray:
    """(d (*) z)(q) = sum_m d(m) z((q - m) mod N), d placed at the top-left."""
    n1, n2 = z.shape
    out = np.zeros((n1, n2))
    for m1 in range(d.shape[0]):
        for m2 in range(d.shape[1]):
            if d[m1, m2] == 0.0:
                continue
            for q1 in range(n1):
                for q2 in range(n2):
                    out[q1, q2] += d[m1, m2] * z[(q1 - m1) % n1, (q2 - m2) % n2]
    return out


def conv_matrix(d: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """Dense matrix T with vec(d (*) z) = T vec(z) (row-major vec).

    T[q, j] = d((q - j) mod N), d zero outside its top-left support.
    """
    P = n1 * n2
    T = np.zeros((P, P))
    m1, m2 = d.shape
    for q1 in range(n1):
        for q2 in range(n2):
            for j1 in range(n1):
                for j2 in range(n2):
                    a1 = (q1 - j1) % n1
                    a2 = (q2 - j2) % n2
                    if a1 < m1 and a2 < m2:
                        T[q1 * n2 + q2, j1 * n2 + j2] = d[a1, a2]
    return T


def dft_matrix_2d(n1: int, n2: int) -> np.ndarray:
    """Dense unnormalised 2D DFT matrix acting on row-major vec."""
    k1 = np.arange(n1)
    k2 = np.arange(n2)
    F1 = np.exp(-2j * np.pi * np.outer(k1, k1) / n1)
    F2 = np.exp(-2j * np.pi * np.outer(k2, k2) / n2)
    return np.kron(F1, F2)


def soft(v, t):
    out = np.zeros_like(v)
    big = v > t
    small = v < -t
    out[big] = v[big] - t
    out[small] = v[small] + t
    return out


def fista_lasso(T: np.ndarray, x: np.ndarray, lam: float, iters: int) -> np.ndarray:
    """Textbook FISTA (Beck & Teboulle 2009) for min 1/2||x - T z||^2 + lam ||z||_1."""
    L = np.linalg.norm(T, 2) ** 2
    z = np.zeros(T.shape[1])
    y = z.copy()
    t = 1.0
    for _ in range(iters):
        g = T.T @ (T @ y - x)
        z_new = soft(y - g / L, lam / L)
        t_new = (1 + np.sqrt(1 + 4 * t * t)) / 2
        y = z_new + ((t - 1) / t_new) * (z_new - z)
        z, t = z_new, t_new
    return z
