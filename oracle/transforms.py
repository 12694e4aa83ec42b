"""Oracle: basis transforms between reciprocal space (coefficients on the box Gamma) and
real space (values on the (theta1, theta2, r) grid).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Array conventions
  coefficients: complex array of shape (2M+1, 2N+1, K) indexed [m+M, n+N, k]; flattened in C
                order this is eq. wavefun_storage.
  grid values:  complex array of shape (N_th1, N_th2, N_r) indexed [i, j, p]; flattened in C
                order this is eq. wavefun_storage_real.

naive_inverse / naive_forward are the direct sums eq. Naive_Inverse_Transform and
eq. Fast_fwd_transform_cont.  fast_inverse / fast_forward follow Algorithms 1-4: a radial
matrix-vector product per (m, n) with the tables frak R_n / frak O_n, and one 2-D FFT per radial
node.  Reading of Algorithms 2 and 4 (listed in the design notes): the angular array has rows
indexed by theta2/n and columns by theta1/m; coefficient (m, n) sits in FFT bin
(n mod N_th2, m mod N_th1), which is what the zero-padding plus ifftshift/fftshift of the
algorithms does when N_th = 4*max+1 and which stays correct for any N_th >= 2*max+1.
"""
from __future__ import annotations

import numpy as np


# ------------------------------------------------------------------------------- naive sums

def naive_inverse(basis, ghat: np.ndarray) -> np.ndarray:
    """g(theta1_i, theta2_j, r_p) = sum_Gamma ghat_{m,n,k} F_{m,n,k}(...) (eq. Naive_Inverse_Transform)."""
    th1, th2 = basis.theta_grid()
    T1, T2, RR = np.meshgrid(th1, th2, basis.r, indexing="ij")
    g = np.zeros(T1.shape, dtype=np.complex128)
    for im, m in enumerate(range(-basis.M, basis.M + 1)):
        for jn, n in enumerate(range(-basis.N, basis.N + 1)):
            for k in range(basis.K):
                c = ghat[im, jn, k]
                if c != 0:
                    g += c * basis.F(m, n, k, T1, T2, RR)
    return g


def naive_forward(basis, g: np.ndarray) -> np.ndarray:
    """ghat_{m,n,k} = 2 pi tau sum_{i,j,p} g F* w_r w_th1 w_th2 (eq. Fast_fwd_transform_cont)."""
    th1, th2 = basis.theta_grid()
    T1, T2, RR = np.meshgrid(th1, th2, basis.r, indexing="ij")
    W = basis.wr[None, None, :] * (1.0 / basis.Nth1) * (1.0 / (basis.ncyc * basis.Nth2))
    out = np.zeros(basis.box_shape, dtype=np.complex128)
    for im, m in enumerate(range(-basis.M, basis.M + 1)):
        for jn, n in enumerate(range(-basis.N, basis.N + 1)):
            for k in range(basis.K):
                out[im, jn, k] = 2 * np.pi * basis.tau * np.sum(
                    g * np.conj(basis.F(m, n, k, T1, T2, RR)) * W)
    return out


# ------------------------------------------------------------------------- Algorithms 1-4

def angular_inverse(basis, vhat: np.ndarray) -> np.ndarray:
    """Algorithm 2.  vhat[m+M, n+N] -> v[i, j] on the angular Fourier grid."""
    W = np.zeros((basis.Nth2, basis.Nth1), dtype=np.complex128)
    mb = np.arange(-basis.M, basis.M + 1) % basis.Nth1
    nb = np.arange(-basis.N, basis.N + 1) % basis.Nth2
    W[np.ix_(nb, mb)] = np.asarray(vhat).T            # bin (n mod N_th2, m mod N_th1)
    U = np.fft.ifft2(W) * (basis.Nth1 * basis.Nth2)
    return U.T            # [i, j]


def angular_forward(basis, u: np.ndarray) -> np.ndarray:
    """Algorithm 4.  u[i, j] on the angular grid -> uhat[m+M, n+N]."""
    W = np.asarray(u).T   # rows theta2, columns theta1
    V = np.fft.fft2(W) / (basis.Nth1 * basis.Nth2)
    mb = np.arange(-basis.M, basis.M + 1) % basis.Nth1
    nb = np.arange(-basis.N, basis.N + 1) % basis.Nth2
    return V[np.ix_(nb, mb)].T                        # [m+M, n+N]


def fast_inverse(basis, ghat: np.ndarray, tables=None) -> np.ndarray:
    """Algorithm 1: G_{m,n}(r_p) = frak R_n ghat_{m,n,:} for every (m, n), then Algorithm 2 at
    every radial node.  tables (optional): other radial tables by n in place of frak R_n (the
    functions B_n of Appendix C for the radial derivative)."""
    tabs = basis.Rtab if tables is None else tables
    G = np.empty((2 * basis.M + 1, 2 * basis.N + 1, basis.Nr), dtype=np.complex128)
    for im in range(2 * basis.M + 1):
        for jn, n in enumerate(range(-basis.N, basis.N + 1)):
            G[im, jn, :] = tabs[n] @ ghat[im, jn, :]
    g = np.empty((basis.Nth1, basis.Nth2, basis.Nr), dtype=np.complex128)
    for p in range(basis.Nr):
        g[:, :, p] = angular_inverse(basis, G[:, :, p])
    return g


def fast_forward(basis, g: np.ndarray) -> np.ndarray:
    """Algorithm 3: Algorithm 4 at every radial node, then ghat_{m,n,:} = frak O_n H(:, (m,n))
    for every (m, n), scaled by 2 pi tau / Ncyc."""
    H = np.empty((2 * basis.M + 1, 2 * basis.N + 1, basis.Nr), dtype=np.complex128)
    for p in range(basis.Nr):
        H[:, :, p] = angular_forward(basis, g[:, :, p])
    out = np.empty(basis.box_shape, dtype=np.complex128)
    for im in range(2 * basis.M + 1):
        for jn, n in enumerate(range(-basis.N, basis.N + 1)):
            out[im, jn, :] = basis.Otab[n] @ H[im, jn, :]
    return (2 * np.pi * basis.tau / basis.ncyc) * out
