"""Oracle: the discretised Hamiltonian at one (eta, nu) point.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

apply_H_box   Algorithm 5, one column at a time, on box vectors.
apply_H       the same restricted to the cutoff mask: Y = M .* H (M .* X), returned in the
              compact (masked) order.
dense_H       dense matrix by columns H e_j (tiny cases).
dense_H_conv  the same matrix written out as D + B^H W diag(V) B, with the angular part of
              B^H W diag(V) B reduced by the discrete convolution theorem:
                  H_V[(m',n',k'), (m,n,k)] = (2 pi tau / Ncyc) sum_p w_p xi_{n',k'}(r_p) xi_{n,k}(r_p)
                                             * Vhat_p(m'-m, n'-n),
              Vhat_p = fft2 of V at node p / (N_th1 N_th2), indices taken modulo the grid.
              Algebraically identical to Algorithm 5 (eqs. Fast_fwd_transform_cont_3 and
              Fast_fwd_transform_cont_2 composed with Algorithm 1) and used where building H by
              columns would be too slow.
eigh_lowest   direct diagonalisation (numpy.linalg.eigh).

The 1/r^2 terms that appear when nu != 0 (eqs. ell_mnk, I_nkk_prime and the I_n loop of
Algorithm 5) are not implemented: every workload here has nu = 0.
"""
from __future__ import annotations

import numpy as np

from . import transforms


def apply_H_box(basis, V, eta, nu, Xbox):
    """Algorithm 5 on box vectors.  Xbox: (box_size,) or (box_size, ns) complex."""
    if nu != 0:
        raise NotImplementedError("nu != 0: I_n term not implemented")
    X = np.asarray(Xbox, dtype=np.complex128)
    one = X.ndim == 1
    if one:
        X = X[:, None]
    m, n, k = basis.box_mnk()
    Lam = basis.lambda0(m, n, k)
    Mv = 2j * np.pi * m
    Nv = 2j * np.pi * basis.ncyc * n
    a, b, c = basis.abc(eta, nu)
    Y = np.zeros_like(X)
    for j in range(X.shape[1]):
        Z = X[:, j]
        P = Mv * Z
        Q = Nv * Z
        y = 0.5 * (Lam * Z)
        y = y - a * Z - b * P - c * Q
        Zr = transforms.fast_inverse(basis, Z.reshape(basis.box_shape))
        y = y + transforms.fast_forward(basis, Zr * V).ravel()
        Y[:, j] = y
    return Y[:, 0] if one else Y


def apply_H(kp, V, Xc):
    """Y = H X in compact (masked) order at the k-point kp."""
    Xc = np.asarray(Xc, dtype=np.complex128)
    Yb = apply_H_box(kp.basis, V, kp.eta, kp.nu, kp.to_box(Xc))
    return kp.from_box(Yb)


def dense_H(kp, V):
    L = kp.L
    H = np.empty((L, L), dtype=np.complex128)
    E = np.eye(L, dtype=np.complex128)
    for j0 in range(0, L, 64):
        H[:, j0:j0 + 64] = apply_H(kp, V, E[:, j0:j0 + 64])
    return H


def dense_H_conv(kp, V):
    basis = kp.basis
    L = kp.L
    H = np.diag(kp.ke.astype(np.complex128))
    Xi = np.empty((basis.Nr, L))
    for n in range(-basis.N, basis.N + 1):
        sel = kp.n == n
        Xi[:, sel] = basis.Rtab[n][:, kp.k[sel]]
    dm = (kp.m[:, None] - kp.m[None, :]) % basis.Nth1
    dn = (kp.n[:, None] - kp.n[None, :]) % basis.Nth2
    pref = 2 * np.pi * basis.tau / basis.ncyc
    for p in range(basis.Nr):
        Vhat = np.fft.fft2(np.asarray(V[:, :, p]).T) / (basis.Nth1 * basis.Nth2)   # [n, m]
        H += (pref * basis.wr[p]) * np.outer(Xi[p], Xi[p]) * Vhat[dn, dm]
    return H


def eigh_lowest(H, nev=None):
    w, U = np.linalg.eigh(H)
    if nev is not None:
        return w[:nev], U[:, :nev]
    return w, U
