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

For nu != 0 the 1/r^2 terms are added as in the I_n loop of Algorithm 5: per angular pair,
T = (nu^2/R^2) Zhat + (i nu/(pi R^2)) Qhat with Zhat = I_n applied to the pair's radial
coefficients and Qhat = I_n applied to (i 2 pi n Ncyc) times them (eqs. ell_mnk and the
expression for the sixth term after it), I_n from Basis.itable.
"""
from __future__ import annotations

import numpy as np

from . import transforms


def apply_H_box(basis, V, eta, nu, Xbox):
    """Algorithm 5 on box vectors.  Xbox: (box_size,) or (box_size, ns) complex."""
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
        if nu != 0:
            y = y + _inverse_square_terms(basis, nu, Z, Q)
        Y[:, j] = y
    return Y[:, 0] if one else Y


def _inverse_square_terms(basis, nu, Z, Q):
    """The I_n loop of Algorithm 5 on one box vector: for every pair (m, n), the K radial
    coefficients i .. i+K-1 give T = (nu^2/R^2) Zhat + (i nu/(pi R^2)) Qhat, Zhat_k' =
    sum_k Z_k I(n, k, k'), Qhat_k' = sum_k Q_k I(n, k, k'), Q = (i 2 pi n Ncyc) Z."""
    Zb = Z.reshape(basis.box_shape)
    Qb = Q.reshape(basis.box_shape)
    T = np.zeros(basis.box_shape, dtype=np.complex128)
    R2 = basis.R ** 2
    for n in range(-basis.N, basis.N + 1):
        I = basis.itable(n)
        i = n + basis.N
        Zhat = Zb[:, i, :] @ I          # rows: m; columns: k'
        Qhat = Qb[:, i, :] @ I
        T[:, i, :] = (nu ** 2 / R2) * Zhat + (1j * nu / (np.pi * R2)) * Qhat
    return T.ravel()


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
    if kp.nu != 0:
        # the 1/r^2 terms: same (m, n), coefficient (nu^2 - 2 nu n Ncyc)/R^2 times I(n, k, k')
        # (the two terms of the I_n loop of Algorithm 5 with i nu/(pi R^2) (i 2 pi n Ncyc)
        # = -2 nu n Ncyc/R^2)
        same = (kp.m[:, None] == kp.m[None, :]) & (kp.n[:, None] == kp.n[None, :])
        coef = (kp.nu ** 2 - 2 * kp.nu * kp.n * basis.ncyc) / basis.R ** 2
        tabs = {n: basis.itable(n) for n in np.unique(kp.n)}
        Ik = np.zeros((L, L))
        for n, I in tabs.items():
            sel = np.nonzero(kp.n == n)[0]
            Ik[np.ix_(sel, sel)] = I[np.ix_(kp.k[sel], kp.k[sel])]
        H += np.where(same, Ik * coef[None, :], 0.0)
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
