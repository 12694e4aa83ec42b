"""Oracle: plain LOBPCG with the Teter-Payne-Allan (TPA) diagonal preconditioner.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. "Eigensolvers and Preconditioning": LOBPCG with the TPA preconditioner, whose diagonal
entries are P(g)/(P(g) + 16 g^4) with P(g) = 27 + 18 g + 12 g^2 + 8 g^3 and
g_i = (kinetic energy of basis function i) / (kinetic energy of the residual vector).

Readings (listed in the design notes):
  9   "kinetic energy of the residual vector" is the |r_i|^2-weighted mean of KE_i over the
      column, with KE_i the shifted kinetic energy used by the cutoff mask.
  10  the LOBPCG variant is the standard three-term one on span[X, W, P] with soft locking of
      converged columns; a column is converged when ||H x - theta x||_2 <= tol with ||x|| = 1.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def tpa(ke: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Apply the TPA diagonal to every column of R."""
    R = np.asarray(R)
    w = np.abs(R) ** 2
    ke_res = (ke @ w) / np.maximum(w.sum(axis=0), 1e-300)
    g = ke[:, None] / ke_res[None, :]
    P = 27 + 18 * g + 12 * g ** 2 + 8 * g ** 3
    return (P / (P + 16 * g ** 4)) * R


def _orthonormalize(W, drop=1e-12):
    """Symmetric orthonormalisation of the columns of W, dropping near-dependent directions."""
    G = W.conj().T @ W
    lam, Q = np.linalg.eigh(G)
    keep = lam > drop * max(lam.max(), 1e-300)
    return W @ (Q[:, keep] / np.sqrt(lam[keep]))


def lobpcg(apply_H, ke, X0, n_eig, tol=1e-6, maxit=500, precond=None, callback=None):
    """Lowest n_eig eigenpairs.  apply_H(X) -> H X on compact blocks; X0: L x nb start block.

    Returns (theta[:n_eig], X[:, :n_eig], iterations, residual norms)."""
    if precond is None:
        precond = lambda R, theta: tpa(ke, R)
    X = _orthonormalize(np.asarray(X0, dtype=np.complex128))
    nb = X.shape[1]
    HX = apply_H(X)
    theta, C = np.linalg.eigh(X.conj().T @ HX)
    X, HX = X @ C, HX @ C
    P = HP = None
    res = None
    it = 0
    for it in range(1, maxit + 1):
        R = HX - X * theta[None, :]
        res = np.linalg.norm(R, axis=0)
        conv = res <= tol
        if conv[:n_eig].all():
            it -= 1
            break
        act = np.nonzero(~conv)[0]
        W = precond(R[:, act], theta[act])
        W = W - X @ (X.conj().T @ W)
        if P is not None:
            W = W - P @ (P.conj().T @ W)
        W = _orthonormalize(W)
        HW = apply_H(W)
        blocks = [X, W] + ([P] if P is not None else [])
        hblocks = [HX, HW] + ([HP] if P is not None else [])
        S = np.hstack(blocks)
        HS = np.hstack(hblocks)
        A = S.conj().T @ HS
        A = 0.5 * (A + A.conj().T)
        G = S.conj().T @ S
        G = 0.5 * (G + G.conj().T)
        try:
            lam, Cf = sla.eigh(A, G)
        except np.linalg.LinAlgError:
            # drop P and retry (restart of the conjugate direction)
            S, HS = np.hstack([X, W]), np.hstack([HX, HW])
            A = S.conj().T @ HS
            A = 0.5 * (A + A.conj().T)
            G = S.conj().T @ S
            lam, Cf = sla.eigh(A, 0.5 * (G + G.conj().T))
        C = Cf[:, :nb]
        theta = lam[:nb]
        Xn = S @ C
        HXn = HS @ C
        Pn = S[:, nb:] @ C[nb:]
        HPn = HS[:, nb:] @ C[nb:]
        # keep P orthonormal (it only spans a search direction)
        Gp = Pn.conj().T @ Pn
        lp, Qp = np.linalg.eigh(0.5 * (Gp + Gp.conj().T))
        keep = lp > 1e-20 * max(lp.max(), 1e-300)
        T = Qp[:, keep] / np.sqrt(lp[keep])
        X, HX, P, HP = Xn, HXn, Pn @ T, HPn @ T
        if callback is not None:
            callback(it, theta, res)
    return theta[:n_eig], X[:, :n_eig], it, res
