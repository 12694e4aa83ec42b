"""Oracle: the per-mode preconditioner network, its loss and gradients (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Not from the paper: the learned
preconditioner is an extension that refines the paper's Teter-Payne-Allan diagonal
(Sec. "Eigensolvers and Preconditioning").  It is pinned by finite differences of the loss
(test_oracle_mlp.py), so its hand-derived gradients do not rest on this file alone.

Model, per mode i of a column with Ritz value theta:
    x_i = [KE_i/E0, (m-eta)/M, (n Ncyc - nu)/N, k/K, theta/E0, Vd_i/E0]      (E0 = 10 Ha)
    h1 = silu(W1 x + b1)   (64)      h2 = silu(W2 h1 + b2)   (64)      o = w3 . h2 + b3
    s_i = tpa_i * exp(o_i)          z_i = s_i r_i
tpa_i is the TPA factor of the column (g_i = KE_i / KE_res).  Vd_i, the potential's diagonal
in mode i, uses the angular mean Vbar(r_p) of V:  Vd_i = (2 pi tau / Ncyc) sum_p w_p
xi_{n,k}(r_p)^2 Vbar(r_p)  (exact for the (m,n)-diagonal of B^H W diag(V) B).
Loss per column (scale invariant, as LOBPCG is):
    loss = 1 - |<z, e>|^2 / (||z||^2 ||e||^2)
with e the target correction direction of the column.
"""
from __future__ import annotations

import numpy as np

E0 = 10.0
HIDDEN = 64
NIN = 6


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    sg = 1.0 / (1.0 + np.exp(-x))
    return sg * (1.0 + x * (1.0 - sg))


def bf16_round(a):
    """Round FP32/FP64 values to bfloat16 (round to nearest even) and return them as FP64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def potential_diagonal(kp, V):
    """Vd_i for every kept mode of the k-point (angular mean of V at each radial node)."""
    b = kp.basis
    Vbar = np.asarray(V).mean(axis=(0, 1))
    out = np.empty(kp.L)
    for i, (n, k) in enumerate(zip(kp.n, kp.k)):
        xi = b.Rtab[n][:, k]
        out[i] = 2 * np.pi * b.tau / b.ncyc * np.sum(b.wr * xi * xi * Vbar)
    return out


def features(kp, vdiag, theta):
    b = kp.basis
    L = kp.L
    X = np.empty((L, NIN))
    X[:, 0] = kp.ke / E0
    X[:, 1] = (kp.m - kp.eta) / max(b.M, 1)
    X[:, 2] = (kp.n * b.ncyc - kp.nu) / max(b.N, 1)
    X[:, 3] = kp.k / max(b.K, 1)
    X[:, 4] = theta / E0
    X[:, 5] = vdiag / E0
    return X


def tpa_factor(ke, r):
    w = np.abs(r) ** 2
    ke_res = (ke @ w) / max(w.sum(), 1e-300)
    g = ke / ke_res
    P = 27 + 18 * g + 12 * g ** 2 + 8 * g ** 3
    return P / (P + 16 * g ** 4)


def forward(params, X):
    W1, b1, W2, b2, w3, b3 = params
    a1 = X @ W1.T + b1
    h1 = silu(a1)
    a2 = h1 @ W2.T + b2
    h2 = silu(a2)
    o = h2 @ w3 + b3
    return o, (X, a1, h1, a2, h2)


def column_loss_and_grad(params, X, tpa, r, e):
    """Loss of one column and gradients w.r.t. (W1, b1, W2, b2, w3, b3)."""
    W1, b1, W2, b2, w3, b3 = params
    o, (X, a1, h1, a2, h2) = forward(params, X)
    s = tpa * np.exp(o)
    A = np.sum(s * np.conj(r) * e)            # <z, e>
    Bn = np.sum(s * s * np.abs(r) ** 2)        # ||z||^2
    Cn = np.sum(np.abs(e) ** 2)
    loss = 1.0 - abs(A) ** 2 / (Bn * Cn)
    # d loss / d s_i
    dA2 = 2.0 * np.real(np.conj(A) * np.conj(r) * e)
    dB = 2.0 * s * np.abs(r) ** 2
    ds = -(dA2 * Bn - abs(A) ** 2 * dB) / (Bn * Bn * Cn)
    do = ds * s                                 # s = tpa exp(o)
    gw3 = h2.T @ do
    gb3 = np.sum(do)
    dh2 = np.outer(do, w3)
    da2 = dh2 * dsilu(a2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    dh1 = da2 @ W2
    da1 = dh1 * dsilu(a1)
    gW1 = da1.T @ X
    gb1 = da1.sum(axis=0)
    return loss, (gW1, gb1, gW2, gb2, gw3, np.array(gb3))


def init_params(seed=0):
    """Small random weights and a zero last layer (the network starts as the TPA diagonal)."""
    g = np.random.default_rng(seed)
    W1 = g.standard_normal((HIDDEN, NIN)) * np.sqrt(2.0 / NIN)
    b1 = np.zeros(HIDDEN)
    W2 = g.standard_normal((HIDDEN, HIDDEN)) * np.sqrt(2.0 / HIDDEN)
    b2 = np.zeros(HIDDEN)
    w3 = np.zeros(HIDDEN)
    b3 = np.zeros(1)
    return [W1, b1, W2, b2, w3, b3]
