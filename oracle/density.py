"""Oracle: electron density on the real-space grid from converged states.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. "Convergence Studies" (the electron-density equation): for every k-point b (weight w_b,
the Monkhorst-Pack weights 1/N_eta of Sec. "eta-space discretization") and every state j with
occupation s_j(eta_b, nu),

    rho(theta1, theta2, r) = (2 / Ncyc) sum_j sum_b sum_nu w_b s_j(eta_b, nu) |phi_j(theta1, theta2, r)|^2,

where phi_j is the inverse basis transform (eq. Naive_Inverse_Transform, computed by
Algorithms 1-2) of the state's coefficient vector.  nu = 0 only (as everywhere in this oracle),
so the sum over nu has the single term nu = 0 and 1/Ncyc times the Ncyc-fold sum over nu is
read as the nu = 0 term with the factor 2 / Ncyc kept as printed.  The helical Bloch phase has
modulus one and drops out of |phi|^2.

Output array: real, shape (N_th1, N_th2, N_r) indexed [i, j, p] (eq. wavefun_storage_real when
flattened in C order), like the potential.
"""
from __future__ import annotations

import numpy as np

from . import transforms as T


def density(kpoints, states, occ, weights, naive=False):
    """kpoints: list of KPoint; states[b]: (L_b, ns) compact coefficient blocks; occ[b]: (ns,)
    occupations; weights[b]: k-point weight w_b."""
    b0 = kpoints[0].basis
    rho = np.zeros((b0.Nth1, b0.Nth2, b0.Nr))
    inv = T.naive_inverse if naive else T.fast_inverse
    for kp, X, s, wb in zip(kpoints, states, occ, weights):
        X = np.asarray(X)
        for j in range(X.shape[1]):
            if s[j] == 0:
                continue
            phi = inv(kp.basis, kp.to_box(X[:, j]).reshape(kp.basis.box_shape))
            rho += wb * s[j] * np.abs(phi) ** 2
    return (2.0 / b0.ncyc) * rho


def charge(basis, rho):
    """Quadrature of rho over the fundamental domain with the weights of the forward transform
    (eq. Fast_fwd_transform_cont): 2 pi tau / Ncyc * sum w_r / (N_th1 N_th2)."""
    W = basis.wr[None, None, :] / (basis.Nth1 * basis.Nth2)
    return 2 * np.pi * basis.tau / basis.ncyc * float(np.sum(rho * W))
