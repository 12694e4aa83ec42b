"""Oracle: Cartesian gradient of a function expressed in helical waves (Appendix C).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64.

For E = sum_Gamma Ehat_{m,n,k} F_{m,n,k} (eq. E_expanded_in_basis_set):
  * E_theta1, E_theta2 are the inverse basis transforms of (i 2 pi m) Ehat and (i 2 pi n Ncyc) Ehat
    (eq. Derivative_of_energy_wrt_theta);
  * E_r is the inverse basis transform of Ehat with the radial functions B_n of eq. B_r in place of
    J_{n Ncyc}(b r / R) (eq. E_r): (b/R)[J_{p-1}(b r/R) - (p R/(b r)) J_p(b r/R)], p = n Ncyc, and
    for the lowest order the equivalent (b/R)[(p R/(b r)) J_p - J_{p+1}] (reading: eq. B_r names
    n = N_max for the exception, the text and eqs. A1/A2 name the order -Ncyc N_max; both forms
    are the same derivative J_p', so the choice only matters for which Bessel orders a table
    holds; the text's order is used);
  * the Cartesian components follow by the chain rule of eq. Cartesian_Derivatives with
    vartheta = 2 pi (alpha theta1 + theta2):
        E_x = -sin(vartheta)/(2 pi r) E_theta2 + cos(vartheta) E_r,
        E_y =  cos(vartheta)/(2 pi r) E_theta2 + sin(vartheta) E_r,
        E_z = (E_theta1 - alpha E_theta2) / tau.
Grid arrays are [i, j, p] (eq. wavefun_storage_real order), as in oracle.transforms.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from . import transforms


def btable(basis, n):
    """c_{n,k} B_n(r_p) for every radial node p and k (N_r x K), eq. B_r times the normalisation
    of eq. Basis_fun_derived."""
    p = n * basis.ncyc
    zs = basis.zeros[abs(n)]
    c = math.sqrt(basis.ncyc / (math.pi * basis.tau)) / (basis.R * special.jv(p + 1, zs))
    q = np.outer(basis.r / basis.R, zs)                 # b r / R, [Nr, K]
    ratio = p / q                                       # p R / (b r)
    if n == -basis.N:
        B = (zs / basis.R) * (ratio * special.jv(p, q) - special.jv(p + 1, q))
    else:
        B = (zs / basis.R) * (special.jv(p - 1, q) - ratio * special.jv(p, q))
    return B * c[None, :]


def helical_derivatives(basis, Ebox):
    """(E_theta1, E_theta2, E_r) on the grid for box coefficients Ebox (shape box_shape)."""
    m = np.arange(-basis.M, basis.M + 1)[:, None, None]
    n = np.arange(-basis.N, basis.N + 1)[None, :, None]
    E1 = transforms.fast_inverse(basis, (2j * np.pi * m) * Ebox)
    E2 = transforms.fast_inverse(basis, (2j * np.pi * basis.ncyc * n) * Ebox)
    Er = transforms.fast_inverse(basis, Ebox, {nn: btable(basis, nn) for nn in range(-basis.N, basis.N + 1)})
    return E1, E2, Er


def cartesian_gradient(basis, Ebox):
    """(E_x, E_y, E_z) on the grid (eq. Cartesian_Derivatives)."""
    E1, E2, Er = helical_derivatives(basis, Ebox)
    th1, th2 = basis.theta_grid()
    T1, T2, RR = np.meshgrid(th1, th2, basis.r, indexing="ij")
    ang = 2 * np.pi * (basis.alpha * T1 + T2)
    Ex = -np.sin(ang) / (2 * np.pi * RR) * E2 + np.cos(ang) * Er
    Ey = np.cos(ang) / (2 * np.pi * RR) * E2 + np.sin(ang) * Er
    Ez = (E1 - basis.alpha * E2) / basis.tau
    return Ex, Ey, Ez


def gradient(kp, Ec):
    """Cartesian gradient of the function with compact coefficients Ec at k-point kp (the
    mask only selects which coefficients exist; no Bloch phase is applied)."""
    return cartesian_gradient(kp.basis, kp.to_box(Ec).reshape(kp.basis.box_shape))
