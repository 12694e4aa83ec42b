"""Oracle: synthetic local potential on the helical grid.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper uses empirical pseudopotentials (Sec. "Description of Physical System") that are not
reproduced here; the stand-in is a sum of Gaussian wells placed on the atoms of a structure
generated by the symmetry group G of eq. symm_opera / eq. sim_atoms:

    V(x) = sum_atoms sum_{zeta, mu} -Z exp(-|x - Upsilon_{zeta,mu} x_a|^2 / (2 sigma^2))

with Upsilon_{zeta,mu} = rotation by 2 pi zeta alpha + mu 2pi/Ncyc about e_Z followed by the
translation zeta tau e_Z.  By construction V obeys eq. Potential_Symmetry.  Images are kept
while |z - z_image| <= 10 sigma (every image within 10 sigma in 3-D is then included; the
terms dropped are below exp(-50)).

Grid points (theta1_i, theta2_j, r_p) map to cylindrical coordinates by inverting
eq. coordinates_conversion: z = tau theta1, vartheta = 2 pi (theta2 + alpha theta1).
Atoms are given in cylindrical coordinates (r_a, vartheta_a, z_a) with charge Z and width sigma.
The returned array has shape (N_th1, N_th2, N_r), which flattened in C order is the real-space
storage order of eq. wavefun_storage_real (theta1 slowest, r fastest).
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_wells(basis, atoms: np.ndarray) -> np.ndarray:
    """V on the whole helical grid, shape (N_th1, N_th2, N_r)."""
    th1, th2 = basis.theta_grid()
    T1, T2, RR = np.meshgrid(th1, th2, basis.r, indexing="ij")
    return well_sum(basis, atoms, T1, T2, RR)


def gaussian_wells_at(basis, atoms: np.ndarray, i, j, p) -> np.ndarray:
    """V at the grid points (theta1_i, theta2_j, r_p) only (integer index arrays of one shape)."""
    th1, th2 = basis.theta_grid()
    return well_sum(basis, atoms, th1[np.asarray(i)], th2[np.asarray(j)], basis.r[np.asarray(p)])


def well_sum(basis, atoms, T1, T2, RR):
    """The image sum of eq. sim_atoms evaluated at helical coordinates (T1, T2, RR) (arrays of one
    shape): z = tau theta1, vartheta = 2 pi (theta2 + alpha theta1)."""
    atoms = np.asarray(atoms, dtype=np.float64).reshape(-1, 5)
    z = basis.tau * T1
    vth = 2 * np.pi * (T2 + basis.alpha * T1)
    V = np.zeros_like(z)
    Theta = 2 * np.pi / basis.ncyc
    for ra, tha, za, Z, sig in atoms:
        cut = 10.0 * sig
        # all zeta whose image z_a + zeta tau can come within cut of z in [0, tau)
        zlo = math.floor((0.0 - cut - za) / basis.tau) - 1
        zhi = math.ceil((basis.tau + cut - za) / basis.tau) + 1
        for zeta in range(zlo, zhi + 1):
            zi = za + zeta * basis.tau
            dz = z - zi
            sel = np.abs(dz) <= cut
            if not sel.any():
                continue
            for mu in range(basis.ncyc):
                ang = tha + 2 * np.pi * zeta * basis.alpha + mu * Theta
                d2 = RR ** 2 + ra ** 2 - 2 * RR * ra * np.cos(vth - ang) + dz ** 2
                V += np.where(sel, -Z * np.exp(-d2 / (2 * sig * sig)), 0.0)
    return V
