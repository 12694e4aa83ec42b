"""Pins of the oracle's Cartesian gradients (Appendix C) to facts outside the oracle.

Each test targets a plausible mistake: a wrong B_n table (a dropped p/q term, a wrong order or
normalisation: the closed-form derivative of one basis function via scipy's J_p'), a wrong sign,
factor or angle in the chain rule or a swapped theta1/theta2 (central finite differences of the
directly summed function in Cartesian coordinates).
"""
import math

import numpy as np
import pytest
from scipy import special

from oracle import basis as B
from oracle import gradient as Gr
from paper_2210_12252_gb300 import inputs


def make_basis(ncyc=1, alpha=0.1, Nr=16, Nth=12):
    return B.Basis(6.0, 3.0, alpha, Nr, Nth, Nth, ncyc, 4)


@pytest.mark.parametrize("ncyc", [1, 3])
def test_radial_derivative_of_one_basis_function_is_bessel_derivative(ncyc):
    """E = F_{m,n,k}: E_r = c (b/R) J_p'(b r/R) e^{i 2 pi (m theta1 + n Ncyc theta2)} with J_p' from
    scipy.special.jvp, for every n including the lowest order (the alternative form of eq. B_r)."""
    b = make_basis(ncyc=ncyc)
    th1, th2 = b.theta_grid()
    T1, T2, RR = np.meshgrid(th1, th2, b.r, indexing="ij")
    for (m, n, k) in [(1, -b.N, 0), (0, 0, 2), (-2, 1, 1), (2, b.N, b.K - 1)]:
        E = np.zeros(b.box_shape, complex)
        E[m + b.M, n + b.N, k] = 1.0
        _, _, Er = Gr.helical_derivatives(b, E)
        p = n * ncyc
        z = b.bzero(n, k)
        c = math.sqrt(ncyc / (math.pi * b.tau)) / (b.R * special.jv(p + 1, z))
        ref = c * (z / b.R) * special.jvp(p, z * RR / b.R) * np.exp(2j * np.pi * (m * T1 + n * ncyc * T2))
        assert np.abs(Er - ref).max() < 1e-12 * np.abs(ref).max()


def _direct(b, Ebox, x, y, z):
    """sum_Gamma Ehat F at one Cartesian point: theta1 = z/tau, vartheta = atan2(y, x),
    theta2 = vartheta/(2 pi) - alpha theta1, r = hypot(x, y) (eq. coordinates_conversion)."""
    t1 = z / b.tau
    t2 = math.atan2(y, x) / (2 * math.pi) - b.alpha * t1
    r = math.hypot(x, y)
    m, n, k = b.box_mnk()
    vals = Ebox.ravel()
    sel = np.nonzero(vals)[0]
    tot = 0.0j
    for i in sel:
        tot += vals[i] * b.F(m[i], n[i], k[i], t1, t2, r)
    return tot


@pytest.mark.parametrize("ncyc,alpha", [(1, 0.1), (3, 0.23)])
def test_cartesian_gradient_matches_finite_differences(ncyc, alpha):
    b = make_basis(ncyc=ncyc, alpha=alpha)
    rng = np.random.default_rng(11 + ncyc)
    E = np.zeros(b.box_shape, complex)
    # a band-limited random function (a few dozen modes keep the direct sums fast)
    idx = rng.choice(E.size, 40, replace=False)
    E.ravel()[idx] = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    Ex, Ey, Ez = Gr.cartesian_gradient(b, E)
    th1, th2 = b.theta_grid()
    h = 1e-5
    for (i, j, p) in [(0, 0, 3), (5, 7, 8), (11, 2, 12), (3, 9, 0)]:
        t1, t2, r = th1[i], th2[j], b.r[p]
        ang = 2 * math.pi * (b.alpha * t1 + t2)
        x, y, z = r * math.cos(ang), r * math.sin(ang), b.tau * t1
        fd = [(_direct(b, E, x + h, y, z) - _direct(b, E, x - h, y, z)) / (2 * h),
              (_direct(b, E, x, y + h, z) - _direct(b, E, x, y - h, z)) / (2 * h),
              (_direct(b, E, x, y, z + h) - _direct(b, E, x, y, z - h)) / (2 * h)]
        got = [Ex[i, j, p], Ey[i, j, p], Ez[i, j, p]]
        scale = max(abs(v) for v in fd)
        for a, bb in zip(got, fd):
            assert abs(a - bb) < 1e-6 * scale, (i, j, p, a, bb)
