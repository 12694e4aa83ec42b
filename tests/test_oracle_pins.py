"""Pins of the CPU oracle to facts fixed by the paper and by mathematics, not by the oracle itself.

Each test targets a plausible mistake: a wrong Bessel zero or normalisation, a wrong quadrature
rule, a flipped twist sign, a transposed angular array, a wrong exponent sign, a dropped term of
the reciprocal-space diagonal, a wrong forward-transform weight.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import basis as B
from oracle import eigensolver as E
from oracle import hamiltonian as Hm
from oracle import potential as P
from oracle import transforms as T
from paper_2210_12252_gb300 import inputs


def make_basis(R=6.0, tau=3.0, alpha=0.1, Nr=24, Nth1=16, Nth2=16, ncyc=1, s=4):
    return B.Basis(R, tau, alpha, Nr, Nth1, Nth2, ncyc, s)


# ------------------------------------------------------------------------- Bessel zeros

@pytest.mark.parametrize("p", [0, 1, 3, 7, 11, 23])
def test_bessel_zeros_match_library_routine_and_are_roots(p):
    z = B.bessel_zeros(p, 48)
    ref = special.jn_zeros(p, 48)                       # independent library routine
    np.testing.assert_allclose(z, ref, rtol=2e-14, atol=0)
    assert np.all(np.abs(special.jv(p, z)) < 1e-13)


def test_bessel_zeros_interlace():
    # b_k^p < b_k^{p+1} < b_{k+1}^p
    for p in range(0, 12):
        a = B.bessel_zeros(p, 20)
        b = B.bessel_zeros(p + 1, 20)
        assert np.all(a < b)
        assert np.all(b[:-1] < a[1:])


def test_bessel_zeros_mcmahon_asymptotics():
    # b_k^p ~ (k + p/2 - 1/4) pi - (4p^2 - 1) / (8 (k + p/2 - 1/4) pi) for k >> p
    p = 2
    z = B.bessel_zeros(p, 200)
    k = np.arange(1, 201)
    beta = (k + p / 2 - 0.25) * np.pi
    mc = beta - (4 * p * p - 1) / (8 * beta)
    assert abs(z[-1] - mc[-1]) < 1e-6


# --------------------------------------------------------------------- Gauss-Jacobi rule

@pytest.mark.parametrize("n", [6, 24, 96, 192])
def test_gauss_jacobi_exact_on_polynomials(n):
    x, w = B.gauss_jacobi_01(n)
    for j in range(0, 2 * n, max(1, n // 8)):
        # int_{-1}^{1} (1+x) x^j dx in closed form
        exact = (1 - (-1) ** (j + 1)) / (j + 1) + (1 - (-1) ** (j + 2)) / (j + 2)
        assert abs(np.sum(w * x ** j) - exact) < 1e-13 * max(1.0, abs(exact)) + 1e-14


def test_gauss_jacobi_matches_library_routine():
    x, w = B.gauss_jacobi_01(40)
    xr, wr = special.roots_jacobi(40, 0.0, 1.0)
    np.testing.assert_allclose(x, xr, atol=1e-14)
    np.testing.assert_allclose(w, wr, rtol=1e-12, atol=1e-16)


def test_radial_weights_integrate_r_dr():
    R = 7.5
    r, wr = B.radial_grid(R, 30)
    assert np.all((r > 0) & (r < R)) and np.all(np.diff(r) > 0)
    # int_0^R r^2 * r dr = R^4/4
    assert abs(np.sum(wr * r ** 2) - R ** 4 / 4) < 1e-11 * R ** 4


# ------------------------------------------------------------------ basis functions

def test_xi_negative_order_equals_positive_order():
    b = make_basis()
    for n in range(1, b.N + 1):
        np.testing.assert_allclose(b.Rtab[-n], b.Rtab[n], rtol=1e-13, atol=1e-15)


def test_xi_normalisation_against_adaptive_quadrature():
    # (2 pi tau / Ncyc) int_0^R xi_{n,k}(r)^2 r dr = 1 (Appendix B), by adaptive quadrature
    b = make_basis()
    for n, k in [(0, 0), (2, 3), (-3, 5)]:
        val, _ = integrate.quad(lambda r: b.xi(n, k, r) ** 2 * r, 0, b.R, limit=200,
                                epsabs=1e-14, epsrel=1e-13)
        assert abs(2 * np.pi * b.tau / b.ncyc * val - 1.0) < 1e-11


def test_orthonormality_under_radial_quadrature():
    for s, bound in [(4, 1e-12)]:
        b = make_basis(s=s)
        for n in range(-b.N, b.N + 1):
            G = (2 * np.pi * b.tau / b.ncyc) * b.Otab[n] @ b.Rtab[n]
            assert np.abs(G - np.eye(b.K)).max() < bound
    # the tube geometry (N_r = 96, K = 24)
    g = inputs.GEOM_TUBE
    b = make_basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2)
    for n in range(-b.N, b.N + 1):
        G = (2 * np.pi * b.tau) * b.Otab[n] @ b.Rtab[n]
        assert np.abs(G - np.eye(b.K)).max() < 1e-13


@pytest.mark.parametrize("alpha", [0.1, -0.07])
def test_basis_functions_are_laplacian_eigenfunctions_in_cartesian_coordinates(alpha):
    """-Delta F = lambda^0 F (eq. Laplacian_of_f_mnk), with Delta the Cartesian Laplacian
    evaluated by 4th-order finite differences of F(x(theta), ...) through the helical
    coordinate map (eq. coordinates_conversion).  Pins lambda^0 including the twist sign."""
    b = make_basis(alpha=alpha)
    rng = np.random.default_rng(3)

    def Fcart(m, n, k, x, y, z):
        r = np.hypot(x, y)
        th1 = z / b.tau
        th2 = np.arctan2(y, x) / (2 * np.pi) - b.alpha * z / b.tau
        return b.F(m, n, k, th1, th2, r)

    h = 2e-3
    c = np.array([-1, 16, -30, 16, -1]) / (12 * h * h)
    offs = np.array([-2, -1, 0, 1, 2]) * h
    for (m, n, k) in [(0, 0, 0), (2, -1, 3), (-3, 2, 1), (1, 3, 5)]:
        for _ in range(3):
            rr = rng.uniform(1.0, 5.0)
            ph = rng.uniform(0, 2 * np.pi)
            x, y, z = rr * np.cos(ph), rr * np.sin(ph), rng.uniform(0, 3)
            lap = 0
            for d in range(3):
                pts = np.array([x, y, z])[:, None] + np.eye(3)[:, d:d + 1] * offs[None, :]
                lap = lap + np.sum(c * Fcart(m, n, k, *pts))
            F0 = Fcart(m, n, k, x, y, z)
            lam = b.lambda0(np.array(m), np.array(n), np.array(k))
            assert abs(-lap - lam * F0) < 1e-6 * max(1.0, abs(lam)) * max(abs(F0), 1e-3)


# ------------------------------------------------------------------------ transforms

def test_fast_transforms_equal_naive_sums():
    b = make_basis()
    rng = np.random.default_rng(0)
    gh = rng.standard_normal(b.box_shape) + 1j * rng.standard_normal(b.box_shape)
    g1 = T.naive_inverse(b, gh)
    g2 = T.fast_inverse(b, gh)
    assert np.abs(g1 - g2).max() < 1e-13 * np.abs(g1).max()
    f1 = T.naive_forward(b, g1)
    f2 = T.fast_forward(b, g1)
    assert np.abs(f1 - f2).max() < 1e-13 * np.abs(f1).max()


def test_transform_round_trip_is_identity_on_band_limited_functions():
    b = make_basis()
    rng = np.random.default_rng(1)
    gh = rng.standard_normal(b.box_shape) + 1j * rng.standard_normal(b.box_shape)
    back = T.fast_forward(b, T.fast_inverse(b, gh))
    assert np.abs(back - gh).max() < 1e-11


def test_inverse_transform_of_one_mode_is_that_basis_function():
    # a single coefficient (m, n, k) must give F_{m,n,k} on the grid: pins bin placement and
    # the +i exponent sign of Algorithm 2 (a transposed angular array fails when m != n)
    b = make_basis()
    th1, th2 = b.theta_grid()
    T1, T2, RR = np.meshgrid(th1, th2, b.r, indexing="ij")
    for (m, n, k) in [(2, -1, 0), (-3, 1, 4)]:
        gh = np.zeros(b.box_shape, complex)
        gh[m + b.M, n + b.N, k] = 1.0
        g = T.fast_inverse(b, gh)
        ref = np.exp(2j * np.pi * (m * T1 + n * T2)) * b.xi(n, k, RR)
        assert np.abs(g - ref).max() < 1e-13


# ----------------------------------------------------------------- reciprocal diagonal

def test_literal_abc_diagonal_equals_closed_form():
    """1/2 Lambda - a - b M - c N (Algorithm 5) = 1/2[(b/R)^2 + (2pi/tau)^2 (m-eta-alpha(nNcyc-nu))^2]."""
    for ncyc, nu in [(1, 0.0), (3, 1.0), (4, 2.0)]:
        b = make_basis(ncyc=ncyc)
        m, n, k = b.box_mnk()
        for eta in [0.0, 0.3, -0.45]:
            lit = b.diagonal_literal(eta, nu)
            assert np.abs(lit.imag).max() == 0.0
            bz = np.array([b.bzero(nn, kk) for nn, kk in zip(n, k)])
            closed = 0.5 * ((bz / b.R) ** 2 + (2 * np.pi / b.tau) ** 2 *
                            (m - eta - b.alpha * (n * ncyc - nu)) ** 2)
            np.testing.assert_allclose(lit.real, closed, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------------------- Hamiltonian

def test_zero_potential_gives_closed_form_eigenvalues(tiny_case):
    w, b, _ = tiny_case
    V0 = np.zeros((b.Nth1, b.Nth2, b.Nr))
    for eta, ecut in [(0.0, 0.0), (0.27, 8.0)]:
        kp = B.KPoint(b, eta, 0.0, ecut)
        H = Hm.dense_H(kp, V0)
        assert np.abs(H - np.diag(np.diag(H))).max() == 0.0
        ev = np.linalg.eigvalsh(H)
        m, n, k = kp.m, kp.n, kp.k
        bz = np.array([b.bzero(nn, kk) for nn, kk in zip(n, k)])
        closed = np.sort(0.5 * ((bz / b.R) ** 2 +
                                (2 * np.pi / b.tau * (m - eta - b.alpha * n)) ** 2))
        np.testing.assert_allclose(ev, closed, rtol=1e-14, atol=1e-14)


def test_hamiltonian_is_hermitian_and_conv_form_matches_algorithm5(tiny_case):
    w, b, V = tiny_case
    kp = B.KPoint(b, 0.13, 0.0, 6.0)
    H = Hm.dense_H(kp, V)
    assert np.abs(H - H.conj().T).max() <= 1e-14 * np.abs(H).max()
    Hc = Hm.dense_H_conv(kp, V)
    assert np.abs(H - Hc).max() <= 1e-13 * np.abs(H).max()


def test_constant_shift_of_potential_shifts_every_eigenvalue(tiny_case):
    w, b, V = tiny_case
    kp = B.KPoint(b, 0.0, 0.0, 0.0)
    e0 = np.linalg.eigvalsh(Hm.dense_H(kp, V))
    c = 1.7
    e1 = np.linalg.eigvalsh(Hm.dense_H(kp, V + c))
    assert np.abs(e1 - e0 - c).max() < 1e-11


def test_theta1_cosine_potential_couples_m_to_m_plus_minus_one_exactly():
    """V = v cos(2 pi theta1 + phi): <F_{m',n,k'}, V F_{m,n,k}> = v/2 e^{+-i phi} delta_{m', m+-1}
    delta_{kk'} (orthogonality of exponentials and radial functions).  Pins the theta1 axis,
    the exponent signs and the forward-transform weights."""
    b = make_basis()
    v, phi = 0.8, 0.6
    th1, th2 = b.theta_grid()
    T1 = th1[:, None, None] + 0 * th2[None, :, None] + 0 * b.r[None, None, :]
    V = v * np.cos(2 * np.pi * T1 + phi)
    kp = B.KPoint(b, 0.1, 0.0, 0.0)
    H = Hm.dense_H(kp, V)
    ref = np.diag(kp.ke.astype(complex))
    pos = {(mm, nn, kk): i for i, (mm, nn, kk) in enumerate(zip(kp.m, kp.n, kp.k))}
    for i, (mm, nn, kk) in enumerate(zip(kp.m, kp.n, kp.k)):
        for dm, ph in [(1, np.exp(1j * phi)), (-1, np.exp(-1j * phi))]:
            j = pos.get((mm + dm, nn, kk))
            if j is not None:
                ref[j, i] += 0.5 * v * ph
    assert np.abs(H - ref).max() < 1e-12


def test_theta2_cosine_potential_against_adaptive_radial_overlaps():
    """V = v cos(2 pi Ncyc theta2): couples n -> n+-1 with the radial overlaps
    (2 pi tau/Ncyc) int_0^R xi_{n',k'} xi_{n,k} r dr, here from adaptive quadrature."""
    b = make_basis(Nth2=16)
    v = 0.5
    th1, th2 = b.theta_grid()
    T2 = 0 * th1[:, None, None] + th2[None, :, None] + 0 * b.r[None, None, :]
    V = v * np.cos(2 * np.pi * T2)
    kp = B.KPoint(b, 0.0, 0.0, 0.0)
    H = Hm.dense_H(kp, V)
    pos = {(mm, nn, kk): i for i, (mm, nn, kk) in enumerate(zip(kp.m, kp.n, kp.k))}
    rng = np.random.default_rng(5)
    for _ in range(12):
        m = int(rng.integers(-b.M, b.M + 1))
        n = int(rng.integers(-b.N, b.N))
        k, kq = int(rng.integers(0, b.K)), int(rng.integers(0, b.K))
        val, _ = integrate.quad(lambda r: b.xi(n + 1, kq, r) * b.xi(n, k, r) * r, 0, b.R,
                                limit=200, epsabs=1e-14, epsrel=1e-12)
        expect = 0.5 * v * 2 * np.pi * b.tau * val
        assert abs(H[pos[(m, n + 1, kq)], pos[(m, n, k)]] - expect) < 1e-11


def _radial_fd_eigs(V_of_r, R, order, kz2, nev, npts):
    """Lowest eigenvalues of -1/2 (u'' + u'/r - order^2 u / r^2) + 1/2 kz2 u + V(r) u on (0, R),
    u(R) = 0, by second-order finite differences on a cell-centred grid (symmetrised)."""
    h = R / npts
    r = (np.arange(npts) + 0.5) * h
    rp = r + h / 2
    rm = r - h / 2
    main = (rp + rm) / (r * h * h) * 0.5 + 0.5 * order ** 2 / r ** 2 + 0.5 * kz2 + V_of_r(r)
    off = -0.5 * rp[:-1] / (h * h)
    # the operator is symmetric in the r-weighted inner product: the similarity by sqrt(r)
    # leaves the diagonal and symmetrises the off-diagonal
    s = np.sqrt(r)
    from scipy.linalg import eigh_tridiagonal
    return eigh_tridiagonal(main, off / (s[:-1] * s[1:]), select="i", select_range=(0, nev - 1))[0]


def test_cylindrical_potential_decouples_angular_orders_and_matches_radial_solver():
    """V = V(r): H is block diagonal in (m, n) to machine precision; the lowest eigenvalue of a
    block equals that of the radial ODE of eq. Expanded_schrodinger (Richardson-extrapolated
    finite differences, an independent discretisation) to the discretisation error."""
    b = make_basis(R=6.0, Nr=64, Nth1=16, Nth2=16)          # K = 16 radial modes
    Vr = lambda r: -3.0 * np.exp(-r ** 2 / (2 * 1.5 ** 2))
    V = np.broadcast_to(Vr(b.r)[None, None, :], (b.Nth1, b.Nth2, b.Nr)).copy()
    kp = B.KPoint(b, 0.2, 0.0, 0.0)
    H = Hm.dense_H(kp, V)
    same = (kp.m[:, None] == kp.m[None, :]) & (kp.n[:, None] == kp.n[None, :])
    assert np.abs(H[~same]).max() < 1e-14 * np.abs(H).max()
    for (m, n) in [(0, 0), (1, -2), (-1, 3)]:
        sel = (kp.m == m) & (kp.n == n)
        lam = np.linalg.eigvalsh(H[np.ix_(sel, sel)])[0]
        kz2 = (2 * np.pi / b.tau * (m - kp.eta - b.alpha * n)) ** 2
        e1, e2, e3 = (_radial_fd_eigs(Vr, b.R, n, kz2, 1, npts)[0] for npts in (4000, 8000, 16000))
        # Richardson extrapolation with the observed order (second order for n = 0, first order
        # otherwise because of the n^2/r^2 term next to the axis)
        order = np.log2((e2 - e1) / (e3 - e2))
        rich = e3 + (e3 - e2) / (2 ** order - 1)
        assert abs(lam - rich) < 2e-8, (m, n, lam, rich)


def test_time_reversal_symmetry_of_the_spectrum(tiny_case):
    """lambda_j(eta, 0) = lambda_j(-eta, 0) (Sec. eta-space discretization), with the cutoff."""
    w, b, V = tiny_case
    for eta in [0.17, 0.41]:
        e_p = np.linalg.eigvalsh(Hm.dense_H(B.KPoint(b, eta, 0.0, 9.0), V))
        e_m = np.linalg.eigvalsh(Hm.dense_H(B.KPoint(b, -eta, 0.0, 9.0), V))
        assert e_p.size == e_m.size
        assert np.abs(e_p - e_m).max() < 1e-12


def test_potential_is_helically_invariant():
    """eq. Potential_Symmetry: V is periodic in theta1 (shift by 1 = the screw operation);
    evaluate the well sum on a grid shifted by one period."""
    b = make_basis()
    w = inputs.tiny()
    V = P.gaussian_wells(b, w.atoms)
    atoms = w.atoms.copy()
    atoms[:, 2] += b.tau              # the atoms' images are the same set
    atoms[:, 1] += 2 * np.pi * b.alpha
    V2 = P.gaussian_wells(b, atoms)
    assert np.abs(V - V2).max() < 1e-12


# ----------------------------------------------------------------------- eigensolver

def test_tpa_formula_values():
    ke = np.array([0.0, 1.0, 2.0, 50.0])
    R = np.ones((4, 1), complex)
    Z = E.tpa(ke, R)[:, 0].real
    g = ke / ke.mean()
    Pg = 27 + 18 * g + 12 * g ** 2 + 8 * g ** 3
    np.testing.assert_allclose(Z, Pg / (Pg + 16 * g ** 4), rtol=1e-15)
    assert Z[0] == 1.0
    # g = 1 gives 65/81
    assert abs(E.tpa(np.array([3.0]), np.ones((1, 1)))[0, 0] - 65 / 81) < 1e-15


def test_tpa_weights_the_residual_kinetic_energy_by_r_squared():
    """Reading 9 of the TPA (Sec. "Eigensolvers and Preconditioning"): KE_res is the
    |r_i|^2-weighted mean of KE_i.  Worked by hand for KE = (1, 2, 4):
      column 0, |r|^2 = (2, 1, 1): KE_res = (2 + 2 + 4) / 4 = 2, so g = (1/2, 1, 2) and
        P(1/2) = 27 + 9 + 3 + 1 = 40,         16 g^4 = 1    -> K = 40/41
        P(1)   = 27 + 18 + 12 + 8 = 65,        16 g^4 = 16   -> K = 65/81
        P(2)   = 27 + 36 + 48 + 64 = 175,      16 g^4 = 256  -> K = 175/431
      column 1, r = (0, 0, 1): KE_res = 4, g = (1/4, 1/2, 1): only the third entry is
        nonzero, scaled by 65/81.
    A |r|-weighted mean gives KE_res = (sqrt2 + 2 + 4)/(sqrt2 + 2) = 2.17 for column 0, an
    unweighted one 7/3; both move every scale of column 0 by more than 1e-3."""
    ke = np.array([1.0, 2.0, 4.0])
    r0 = np.array([np.sqrt(2.0) * np.exp(0.25j * np.pi), -1.0, 1j])
    r1 = np.array([0.0, 0.0, 0.5 - 0.5j])
    Z = E.tpa(ke, np.stack([r0, r1], axis=1))
    np.testing.assert_allclose(Z[:, 0], np.array([40 / 41, 65 / 81, 175 / 431]) * r0, rtol=1e-14, atol=0)
    np.testing.assert_allclose(Z[:, 1], np.array([0.0, 0.0, 65 / 81]) * r1, rtol=1e-14, atol=0)
    # the other two readings of "kinetic energy of the residual vector" fail this pin
    for w in (np.abs(r0), np.ones(3)):
        ke_res = (ke * w).sum() / w.sum()
        g = ke / ke_res
        Pg = 27 + 18 * g + 12 * g ** 2 + 8 * g ** 3
        assert np.abs(Pg / (Pg + 16 * g ** 4) - np.array([40 / 41, 65 / 81, 175 / 431])).max() > 1e-3


def test_lobpcg_matches_direct_diagonalisation(tiny_case):
    w, b, V = tiny_case
    kp = B.KPoint(b, 0.0, 0.0, 0.0)
    H = Hm.dense_H(kp, V)
    ev = np.linalg.eigvalsh(H)
    X0 = inputs.random_block(kp.L, 12, 11)
    th, X, it, res = E.lobpcg(lambda X: H @ X, kp.ke, X0, 8, tol=1e-9)
    assert np.abs(th - ev[:8]).max() < 1e-12
    assert res[:8].max() <= 1e-9


def test_potential_at_points_equals_the_grid_potential(tiny_case):
    """gaussian_wells_at (used to check the nanowire's 300-well potential at sampled points) is
    the same image sum as the full-grid gaussian_wells."""
    w, b, V = tiny_case
    g = np.random.default_rng(3)
    i, j, p = (g.integers(0, n, 200) for n in (b.Nth1, b.Nth2, b.Nr))
    np.testing.assert_allclose(P.gaussian_wells_at(b, w.atoms, i, j, p), V[i, j, p], rtol=1e-13,
                               atol=1e-15 * np.abs(V).max())
