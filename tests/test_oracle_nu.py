"""Pins of the oracle's nu != 0 terms (cyclic symmetry Ncyc > 1, cyclic wavenumber nu != 0):
the table I(n, k, k') of eq. I_nkk_prime and the I_n loop of Algorithm 5.

Each test targets a plausible mistake: a dropped 1/q or a wrong normalisation of the table (the
integration-by-parts identity), a wrong factor or sign in either of the two 1/r^2 terms (exact
cancellation at nu = 2 n Ncyc; convergence of the V = 0 spectrum to the Bessel zeros of order
|n Ncyc - nu|), a mistake in either assembly route (columns through Algorithm 5 vs the
written-out matrix).
"""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import basis as B
from oracle import hamiltonian as Hm
from oracle import potential as P
from paper_2210_12252_gb300 import inputs


def make_basis(R=6.0, tau=3.0, alpha=0.1, Nr=24, Nth1=16, Nth2=16, ncyc=3, s=4):
    return B.Basis(R, tau, alpha, Nr, Nth1, Nth2, ncyc, s)


@pytest.mark.parametrize("ncyc,n", [(1, 1), (3, 1), (3, -1), (3, 2), (2, 3)])
def test_itable_matches_integration_by_parts(ncyc, n):
    """For u = J_p(a q), v = J_p(b q) with a, b zeros of J_p, Bessel's equation and one
    integration by parts give p^2 int_0^1 u v / q dq = a^2 int_0^1 q u v dq - a b int_0^1 q
    J_p'(a q) J_p'(b q) dq, and int_0^1 q u v dq = delta_ab J_{p+1}(a)^2 / 2.  The derivative
    integral is taken by adaptive quadrature (scipy.integrate.quad), a route that shares nothing
    with the table's Gauss-Legendre sum of J J / q."""
    b = make_basis(ncyc=ncyc)
    p = abs(n * ncyc)
    I = b.itable(n)
    z = b.zeros[abs(n)]
    jp1 = special.jv(p + 1, z)
    for k in range(b.K):
        for kk in range(k, b.K):
            d, _ = integrate.quad(lambda q: q * special.jvp(p, z[k] * q) * special.jvp(p, z[kk] * q),
                                  0.0, 1.0, epsabs=1e-14, epsrel=1e-13, limit=200)
            rhs = (z[k] ** 2 * (0.5 * jp1[k] ** 2 if k == kk else 0.0) - z[k] * z[kk] * d) / p ** 2
            # for n < 0 the signed orders of eq. I_nkk_prime give the same value as |p|
            # (J_{-q} = (-1)^q J_q and J_{1-q}(b) = (-1)^q J_{q+1}(b) at a zero b of J_q)
            assert abs(I[k, kk] - rhs / (jp1[k] * jp1[kk])) < 1e-11 * max(1.0, abs(I[k, kk]))


def test_itable_symmetric_and_even_in_n():
    b = make_basis(ncyc=3)
    for n in range(0, b.N + 1):
        I = b.itable(n)
        assert np.abs(I - I.T).max() < 1e-13 * np.abs(I).max()
        np.testing.assert_allclose(b.itable(-n), I, rtol=1e-13, atol=1e-13)


def test_inverse_square_terms_cancel_at_nu_twice_the_order():
    """The I_n loop adds (nu^2/R^2) I Z + (i nu/(pi R^2)) I (i 2 pi n Ncyc Z)
    = (nu^2 - 2 nu n Ncyc)/R^2 I Z, which vanishes in the channel n = nu/(2 Ncyc) and nowhere
    else.  With V = 0 that channel's block stays exactly diagonal (the two terms, with different
    prefactors, cancel), while its mirror channel -n picks up a full I block."""
    b = make_basis(ncyc=1)
    V0 = np.zeros((b.Nth1, b.Nth2, b.Nr))
    eta, nu = 0.15, 2.0                      # n = 1 cancels (a value of nu outside 0..Ncyc-1)
    D = b.diagonal_literal(eta, nu)
    for n, cancels in [(1, True), (-1, False), (2, False)]:
        idx = [b.box_index(0, n, k) for k in range(b.K)]
        E = np.zeros((b.box_size, b.K), complex)
        E[idx, np.arange(b.K)] = 1.0
        Hc = Hm.apply_H_box(b, V0, eta, nu, E)[idx, :]
        off = Hc - np.diag(D[idx])
        if cancels:
            assert np.abs(off).max() < 1e-13 * np.abs(D[idx]).max()
        else:
            assert np.abs(off).max() > 1e-2


@pytest.mark.parametrize("n", [1, -1, 2])
def test_zero_potential_spectrum_approaches_bessel_order_n_ncyc_minus_nu(n):
    """With V = 0 the Bloch state in channel (m, n) has angular order n Ncyc - nu, so the exact
    levels are 1/2[(b_k^{|n Ncyc - nu|}/R)^2 + (2 pi/tau)^2 (m - eta - alpha(n Ncyc - nu))^2].
    The Galerkin block (orders n Ncyc basis functions plus the 1/r^2 terms) approaches them from
    above (Rayleigh-Ritz upper bounds), the error falling as N_r grows.  A sign error in the
    2 nu n Ncyc term sends channel n to order |n Ncyc + nu| instead (an O(1) error)."""
    ncyc, eta, nu, m = 3, 0.2, 1.0, 0
    q = abs(n * ncyc - nu)
    errs = []
    for Nr in (48, 96):
        b = make_basis(Nr=Nr, ncyc=ncyc)
        V0 = np.zeros((b.Nth1, b.Nth2, b.Nr))
        idx = [b.box_index(m, n, k) for k in range(b.K)]
        E = np.zeros((b.box_size, b.K), complex)
        E[idx, np.arange(b.K)] = 1.0
        Hc = Hm.apply_H_box(b, V0, eta, nu, E)[idx, :]
        assert np.abs(Hc - Hc.conj().T).max() < 1e-12 * np.abs(Hc).max()
        w = np.linalg.eigvalsh(Hc)[:3]
        exact = 0.5 * ((special.jn_zeros(int(q), 3) / b.R) ** 2 +
                       (2 * np.pi / b.tau) ** 2 * (m - eta - b.alpha * (n * ncyc - nu)) ** 2)
        rel = (w - exact) / exact
        assert np.all(rel > -1e-12)          # upper bounds
        errs.append(rel)
    assert np.all(errs[1] < errs[0])         # convergence
    # the order-2 target in the order-3 basis (n = 1) converges algebraically, the others fast
    assert errs[0][0] < (1e-3 if n == 1 else 1e-6)


def test_dense_routes_agree_with_nu():
    """Columns H e_j through the literal Algorithm 5 (fast transforms + the I_n loop) equal the
    written-out matrix D + B^H W diag(V) B + (nu^2 - 2 nu n Ncyc)/R^2 (+) I_n, and H is Hermitian."""
    b = make_basis(Nr=16, Nth1=12, Nth2=12, ncyc=3)
    atoms = inputs.ring_atoms(4, 2.5, b.tau, 4.0, 0.8, seed=5)
    V = P.gaussian_wells(b, atoms)
    for eta, nu, ecut in [(0.1, 1.0, 0.0), (-0.3, 2.0, 12.0)]:
        kp = B.KPoint(b, eta, nu, ecut)
        assert kp.n0_quadrature
        H1 = Hm.dense_H(kp, V)
        H2 = Hm.dense_H_conv(kp, V)
        assert np.abs(H1 - H2).max() < 1e-12 * np.abs(H2).max()
        assert np.abs(H1 - H1.conj().T).max() < 1e-12 * np.abs(H1).max()
