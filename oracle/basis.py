"""Oracle: helical-wave basis set, radial quadrature and reciprocal-space bookkeeping.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  FP64 throughout.

Follows arXiv 2210.12252:
  * basis functions F_{m,n,k} and normalisation c_{m,n,k}: Sec. "Basis Set and Discretization",
    eq. Phi_expanded_in_basis_set and the normalisation constant after it; Appendix B,
    eq. Basis_fun_derived;
  * Laplacian eigenvalues lambda^0: eq. Laplacian_of_f_mnk;
  * index set Gamma and the linear order i(m,n,k): eq. wavefun_storage;
  * grids: Sec. "Wave function storage" (Fourier nodes in theta1/theta2, Gauss-Jacobi nodes in r,
    N_theta ~ 4*M_max+1, N_r = 4*K_max);
  * kinetic-energy cutoff and mask: eq. Energy_cutoff and the mask definition after it,
    "modified appropriately" at each (eta, nu);
  * reciprocal-space diagonal terms: eq. constants_abc and Algorithm 5 (the a, b, c terms);
  * the 1/r^2 integrals I(n, k, k'): eq. I_nkk_prime.

Readings taken where the paper is silent (also listed in the design notes):
  R3  the basis box follows from the grids: M = floor((N_th1-1)/s), N = floor((N_th2-1)/s),
      K = floor(N_r/s), with the oversampling s (default 4) of the grid rule above.
  R5  the cutoff kinetic energy at (eta, nu) is 1/2 lambda^0 - a - b(i2pi m) - c(i2pi n Ncyc),
      i.e. exactly the reciprocal-space diagonal of Algorithm 5; the tie is inclusive and a
      relative slack of 1e-12 guards against rounding flips.
  R6  Gauss-Jacobi with (alpha, beta) = (0, 1) on x in [-1, 1], r = R(1+x)/2, and the radial
      weights omega_r = (R^2/4) w absorb the r dr of the inner product.
  I0  for nu != 0 the table I(0, k, k') of eq. I_nkk_prime is a divergent integral (J_0 does not
      vanish at r = 0); it is replaced by its value under the radial rule above, and flagged.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import special

# ----------------------------------------------------------------------------------------
# Bessel zeros b_k^p (the paper does not say how it computes them; Appendix B only needs the
# k-th positive root of J_p).  Bracket by scanning for sign changes, bisect, polish by Newton.
# ----------------------------------------------------------------------------------------


def bessel_zeros(p: int, K: int) -> np.ndarray:
    """First K positive zeros of J_p for an integer order p >= 0 (Appendix B, b_k^p)."""
    if p < 0:
        raise ValueError("use |p|: J_{-p} = (-1)^p J_p has the same zeros")
    zeros = []
    h = 0.05
    x = max(float(p), 0.5)
    fx = special.jv(p, x)
    while len(zeros) < K:
        y = x + h
        fy = special.jv(p, y)
        if fx == 0.0:
            zeros.append(x)
        elif fx * fy < 0.0:
            a, b, fa = x, y, fx
            for _ in range(200):          # bisection to a tight bracket
                c = 0.5 * (a + b)
                fc = special.jv(p, c)
                if fa * fc <= 0.0:
                    b = c
                else:
                    a, fa = c, fc
                if b - a < 1e-13 * max(1.0, abs(a)):
                    break
            z = 0.5 * (a + b)
            for _ in range(3):            # Newton polish, J_p' = (J_{p-1} - J_{p+1}) / 2
                d = 0.5 * (special.jv(p - 1, z) - special.jv(p + 1, z))
                z = z - special.jv(p, z) / d
            zeros.append(z)
        x, fx = y, fy
    return np.array(zeros[:K])


# ----------------------------------------------------------------------------------------
# Gauss-Jacobi (0, 1) rule by Golub-Welsch: eigenvalues of the Jacobi matrix of the monic
# Jacobi polynomials are the nodes, weights = mu_0 * (first eigenvector component)^2.
# ----------------------------------------------------------------------------------------


def gauss_jacobi_01(n: int) -> tuple[np.ndarray, np.ndarray]:
    """Nodes/weights of the n-point rule for int_{-1}^{1} (1+x) f(x) dx (reading R6)."""
    k = np.arange(n, dtype=np.float64)
    # recurrence coefficients of the monic P_k^{(0,1)}: diagonal 1/((2k+1)(2k+3)),
    # off-diagonal sqrt(k(k+1))/(2k+1) for k >= 1
    diag = 1.0 / ((2 * k + 1) * (2 * k + 3))
    kk = np.arange(1, n, dtype=np.float64)
    off = np.sqrt(kk * (kk + 1)) / (2 * kk + 1)
    J = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(J)
    w = 2.0 * V[0, :] ** 2          # mu_0 = int (1+x) dx = 2
    return x, w


def radial_grid(R: float, Nr: int) -> tuple[np.ndarray, np.ndarray]:
    """Radial nodes r_p in (0, R), ascending, and weights with sum_p w_p f(r_p) ~ int_0^R f r dr."""
    x, w = gauss_jacobi_01(Nr)
    return R * (1.0 + x) / 2.0, (R * R / 4.0) * w


# ----------------------------------------------------------------------------------------
# The basis
# ----------------------------------------------------------------------------------------


@dataclass
class Basis:
    R: float
    tau: float
    alpha: float
    Nr: int
    Nth1: int
    Nth2: int
    ncyc: int = 1
    s: int = 4
    # filled by __post_init__
    M: int = field(init=False)
    N: int = field(init=False)
    K: int = field(init=False)

    def __post_init__(self):
        if not (self.R > 0 and self.tau > 0 and self.ncyc >= 1):
            raise ValueError("need R > 0, tau > 0, ncyc >= 1")
        # reading R3
        self.M = (self.Nth1 - 1) // self.s
        self.N = (self.Nth2 - 1) // self.s
        self.K = self.Nr // self.s
        if self.K < 1:
            raise ValueError("N_r too small for the oversampling")
        self.r, self.wr = radial_grid(self.R, self.Nr)
        # zeros for every |n Ncyc| used
        self.zeros = {}
        for n in range(0, self.N + 1):
            self.zeros[n] = bessel_zeros(n * self.ncyc, self.K)
        # radial tables (Algorithms 1 and 3): Rtab[n] = frak R_n (Nr x K), Otab[n] = frak O_n (K x Nr)
        self.Rtab = {}
        self.Otab = {}
        for n in range(-self.N, self.N + 1):
            T = np.empty((self.Nr, self.K))
            for k in range(self.K):
                T[:, k] = self.xi(n, k, self.r)
            self.Rtab[n] = T
            self.Otab[n] = (T * self.wr[:, None]).T.copy()

    # -- sizes / order ------------------------------------------------------------------
    @property
    def box_shape(self):
        return (2 * self.M + 1, 2 * self.N + 1, self.K)

    @property
    def box_size(self):
        return (2 * self.M + 1) * (2 * self.N + 1) * self.K

    def box_index(self, m, n, k):
        """eq. wavefun_storage, 0-based in k (k = 0 is the paper's k = 1)."""
        return (m + self.M) * (2 * self.N + 1) * self.K + (n + self.N) * self.K + k

    def box_mnk(self):
        """(m, n, k) of every box entry in the order of eq. wavefun_storage (k 0-based)."""
        m, n, k = np.meshgrid(np.arange(-self.M, self.M + 1), np.arange(-self.N, self.N + 1),
                              np.arange(self.K), indexing="ij")
        return m.ravel(), n.ravel(), k.ravel()

    # -- basis functions ------------------------------------------------------------------
    def bzero(self, n, k):
        return self.zeros[abs(n)][k]

    def xi(self, n, k, r):
        """Radial part xi_{n,k}(r) of eq. Basis_fun_derived (literal, signed order n*Ncyc)."""
        p = n * self.ncyc
        b = self.bzero(n, k)
        c = math.sqrt(self.ncyc / (math.pi * self.tau)) / (self.R * special.jv(p + 1, b))
        return c * special.jv(p, b * np.asarray(r) / self.R)

    def F(self, m, n, k, th1, th2, r):
        """F_{m,n,k}(theta1, theta2, r) of eq. Basis_fun_derived."""
        ph = np.exp(2j * np.pi * (m * np.asarray(th1) + n * self.ncyc * np.asarray(th2)))
        return ph * self.xi(n, k, r)

    def itable(self, n):
        """K x K table I(n, k, k') of eq. I_nkk_prime (k, k' 0-based), the radial integral of the
        1/r^2 terms (eqs. ell_coeff and ell_mnk):

            I(n, k, k') = int_0^1 J_p(b_k q) J_p(b_k' q) / q dq / (J_{p+1}(b_k) J_{p+1}(b_k')),

        p = n Ncyc, b_k = b_k^p.  For p != 0 the integrand is smooth (it behaves as q^(2|p|-1)) and
        the integral is taken as written by Gauss-Legendre quadrature on [0, 1] with enough nodes
        for the band limit b_k + b_k' (the paper's recurrence of Appendix D only serves to remove
        the 1/q, which plain Gauss-Legendre does not need).  For p = 0 the integral diverges at
        q = 0; reading: it is replaced by the transform's own radial rule, sum_p w_p J J / r_p^2
        (nodes avoid r = 0, so the value is finite), and KPoint.n0_quadrature flags its use."""
        cache = self.__dict__.setdefault("_itable_cache", {})
        if n in cache:
            return cache[n]
        p = n * self.ncyc
        zs = self.zeros[abs(n)]
        jp1 = special.jv(p + 1, zs)
        if p == 0:
            Jr = special.jv(0, np.outer(self.r / self.R, zs))            # [Nr, K]
            integ = (Jr * (self.wr / self.r ** 2)[:, None]).T @ Jr
        else:
            nq = 64 + 2 * int(math.ceil(zs[-1]))
            x, w = np.polynomial.legendre.leggauss(nq)
            q = 0.5 * (x + 1.0)
            w = 0.5 * w
            Jq = special.jv(p, np.outer(q, zs))                          # [nq, K]
            integ = (Jq * (w / q)[:, None]).T @ Jq
        cache[n] = integ / np.outer(jp1, jp1)
        return cache[n]

    def lambda0(self, m, n, k):
        """eq. Laplacian_of_f_mnk."""
        b = np.vectorize(self.bzero)(n, k)
        return (b / self.R) ** 2 + (2 * np.pi / self.tau * (m - self.alpha * n * self.ncyc)) ** 2

    # -- grids ----------------------------------------------------------------------------
    def theta_grid(self):
        """Fourier nodes theta1_i = i/N_th1, theta2_j = j/(Ncyc N_th2), from the trapezoid
        weights 1/N_th1 and 1/(Ncyc N_th2) of eq. Fast_fwd_transform_cont (reading 3)."""
        return (np.arange(self.Nth1) / self.Nth1,
                np.arange(self.Nth2) / (self.ncyc * self.Nth2))

    # -- reciprocal-space diagonal at (eta, nu) --------------------------------------------
    def abc(self, eta, nu):
        """Constants a, b, c of eq. constants_abc."""
        al, t = self.alpha, self.tau
        a = 2 * np.pi ** 2 / t ** 2 * (nu * al * (2 * eta - nu * al) - eta ** 2)
        b = 2j * np.pi / t ** 2 * (nu * al - eta)
        c = 2j * np.pi * al / t ** 2 * (eta - nu * al)
        return a, b, c

    def diagonal_literal(self, eta, nu):
        """Box vector 1/2 Lambda - a - b M - c N of Algorithm 5 (its first four lines),
        evaluated literally; returned as a complex array (its imaginary part is zero)."""
        m, n, k = self.box_mnk()
        Lam = self.lambda0(m, n, k)
        Mv = 2j * np.pi * m
        Nv = 2j * np.pi * self.ncyc * n
        a, b, c = self.abc(eta, nu)
        return 0.5 * Lam - a - b * Mv - c * Nv

    def kinetic(self, eta, nu):
        """Shifted kinetic energy KE_i of every box entry (reading R5): the real part of the
        literal Algorithm-5 diagonal."""
        return self.diagonal_literal(eta, nu).real

    def mask(self, eta, nu, ecut):
        """Boolean box mask of eq. Energy_cutoff at (eta, nu); ecut <= 0 keeps the whole box."""
        if ecut is None or ecut <= 0:
            return np.ones(self.box_size, dtype=bool)
        return self.kinetic(eta, nu) <= ecut * (1.0 + 1e-12)


class KPoint:
    """One (eta, nu) point with its cutoff mask; compact order = box order restricted to the mask."""

    def __init__(self, basis: Basis, eta: float, nu: float, ecut: float | None):
        self.basis = basis
        self.eta = float(eta)
        self.nu = float(nu)
        self.ecut = ecut
        self.mask = basis.mask(eta, nu, ecut)
        self.idx = np.nonzero(self.mask)[0]          # compact -> box
        self.L = int(self.idx.size)
        m, n, k = basis.box_mnk()
        self.m, self.n, self.k = m[self.idx], n[self.idx], k[self.idx]
        self.ke = basis.kinetic(eta, nu)[self.idx]
        # nu != 0 with n = 0 modes kept: their 1/r^2 integrals diverge and take the radial-rule
        # value (see Basis.itable)
        self.n0_quadrature = bool(self.nu != 0 and np.any(self.n == 0))

    def to_box(self, Xc):
        Xc = np.asarray(Xc)
        out = np.zeros((self.basis.box_size,) + Xc.shape[1:], dtype=np.complex128)
        out[self.idx] = Xc
        return out

    def from_box(self, Xb):
        return np.asarray(Xb)[self.idx]
