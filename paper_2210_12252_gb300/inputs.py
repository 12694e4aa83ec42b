"""Seeded synthetic inputs shared by the library's tests, the benchmark and the CPU oracle.

This module draws random numbers and fixes workload sizes; it holds none of the method's
arithmetic (no basis, grid, transform or Hamiltonian code).  Atoms are returned in cylindrical
coordinates as rows (r, vartheta, z, Z, sigma) in bohr / radians / Hartree units, the form
both the library (hw_build_potential) and the oracle (oracle.potential) take.

The workloads stand in for the paper's nanotube / nanowire systems, whose empirical
pseudopotentials and atomic structures are not available: Gaussian wells of depth Z and width
sigma placed in helical patterns of the same geometry class (radius, pitch, twist, grids and
kinetic cutoff as listed below).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Geometry:
    R: float
    tau: float
    alpha: float
    Nr: int
    Nth1: int
    Nth2: int
    ecut: float            # Hartree; <= 0 keeps the whole basis box
    ncyc: int = 1
    oversample: int = 4


@dataclass
class Workload:
    name: str
    geom: Geometry
    atoms: np.ndarray                  # (n_atoms, 5)
    etas: np.ndarray                   # helical wavevectors eta_b
    n_eig: int
    seed: int
    ecuts: np.ndarray | None = None    # optional per-k-point cutoff (uneven-basis stressor)
    nus: np.ndarray | None = None      # cyclic wavenumbers nu_b (None: all zero)
    notes: str = ""
    extra: dict = field(default_factory=dict)


def _rng(seed):
    return np.random.default_rng(seed)


def ring_atoms(n, radius, tau, Z, sigma, seed):
    """n atoms on a cylinder of the given radius, uniform random angle and height."""
    g = _rng(seed)
    th = g.uniform(0.0, 2 * np.pi, n)
    z = g.uniform(0.0, tau, n)
    return np.column_stack([np.full(n, radius), th, z, np.full(n, Z), np.full(n, sigma)])


def chiral_lattice_atoms(n, radius, tau, Z, sigma, seed, step=7, jitter=0.02):
    """n atoms on a cylinder in a chiral lattice: heights (a + 1/2) tau / n, angles
    2 pi frac(a * step / n + u_a) with u_a ~ U(-jitter, jitter) (step coprime to n)."""
    g = _rng(seed)
    a = np.arange(n)
    u = g.uniform(-jitter, jitter, n)
    th = 2 * np.pi * np.mod(a * step / n + u, 1.0)
    z = (a + 0.5) * tau / n
    return np.column_stack([np.full(n, radius), th, z, np.full(n, Z), np.full(n, sigma)])


def core_atoms(n, rmax, tau, Z, sigma, seed):
    """n atoms uniform in the disc r <= rmax (r^2 uniform) times [0, tau)."""
    g = _rng(seed)
    r = np.sqrt(g.uniform(0.0, rmax * rmax, n))
    th = g.uniform(0.0, 2 * np.pi, n)
    z = g.uniform(0.0, tau, n)
    return np.column_stack([r, th, z, np.full(n, Z), np.full(n, sigma)])


def random_family_atoms(seed, tau, n_range=(20, 60), Z_range=(2.0, 6.0),
                        sigma_range=(0.6, 1.2), r_range=(3.0, 8.0)):
    """One member of the random-potential family: atom count, depth and width drawn per
    potential, positions uniform in an annulus."""
    g = _rng(seed)
    n = int(g.integers(n_range[0], n_range[1] + 1))
    Z = g.uniform(*Z_range)
    sig = g.uniform(*sigma_range)
    r = g.uniform(r_range[0], r_range[1], n)
    th = g.uniform(0.0, 2 * np.pi, n)
    z = g.uniform(0.0, tau, n)
    return np.column_stack([r, th, z, np.full(n, Z), np.full(n, sig)])


def random_block(L, ns, seed):
    """Complex Gaussian L x ns block (column-major use: column j is X[:, j])."""
    g = _rng(seed)
    return (g.standard_normal((L, ns)) + 1j * g.standard_normal((L, ns))) / np.sqrt(2.0)


# ------------------------------------------------------------------------------ workloads

GEOM_TINY = Geometry(R=6.0, tau=3.0, alpha=0.1, Nr=24, Nth1=16, Nth2=16, ecut=0.0)
GEOM_TUBE = Geometry(R=12.0, tau=4.6, alpha=0.05, Nr=96, Nth1=64, Nth2=48, ecut=30.0)
GEOM_WIRE = Geometry(R=20.0, tau=8.0, alpha=0.02, Nr=192, Nth1=192, Nth2=96, ecut=40.0)


def tiny(seed=1, zero_potential=False):
    """R=6, tau=3, alpha=0.1; 4 wells (Z=4, sigma=0.8) at r=2.5; 16x16 angular grid, 24 radial
    nodes; one k-point; 8 eigenpairs."""
    atoms = ring_atoms(4, 2.5, GEOM_TINY.tau, 4.0, 0.8, seed)
    if zero_potential:
        atoms = atoms[:0]
    return Workload("tiny_R6_16x16x24", GEOM_TINY, atoms, np.array([0.0]), 8, seed)


def tiny_s2(seed=1):
    """The tiny geometry with oversampling 2 (a larger, still unmasked basis)."""
    g = Geometry(**{**GEOM_TINY.__dict__, "oversample": 2})
    atoms = ring_atoms(4, 2.5, g.tau, 4.0, 0.8, seed)
    return Workload("tiny_R6_16x16x24_s2", g, atoms, np.array([0.0]), 8, seed)


def tiny_cyclic(seed=1, ncyc=3):
    """The tiny geometry with an Ncyc-fold cyclic symmetry (theta2 spans 1/Ncyc of a turn): 4
    wells (Z=4, sigma=0.8) at r=2.5 per fundamental domain, repeated by the cyclic rotations;
    k-points (eta, nu) = (0.1, 1), (-0.3, 2), (0.25, 0); 8 eigenpairs."""
    g = Geometry(**{**GEOM_TINY.__dict__, "ncyc": ncyc})
    atoms = ring_atoms(4, 2.5, g.tau, 4.0, 0.8, seed)
    return Workload(f"tiny_c{ncyc}_R6_16x16x24", g, atoms, np.array([0.1, -0.3, 0.25]), 8, seed,
                    nus=np.array([1.0, 2.0, 0.0]))


def tube_cyclic(seed=4, ncyc=3, nk=3):
    """The tube geometry (R=12, tau=4.6, alpha=0.05, 64x48x96 grid, 30 Ha) with a 3-fold cyclic
    symmetry: 40 wells (Z=4, sigma=0.8) on r=6 in a chiral lattice per fundamental domain;
    one k-point per nu = 0..nk-1 at seeded eta ~ U[-1/2, 1/2); 32 eigenpairs each."""
    g = Geometry(**{**GEOM_TUBE.__dict__, "ncyc": ncyc})
    atoms = chiral_lattice_atoms(40, 6.0, g.tau, 4.0, 0.8, seed)
    etas = _rng(seed + 1).uniform(-0.5, 0.5, nk)
    nus = np.arange(nk, dtype=np.float64) % ncyc
    return Workload(f"tube_c{ncyc}_{nk}k", g, atoms, etas, 32, seed, nus=nus)


def tube(seed=2):
    """Nanotube-like: R=12, tau=4.6, alpha=0.05; 40 wells (Z=4, sigma=0.8) on r=6 in a chiral
    lattice; N_r=96, 64x48 angular grid, cutoff 30 Ha; one k-point; 64 eigenpairs."""
    atoms = chiral_lattice_atoms(40, 6.0, GEOM_TUBE.tau, 4.0, 0.8, seed)
    return Workload("tube_R12_64x48x96_ec30", GEOM_TUBE, atoms, np.array([0.0]), 64, seed)


def tube_kpoints(seed=3, nk=32, uneven=False):
    """The tube potential at nk seeded eta ~ U[0,1) (nu = 0), 48 eigenpairs each.  With
    uneven=True every k-point also draws its own cutoff in [10, 30] Ha."""
    w = tube(seed=2)
    g = _rng(seed)
    etas = g.uniform(0.0, 1.0, nk)
    ecuts = g.uniform(10.0, 30.0, nk) if uneven else None
    name = f"tube_{nk}k" + ("_uneven" if uneven else "")
    return Workload(name, GEOM_TUBE, w.atoms, etas, 48, seed, ecuts=ecuts)


def tube_family(index, seed0=1000):
    """Member `index` of the random-potential family on the tube geometry (training:
    0..255, held out: 256..319)."""
    atoms = random_family_atoms(seed0 + index, GEOM_TUBE.tau)
    return Workload(f"tube_family_{index}", GEOM_TUBE, atoms, np.array([0.0]), 64, seed0 + index)


def wire(seed=5, nk=16):
    """Nanowire-like: R=20, tau=8, alpha=0.02; 300 wells (Z=4, sigma=0.8) uniform in r <= 14;
    N_r=192, 192x96 angular grid, cutoff 40 Ha; nk seeded eta ~ U[0,1); 400 eigenpairs."""
    atoms = core_atoms(300, 14.0, GEOM_WIRE.tau, 4.0, 0.8, seed)
    etas = _rng(seed + 1).uniform(0.0, 1.0, nk)
    return Workload("wire_R20_192x96x192_ec40", GEOM_WIRE, atoms, etas, 400, seed)
