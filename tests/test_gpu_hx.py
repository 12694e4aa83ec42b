"""GPU parity of H X and the TPA preconditioner (through the C ABI) against the CPU oracle.

Tolerances: the FP64 path must match Algorithm 5 of the oracle to 1e-10 relative (per column,
in the 2-norm); the mixed path (FP32 transforms, FP64 diagonal) to 2e-6 relative, the FP32
rounding of O(100) accumulated terms.  Every entry is bounded too (tests/_parity.py):
|dY_ij| <= tol |Y_ij| + floor max_i |Y_ij| with floor 1e-13 (FP64: a few ulps of the column's
largest entry) and 2e-7 (mixed: the FP32 transforms leave absolute errors of a few 1e-8 of the
column's largest entry, measured by an FP32 emulation of Algorithms 1-4 on the tube; the
diagonal term, the largest part of most entries, is FP64).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import basis as B
from oracle import eigensolver as E
from oracle import hamiltonian as Hm
from oracle import potential as P
from paper_2210_12252_gb300 import inputs
from _parity import assert_entrywise

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 2e-6
FP64_FLOOR = 1e-13
MIXED_FLOOR = 2e-7


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


def oracle_basis(g):
    return B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)


def to_dev(X, ld=None):
    """column-major L x ns numpy block -> (ns, ld) complex128 CUDA tensor"""
    L, ns = X.shape
    ld = ld or L
    T = torch.zeros((ns, ld), dtype=torch.complex128)
    T[:, :L] = torch.from_numpy(np.ascontiguousarray(X.T))
    return T.cuda()


def from_dev(T, L):
    return T[:, :L].cpu().numpy().T


def rel_err(Y, Yref):
    return (np.linalg.norm(Y - Yref, axis=0) / np.linalg.norm(Yref, axis=0)).max()


class Case:
    def __init__(self, hwmod, w, etas=None, ecuts=None):
        self.w = w
        self.etas = np.asarray(w.etas if etas is None else etas, dtype=float)
        self.ecuts = ecuts
        self.ctx = hwmod.Context(0)
        self.L = self.ctx.setup_basis(w.geom, self.etas, None, ecuts)
        self.ctx.build_potential(w.atoms)
        self.b = oracle_basis(w.geom)
        self.V = P.gaussian_wells(self.b, w.atoms)
        self.kps = [B.KPoint(self.b, e, 0.0, w.geom.ecut if ecuts is None else ecuts[i])
                    for i, e in enumerate(self.etas)]


@pytest.fixture(scope="module")
def tiny(hwmod):
    return Case(hwmod, inputs.tiny())


@pytest.fixture(scope="module")
def tube(hwmod):
    return Case(hwmod, inputs.tube())


@pytest.mark.parametrize("ns", [1, 5, 16])
def test_apply_H_fp64_tiny(tiny, ns):
    kp = tiny.kps[0]
    X = inputs.random_block(kp.L, ns, 100 + ns)
    Yref = Hm.apply_H(kp, tiny.V, X)
    Y = from_dev(tiny.ctx.apply_H(0, to_dev(X)), kp.L)
    assert rel_err(Y, Yref) < FP64_TOL
    assert_entrywise(Y, Yref, FP64_TOL, FP64_FLOOR, "tiny fp64")


def test_apply_H_fp64_tube_ragged_with_padding(tube):
    kp = tube.kps[0]
    assert tube.L[0] == kp.L
    X = inputs.random_block(kp.L, 3, 7)
    Xd = to_dev(X, ld=kp.L + 13)
    Yd = torch.full_like(Xd, complex(7.0, -3.0))
    tube.ctx.apply_H(0, Xd, Yd)
    Y = from_dev(Yd, kp.L)
    Yref = Hm.apply_H(kp, tube.V, X)
    assert rel_err(Y, Yref) < FP64_TOL
    assert_entrywise(Y, Yref, FP64_TOL, FP64_FLOOR, "tube fp64")
    # padding rows untouched
    assert torch.all(Yd[:, kp.L:] == complex(7.0, -3.0))


def test_apply_H_mixed_tube(tube):
    kp = tube.kps[0]
    X = inputs.random_block(kp.L, 4, 8)
    Yref = Hm.apply_H(kp, tube.V, X)
    Y = from_dev(tube.ctx.apply_H(0, to_dev(X), prec="mixed"), kp.L)
    e = rel_err(Y, Yref)
    assert e < MIXED_TOL and e > 1e-12   # really ran in reduced precision
    assert_entrywise(Y, Yref, MIXED_TOL, MIXED_FLOOR, "tube mixed")


def test_apply_H_is_hermitian_on_device(tiny):
    kp = tiny.kps[0]
    X = inputs.random_block(kp.L, 6, 21)
    Y = from_dev(tiny.ctx.apply_H(0, to_dev(X)), kp.L)
    G = X.conj().T @ Y
    assert np.abs(G - G.conj().T).max() < 1e-12 * np.abs(G).max()


def test_apply_H_batched_uneven_kpoints(hwmod):
    w = inputs.tube_kpoints(nk=4, uneven=True)
    case = Case(hwmod, w, ecuts=w.ecuts)
    ns = 3
    Lmax = int(max(case.L))
    Xs, Ys, refs = [], [], []
    for b, kp in enumerate(case.kps):
        X = inputs.random_block(kp.L, ns, 300 + b)
        Xs.append(to_dev(X, ld=Lmax))
        Ys.append(torch.zeros_like(Xs[-1]))
        refs.append(Hm.apply_H(kp, case.V, X))
    case.ctx.apply_H_batched(list(range(len(case.kps))), Xs, Ys)
    for b, kp in enumerate(case.kps):
        assert rel_err(from_dev(Ys[b], kp.L), refs[b]) < FP64_TOL
        assert_entrywise(from_dev(Ys[b], kp.L), refs[b], FP64_TOL, FP64_FLOOR, f"batched k{b}")


def test_tpa_preconditioner_matches_oracle(tube):
    kp = tube.kps[0]
    R = inputs.random_block(kp.L, 5, 9) * np.exp(-0.01 * np.arange(kp.L))[:, None]
    Z = from_dev(tube.ctx.apply_precond(0, to_dev(R)), kp.L)
    Zref = E.tpa(kp.ke, R)
    assert rel_err(Z, Zref) < 1e-13
    assert_entrywise(Z, Zref, 1e-13, 1e-15, "tpa")


def test_set_potential_from_device_matches_host_build(tube):
    kp = tube.kps[0]
    V = torch.from_numpy(tube.V.ravel().copy()).cuda()
    tube.ctx.set_potential(V)       # oracle-built V from device memory
    X = inputs.random_block(kp.L, 2, 5)
    Y = from_dev(tube.ctx.apply_H(0, to_dev(X)), kp.L)
    Yref = Hm.apply_H(kp, tube.V, X)
    assert rel_err(Y, Yref) < FP64_TOL
    assert_entrywise(Y, Yref, FP64_TOL, FP64_FLOOR, "V from device")
    tube.ctx.build_potential(tube.w.atoms)   # restore the library-built V


def test_apply_H_mixed_tube_slab_variants_agree(tube, hwmod):
    """The angular kernels on the 64 x 48 grid: the all-register variant (theta2 as 4 lanes x
    12-point DFTs joined by a 4-point DFT across the lanes, theta1 bins in registers; 2), the
    4 x 16 register-DFT theta1 variant with Stockham theta2 passes (1) and the Stockham FFTs
    (0) agree with each other at FP32 rounding and with the oracle within the mixed tolerance.
    5 columns: the all-register kernel takes 4 slabs per CTA, so its second CTA has one."""
    kp = tube.kps[0]
    X = inputs.random_block(kp.L, 5, 81)
    Yref = Hm.apply_H(kp, tube.V, X)
    Xd = to_dev(X)
    out = {}
    keep = tube.ctx.get_option(hwmod.HW_OPT_SLAB_KERNEL)
    try:
        for v in (2, 1, 0):
            tube.ctx.set_option(hwmod.HW_OPT_SLAB_KERNEL, v)
            out[v] = from_dev(tube.ctx.apply_H(0, Xd, prec="mixed"), kp.L)
            assert rel_err(out[v], Yref) < MIXED_TOL
            assert_entrywise(out[v], Yref, MIXED_TOL, MIXED_FLOOR, f"slab variant {v}")
    finally:
        tube.ctx.set_option(hwmod.HW_OPT_SLAB_KERNEL, keep)
    assert rel_err(out[1], out[0]) < MIXED_TOL
    assert rel_err(out[2], out[0]) < MIXED_TOL


def test_apply_H_fp64_tube_slab_variants_agree(tube, hwmod):
    """The same three angular kernels in FP64 (the register kernel by option 3) against the
    oracle (FP64 tolerance, entry-wise), on 7 ragged columns with a padded leading dimension."""
    kp = tube.kps[0]
    X = inputs.random_block(kp.L, 7, 83)
    Yref = Hm.apply_H(kp, tube.V, X)
    Xd = to_dev(X, kp.L + 6)
    keep = tube.ctx.get_option(hwmod.HW_OPT_SLAB_KERNEL)
    try:
        for v in (3, 1, 0):
            tube.ctx.set_option(hwmod.HW_OPT_SLAB_KERNEL, v)
            Y = from_dev(tube.ctx.apply_H(0, Xd, prec="fp64"), kp.L)
            assert rel_err(Y, Yref) < FP64_TOL, v
            assert_entrywise(Y, Yref, FP64_TOL, FP64_FLOOR, f"FP64 slab variant {v}")
    finally:
        tube.ctx.set_option(hwmod.HW_OPT_SLAB_KERNEL, keep)


def test_apply_H_fp64_df_tube_matches_oracle(tube, hwmod):
    """hw_apply_H with HW_FP64_DF: the radial and angular transforms in double-float arithmetic
    (FP32 pairs), the diagonal in FP64.  Entry-wise within the FP64 tolerance of the oracle,
    and within 1e-12 (column norms) of the FP64 kernel; 9 ragged columns (three CTAs of 4 slabs,
    the last with one), padded leading dimension."""
    kp = tube.kps[0]
    X = inputs.random_block(kp.L, 9, 85)
    Yref = Hm.apply_H(kp, tube.V, X)
    Xd = to_dev(X, kp.L + 2)
    Ydf = from_dev(tube.ctx.apply_H(0, Xd, prec="fp64_df"), kp.L)
    Y64 = from_dev(tube.ctx.apply_H(0, Xd, prec="fp64"), kp.L)
    assert rel_err(Ydf, Yref) < FP64_TOL
    assert_entrywise(Ydf, Yref, FP64_TOL, FP64_FLOOR, "double-float angular transforms")
    assert rel_err(Ydf, Y64) < 1e-12
    print(f"double-float vs FP64 kernel: {rel_err(Ydf, Y64):.2e}; vs oracle {rel_err(Ydf, Yref):.2e}")


def test_apply_H_mixed_overlapped_launches_bit_identical(tube, hwmod):
    """HW_OPT_OVERLAP_LAUNCH only changes when the FP32 H X's three kernels start, not what they
    compute: 76 columns (the Chebyshev block; ragged tiles in every |n| group), four chained
    products (each output the next input), bit for bit the same with the option on and off."""
    kp = tube.kps[0]
    X = to_dev(inputs.random_block(kp.L, 76, 85))
    keep = tube.ctx.get_option(hwmod.HW_OPT_OVERLAP_LAUNCH)
    out = {}
    try:
        for ov in (1, 0):
            tube.ctx.set_option(hwmod.HW_OPT_OVERLAP_LAUNCH, ov)
            Z = X
            chain = []
            for _ in range(4):
                Z = tube.ctx.apply_H(0, Z, prec="mixed")
                chain.append(Z.clone())
            torch.cuda.synchronize()
            out[ov] = chain
    finally:
        tube.ctx.set_option(hwmod.HW_OPT_OVERLAP_LAUNCH, keep)
    for a, b in zip(out[1], out[0]):
        assert torch.equal(a, b)
    assert torch.isfinite(torch.view_as_real(out[1][-1])).all()
