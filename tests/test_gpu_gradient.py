"""GPU parity of the Cartesian gradients (hw_gradient, Appendix C) against the oracle's
oracle.gradient on the same seeded coefficients.

Tolerances (max |difference| over the grid relative to max |oracle value| of that component):
1e-10 for the FP64 path; 2e-5 for the mixed path (FP32 radial and angular transforms of
O(100)-term sums, FP64 chain rule).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import basis as B
from oracle import gradient as Gr
from paper_2210_12252_gb300 import inputs
from _parity import assert_entrywise

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 2e-5


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


def to_dev(X, ld=None):
    L, ns = X.shape
    ld = ld or L
    T = torch.zeros((ns, ld), dtype=torch.complex128)
    T[:, :L] = torch.from_numpy(np.ascontiguousarray(X.T))
    return T.cuda()


def check(hwmod, w, k, ns, seed, precs=("fp64", "mixed"), ld_pad=0):
    g = w.geom
    ctx = hwmod.Context(0)
    L = ctx.setup_basis(g, w.etas, w.nus)
    ctx.build_potential(w.atoms)
    b = B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)
    nu = 0.0 if w.nus is None else w.nus[k]
    kp = B.KPoint(b, w.etas[k], nu, g.ecut)
    assert L[k] == kp.L
    X = inputs.random_block(kp.L, ns, seed)
    refs = [Gr.gradient(kp, X[:, c]) for c in range(ns)]
    Xd = to_dev(X, kp.L + ld_pad)
    for prec in precs:
        D = ctx.gradient(k, Xd, prec=prec).cpu().numpy()
        tol = FP64_TOL if prec == "fp64" else MIXED_TOL
        for c in range(ns):
            for comp in range(3):
                ref = refs[c][comp]
                err = np.abs(D[c, comp] - ref).max() / np.abs(ref).max()
                assert err < tol, (prec, c, comp, err)
                assert_entrywise(D[c, comp].ravel(), ref.ravel(), tol, tol * 1e-1 if prec == "mixed" else tol * 1e-3,
                                 f"gradient {prec} column {c} component {comp}")
                if prec == "mixed":
                    assert err > 1e-13   # really ran in reduced precision
    ctx.close()


def test_gradient_tiny(hwmod):
    check(hwmod, inputs.tiny(), 0, 3, 71)


def test_gradient_tiny_cyclic_padded_ld(hwmod):
    check(hwmod, inputs.tiny_cyclic(), 1, 2, 72, ld_pad=9)


def test_gradient_tube_cutoff(hwmod):
    check(hwmod, inputs.tube(), 0, 2, 73)


def test_gradient_rejects_bad_arguments(hwmod):
    w = inputs.tiny()
    ctx = hwmod.Context(0)
    ctx.setup_basis(w.geom, w.etas)
    X = torch.zeros((1, int(ctx.L[0])), dtype=torch.complex128, device="cuda")
    D = torch.zeros((1, 3), dtype=torch.complex128, device="cuda")
    for args in [(1, X.data_ptr(), 1, int(ctx.L[0])), (0, X.data_ptr(), 1, int(ctx.L[0]) - 1),
                 (0, X.data_ptr(), 0, int(ctx.L[0]))]:
        st = hwmod.load_library().hw_gradient(ctx.h, args[0], hwmod.C.c_void_p(args[1]), args[2], args[3],
                                              hwmod.C.c_void_p(D.data_ptr()), hwmod.HW_FP64)
        assert st == hwmod.HW_EINVAL
    ctx.close()
