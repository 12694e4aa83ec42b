"""hw_density (electron density from state blocks) against the CPU oracle (oracle/density.py).

Bars: FP64 transforms within 1e-12 of max rho entry by entry; mixed (FP32 transforms and
accumulation) within 2e-6 of max rho; the quadrature of rho equals the electron count
2 sum_b w_b sum_j occ_bj for orthonormal states (radial quadrature error 1e-9)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import basis as B
from oracle import density as D
from paper_2210_12252_gb300 import inputs
from _parity import assert_entrywise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


def setup(hwmod, w, etas):
    ctx = hwmod.Context(0)
    L = ctx.setup_basis(w.geom, etas)
    ctx.build_potential(w.atoms)
    g = w.geom
    b = B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)
    kps = [B.KPoint(b, e, 0.0, g.ecut) for e in etas]
    return ctx, L, b, kps


def states(L, ns, seed, ld=None):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((L, ns)) + 1j * g.standard_normal((L, ns)))
    ld = ld or L
    Xd = torch.zeros((ns, ld), dtype=torch.complex128)
    Xd[:, :L] = torch.from_numpy(np.ascontiguousarray(Q.T))
    return Q, Xd.cuda()


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-12), ("mixed", 2e-6)])
def test_tiny_two_kpoints_match_oracle(hwmod, prec, bar):
    w = inputs.tiny()
    etas = [0.0, 0.3]
    ctx, L, b, kps = setup(hwmod, w, etas)
    ns, ld = 5, int(max(L)) + 3
    Qs, Xs = zip(*[states(int(L[i]), ns, 10 + i, ld) for i in range(2)])
    occ = np.array([[1.0, 1.0, 0.5, 0.25, 0.0], [1.0, 0.8, 0.6, 0.0, 0.1]])
    wk = np.array([0.5, 0.5])
    rho = ctx.density([0, 1], list(Xs), occ, wk, prec=prec).cpu().numpy()
    ref = D.density(kps, list(Qs), list(occ), list(wk))
    assert np.abs(rho - ref).max() <= bar * np.abs(ref).max()
    # every grid value on its own (the density is smallest near the wall)
    assert_entrywise(rho.ravel(), ref.ravel(), bar, bar * (1e-2 if prec == "fp64" else 1e-1), f"tiny {prec}")
    assert abs(D.charge(b, rho) - 2 * (wk[:, None] * occ).sum()) < (1e-9 if prec == "fp64" else 1e-5)
    ctx.close()


def test_tube_converged_states_match_oracle(hwmod):
    w = inputs.tube()
    ctx, L, b, kps = setup(hwmod, w, [0.0])
    r = ctx.solve_eigs([0], 16, tol=1e-6, maxit=400, prec="mixed", vectors=True)
    X = r["evecs"][0].contiguous()
    occ = np.ones((1, 16))
    rho = ctx.density([0], [X], occ, [1.0]).cpu().numpy()
    ref = D.density(kps, [X.cpu().numpy().T], list(occ), [1.0])
    assert np.abs(rho - ref).max() <= 1e-11 * np.abs(ref).max()
    assert_entrywise(rho.ravel(), ref.ravel(), 1e-11, 1e-13, "tube fp64")
    assert abs(D.charge(b, rho) - 32.0) < 1e-6
    ctx.close()


def test_density_rejects_bad_arguments(hwmod):
    w = inputs.tiny()
    ctx, L, b, kps = setup(hwmod, w, [0.0])
    X = torch.zeros((2, int(L[0]) - 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(hwmod.HwError) as e:
        ctx.density([0], [X], np.ones((1, 2)), [1.0])      # ld < L
    assert e.value.status == hwmod.HW_EINVAL
    X = torch.zeros((2, int(L[0])), dtype=torch.complex128, device="cuda")
    with pytest.raises(hwmod.HwError) as e:
        ctx.density([3], [X], np.ones((1, 2)), [1.0])      # k-point out of range
    assert e.value.status == hwmod.HW_EINVAL
    ctx.close()
