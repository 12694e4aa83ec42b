"""The Rayleigh-Ritz dense Hermitian eigensolver (hw_heev) against numpy.linalg.eigh: FP64
Jacobi (all pairs) and the Householder route (FP32 reduction + FP64 refinement of the lowest
nw pairs), on spectra with well-separated, exactly degenerate and near-degenerate eigenvalues
and with the padded rows the eigensolver uses for inactive columns."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


def hermitian_with_spectrum(lam, seed):
    g = np.random.default_rng(seed)
    n = lam.size
    Q, _ = np.linalg.qr(g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)))
    return (Q * lam) @ Q.conj().T


def spectra(n, seed):
    g = np.random.default_rng(seed)
    out = []
    out.append(np.sort(g.uniform(-5, 30, n)))                       # separated
    lam = np.sort(g.uniform(-5, 30, n))
    lam[3] = lam[2]                                                   # exact pair
    lam[10:13] = lam[10] + np.array([0.0, 1e-9, 2e-9])               # tight triple
    lam[20] = lam[19] + 1e-6                                          # near pair
    out.append(np.sort(lam))
    return out


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("n", [72, 216])
def test_heev_matches_numpy(hwmod, method, n):
    ctx = hwmod.Context(0)
    nw = n // 3
    mats = [hermitian_with_spectrum(l, 7 + i) for i, l in enumerate(spectra(n, n))]
    A = np.stack(mats)
    # rows/cols of a padded index: decoupled with a huge diagonal (sorts last)
    A[0, -1, :] = 0.0
    A[0, :, -1] = 0.0
    A[0, -1, -1] = 1e10
    At = torch.from_numpy(np.ascontiguousarray(np.transpose(A, (0, 2, 1)))).cuda()   # rows = columns
    w, Z = hwmod.hw_heev(ctx.h, At, nw, method)
    w = w.cpu().numpy()
    Z = Z.cpu().numpy()   # Z[b][j] = eigenvector j
    for b in range(A.shape[0]):
        ref = np.linalg.eigvalsh(A[b])
        scale = np.abs(ref[:-1]).max()
        assert np.abs(w[b, :nw] - ref[:nw]).max() < 1e-10 * scale, (b, np.abs(w[b, :nw] - ref[:nw]).max())
        Zb = Z[b, :nw].T                     # n x nw
        G = Zb.conj().T @ Zb
        assert np.abs(G - np.eye(nw)).max() < 1e-11
        R = A[b] @ Zb - Zb * w[b, :nw]
        assert np.linalg.norm(R, axis=0).max() < 1e-10 * scale
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 2e-5)])
@pytest.mark.parametrize("n", [1, 17, 76, 112, 130])
def test_cholesky_matches_numpy(hwmod, prec, tol, n):
    """hw_cholesky (the Cholesky-QR's factor step): lower factors of Gram matrices X^H X of
    random tall complex blocks (condition ~1e2) against numpy.linalg.cholesky, entry-wise
    relative to the largest entry of the factor; n <= 112 is the unblocked kernel, 130 the
    blocked one.  The upper triangle comes back zero; only the lower triangle of G is read
    (the strict upper triangle here holds garbage)."""
    ctx = hwmod.Context(0)
    g = np.random.default_rng(100 + n)
    mats = []
    for b in range(3):
        X = g.standard_normal((2 * n + 8, n)) + 1j * g.standard_normal((2 * n + 8, n))
        X *= np.exp(g.uniform(-1.0, 1.0, n))        # column scales
        mats.append(X.conj().T @ X)
    A = np.stack(mats)
    Ag = A.copy()
    iu = np.triu_indices(n, 1)
    for b in range(3):
        Ag[b][iu] = 7.0 - 5.0j                        # never read
    Gt = torch.from_numpy(np.ascontiguousarray(np.transpose(Ag, (0, 2, 1)))).cuda()
    L, fail = hwmod.hw_cholesky(ctx.h, Gt, prec)
    assert fail == [0, 0, 0]
    L = np.transpose(L.cpu().numpy(), (0, 2, 1))      # back to L[b][i][j]
    for b in range(3):
        ref = np.linalg.cholesky(A[b])
        err = np.abs(L[b] - ref).max() / np.abs(ref).max()
        assert err < tol, (b, err)
        assert np.all(L[b][iu] == 0)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [40, 130])
def test_cholesky_reports_the_first_bad_pivot(hwmod, prec, n):
    """A Hermitian matrix whose leading 9 x 9 block is positive definite and whose 10th pivot is
    negative: fail = 10 (1 + its column); the other problem of the batch factors normally."""
    ctx = hwmod.Context(0)
    g = np.random.default_rng(7)
    X = g.standard_normal((2 * n, n)) + 1j * g.standard_normal((2 * n, n))
    good = X.conj().T @ X
    bad = good.copy()
    # make the Schur complement at column 9 negative: set G[9][9] below the part explained by
    # the first 9 columns
    L9 = np.linalg.cholesky(good[:9, :9])
    v = np.linalg.solve(L9, good[:9, 9])
    bad[9, 9] = np.vdot(v, v).real - 1.0
    A = np.stack([good, bad])
    Gt = torch.from_numpy(np.ascontiguousarray(np.transpose(A, (0, 2, 1)))).cuda()
    _, fail = hwmod.hw_cholesky(ctx.h, Gt, prec)
    assert fail == [0, 10]
    ctx.close()
