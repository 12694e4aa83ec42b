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
