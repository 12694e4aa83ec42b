"""The eigensolver's block products on the tensor cores (hw_block_product) against FP64 numpy.

C_b = alpha op(A_b) B_b + beta C_b with op = ^H (Gram matrices and projections: the reduction runs
over the basis dimension) or none (block updates: the rows run over it), on the shapes the
solver uses (tube basis L = 5066, blocks of 72 / 216 columns), ragged and batched shapes,
padded leading dimensions, and a nanowire-length reduction (L = 40,527: many drains of the
FP64 class's exact group sums).

Bounds, per entry, against the plain FP64 product (whose own error is ~1e-16 of |op(A)||B|):
  FP64 class (8 digits of 7 bits, exact sums): |dC_ij| <= 1e-13 (|op(A)| |B|)_ij
  FP32 class (3 digits of 8 bits, FP32 sums):   |dC_ij| <= 1e-5 (|op(A)| |B|)_ij
(the operands' dynamic range here is e^2; the splitting scales each row by its largest entry).
Both classes are deterministic: a repeated call gives the same bits.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 1e-5}


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


@pytest.fixture(scope="module")
def ctx(hwmod):
    c = hwmod.Context(0)
    yield c
    c.close()


def blocks(rng, batch, cols, rows, ld):
    """(batch, cols, ld) complex128: column-major blocks rows x cols, padding rows = 7 - 3i."""
    X = np.full((batch, cols, ld), 7.0 - 3.0j)
    mag = np.exp(rng.uniform(-2.0, 0.0, (batch, cols, rows)))
    X[:, :, :rows] = mag * (rng.standard_normal((batch, cols, rows)) + 1j * rng.standard_normal((batch, cols, rows)))
    return X


def run_case(hwmod, ctx, trans, m, n, k, batch=1, pad=(0, 0, 0), alpha=1.0, beta=0.0, cls=0, seed=0):
    rng = np.random.default_rng(seed)
    ra, ca = (k, m) if trans else (m, k)
    A = blocks(rng, batch, ca, ra, ra + pad[0])
    B = blocks(rng, batch, n, k, k + pad[1])
    C0 = blocks(rng, batch, n, m, m + pad[2])
    Ad, Bd, Cd = (torch.from_numpy(x.copy()).cuda() for x in (A, B, C0))
    hwmod.hw_block_product(ctx.h, trans, m, n, k, Ad, Bd, Cd, alpha, beta, cls)
    C = Cd.cpu().numpy()
    # again on a fresh output: the same bits
    Cd2 = torch.from_numpy(C0.copy()).cuda()
    hwmod.hw_block_product(ctx.h, trans, m, n, k, Ad, Bd, Cd2, alpha, beta, cls)
    assert np.array_equal(Cd2.cpu().numpy(), C)
    worst = 0.0
    for b in range(batch):
        a = A[b, :, :ra].T          # ra x ca
        bb = B[b, :, :k].T          # k x n
        opA = a.conj().T if trans else a
        ref = alpha * (opA @ bb) + beta * C0[b, :, :m].T
        scale = np.abs(alpha) * (np.abs(opA) @ np.abs(bb)) + abs(beta) * np.abs(C0[b, :, :m].T)
        d = np.abs(C[b, :, :m].T - ref)
        r = float((d / scale).max())
        worst = max(worst, r)
        assert r <= TOL[cls], (b, r)
        # padding rows of C untouched
        assert np.all(C[b, :, m:] == 7.0 - 3.0j)
    return worst


@pytest.mark.parametrize("cls", [0, 1])
def test_gram_tube_shape(hwmod, ctx, cls):
    r = run_case(hwmod, ctx, 1, 216, 216, 5066, cls=cls, seed=1)
    print(f"Gram 216 x 216 over 5066, class {cls}: max |dC|/(|A^H||B|) = {r:.3e}")


@pytest.mark.parametrize("cls", [0, 1])
def test_gram_ragged_batched_padded(hwmod, ctx, cls):
    r = run_case(hwmod, ctx, 1, 37, 53, 1000, batch=3, pad=(3, 5, 2), alpha=0.5, beta=-1.0, cls=cls, seed=2)
    print(f"Gram 37 x 53 over 1000 (3 problems), class {cls}: {r:.3e}")


@pytest.mark.parametrize("cls", [0, 1])
def test_update_tube_shape(hwmod, ctx, cls):
    r = run_case(hwmod, ctx, 0, 5066, 72, 216, batch=2, pad=(6, 0, 6), alpha=-1.0, beta=1.0, cls=cls, seed=3)
    print(f"update 5066 x 72 x 216 (2 problems), class {cls}: {r:.3e}")


@pytest.mark.parametrize("cls", [0, 1])
def test_small_square(hwmod, ctx, cls):
    r = run_case(hwmod, ctx, 0, 40, 24, 40, cls=cls, seed=4)
    r2 = run_case(hwmod, ctx, 1, 24, 40, 40, cls=cls, seed=5)
    print(f"small products, class {cls}: {r:.3e} {r2:.3e}")


def test_gram_nanowire_length(hwmod, ctx):
    """Reduction over 40,527 complex entries (81,054 real): 159 windows of exact group sums per
    output tile, spread over the reduction splits."""
    r = run_case(hwmod, ctx, 1, 64, 48, 40527, cls=0, seed=6)
    print(f"Gram 64 x 48 over 40527, class 0: {r:.3e}")


def test_block_product_rejects_bad_arguments(hwmod, ctx):
    A = torch.zeros((1, 4, 8), dtype=torch.complex128, device="cuda")
    for args in ((2, 4, 4, 8), (1, 0, 4, 8), (1, 4, 4, 0)):
        with pytest.raises(hwmod.HwError) as e:
            hwmod.hw_block_product(ctx.h, args[0], args[1], args[2], args[3], A, A, A)
        assert e.value.status == hwmod.HW_EINVAL
    with pytest.raises(hwmod.HwError) as e:
        hwmod.hw_block_product(ctx.h, 1, 4, 4, 8, A, A, A, cls=4)
    assert e.value.status == hwmod.HW_EINVAL


SMALL_TOL = {2: 1e-12, 3: 2e-6}


@pytest.mark.parametrize("cls", [2, 3])
def test_small_products_refinement_shapes(hwmod, ctx, cls):
    """The small-product classes (the Rayleigh-Ritz refinement's shapes: n x nb x n with
    n = 228, nb = 76; the Newton-Schulz nb x nb x n), both ops, alpha/beta, a batch of 2,
    ragged tiles (n not a multiple of 8), padded leading dimensions; entry-wise against FP64
    relative to (|op(A)||B|)_ij."""
    worst = 0.0
    for (trans, m, n, k, pad, alpha, beta, seed) in ((0, 228, 76, 228, (0, 0, 0), 1.0, 0.0, 11),
                                                    (1, 228, 76, 228, (3, 0, 5), 1.0, 0.0, 12),
                                                    (1, 76, 76, 228, (0, 2, 0), 0.5, -1.0, 13),
                                                    (0, 228, 76, 76, (5, 0, 1), -1.0, 1.0, 14),
                                                    (1, 5, 3, 1, (0, 0, 0), 1.0, 0.0, 15)):
        rng = np.random.default_rng(seed)
        ra, ca = (k, m) if trans else (m, k)
        A = blocks(rng, 2, ca, ra, ra + pad[0])
        B = blocks(rng, 2, n, k, k + pad[1])
        C0 = blocks(rng, 2, n, m, m + pad[2])
        Ad, Bd, Cd = (torch.from_numpy(x.copy()).cuda() for x in (A, B, C0))
        hwmod.hw_block_product(ctx.h, trans, m, n, k, Ad, Bd, Cd, alpha, beta, cls)
        C = Cd.cpu().numpy()
        for b in range(2):
            a = A[b, :, :ra].T
            opA = a.conj().T if trans else a
            ref = alpha * (opA @ B[b, :, :k].T) + beta * C0[b, :, :m].T
            scale = abs(alpha) * (np.abs(opA) @ np.abs(B[b, :, :k].T)) + abs(beta) * np.abs(C0[b, :, :m].T)
            r = float((np.abs(C[b, :, :m].T - ref) / scale).max())
            worst = max(worst, r)
            assert r <= SMALL_TOL[cls], (trans, m, n, k, b, r)
            assert np.all(C[b, :, m:] == 7.0 - 3.0j)
    print(f"small products, class {cls}: max |dC|/(|op(A)||B|) = {worst:.3e}")


def test_small_products_reject_large_extents(hwmod, ctx):
    A = torch.zeros((1, 1024, 1024), dtype=torch.complex128, device="cuda")
    with pytest.raises(hwmod.HwError) as e:
        hwmod.hw_block_product(ctx.h, 0, 1024, 8, 8, A, A, A, cls=2)
    assert e.value.status == hwmod.HW_EINVAL
