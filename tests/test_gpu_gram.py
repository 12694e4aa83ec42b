"""hw_gram (FP32 products, FP64 accumulation every 32 rows) against a plain FP64 product.

Bounds: each entry's error is at most 2^-23 (two roundings of the factors) plus 32 FP32
additions of at most 2^-24 of a partial sum of 32 terms, i.e. below 2.5e-6 of
sum_k |a_k||b_k| in the worst case; the test checks that bound entry by entry and that the
typical error is far smaller (random rounding signs)."""
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


def crand(g, *shape):
    return torch.from_numpy(g.standard_normal(shape) + 1j * g.standard_normal(shape))


@pytest.mark.parametrize("nprob,m,n,K", [(1, 216, 216, 5066), (3, 72, 144, 1000), (2, 5, 33, 31), (1, 1, 1, 257)])
def test_gram_matches_fp64(hwmod, nprob, m, n, K):
    g = np.random.default_rng(m * 7 + n + K)
    A = (crand(g, nprob, m, K) / np.sqrt(K)).cuda()
    B = (crand(g, nprob, n, K) * 3.0).cuda()
    ctx = hwmod.Context(0)
    C = hwmod.hw_gram(ctx.h, A, B)                       # (nprob, n, m): row j = column j
    ref = torch.einsum("bik,bjk->bji", A.conj(), B)
    bound = torch.einsum("bik,bjk->bji", A.abs(), B.abs())
    err = (C - ref).abs()
    assert (err <= 2.5e-6 * bound).all()
    rel = (err / bound).max().item()
    assert rel < 2e-7, rel
    ctx.close()


def test_gram_hermitian_gram_of_one_block(hwmod):
    """A^H A: exactly Hermitian in exact arithmetic; the diagonal (a coherent sum) to 1e-7."""
    g = np.random.default_rng(3)
    A = crand(g, 1, 72, 5066).cuda()
    ctx = hwmod.Context(0)
    C = hwmod.hw_gram(ctx.h, A, A)[0]
    ref = (A[0].conj() @ A[0].T).T
    d = torch.diagonal(C).real
    assert ((d - torch.diagonal(ref).real).abs() / torch.diagonal(ref).real).max().item() < 1e-7
    assert (C - ref).abs().max().item() < 1e-6 * torch.diagonal(ref).real.max().item()
    ctx.close()


def test_gram_rejects_bad_sizes(hwmod):
    A = torch.zeros((1, 4, 8), dtype=torch.complex128, device="cuda")
    ctx = hwmod.Context(0)
    with pytest.raises(hwmod.HwError) as e:
        hwmod.load_library().hw_gram  # noqa: B018 (symbol present)
        st = hwmod.load_library().hw_gram(ctx.h, 4, 4, 8, 1, A.data_ptr(), 4, 32, A.data_ptr(), 8, 32,
                                          A.data_ptr(), 4, 16)   # lda < K
        hwmod._check(ctx.h, st)
    assert e.value.status == hwmod.HW_EINVAL
    ctx.close()
