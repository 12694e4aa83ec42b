"""hw_apply_H_noalloc: the H X entry point for callers that cannot allocate device memory.

It must give the same product as hw_apply_H (same kernels, intermediates in the library's
fixed 64 MiB device array instead of the context workspace).  Two calls in a row with
different inputs check that the array's leftover contents never leak into a result; 100
columns of the tube basis need two passes through the array.  Collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_12252_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


def rel_err(Y, Yref):
    return ((Y - Yref).abs().pow(2).sum(dim=1).sqrt() / Yref.abs().pow(2).sum(dim=1).sqrt()).max().item()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_noalloc_matches_apply_H_on_two_calls(hwmod, prec, tol):
    w = inputs.tube()
    ctx = hwmod.Context(0)
    L = int(ctx.setup_basis(w.geom, w.etas)[0])
    ctx.build_potential(w.atoms)
    ns, ld = 100, L + 6
    code = {"fp64": hwmod.HW_FP64, "mixed": hwmod.HW_MIXED}[prec]
    for call in range(2):
        X = torch.zeros((ns, ld), dtype=torch.complex128)
        X[:, :L] = torch.from_numpy(np.ascontiguousarray(inputs.random_block(L, ns, 500 + call).T))
        X = X.cuda()
        Yref = torch.zeros_like(X)
        hwmod.hw_apply_H(ctx.h, 0, X.data_ptr(), Yref.data_ptr(), ns, ld, code)
        Y = torch.full_like(X, complex(3.0, 1.0))
        hwmod.hw_apply_H_noalloc(ctx.h, 0, X.data_ptr(), Y.data_ptr(), ns, ld, code)
        torch.cuda.synchronize()
        assert rel_err(Y[:, :L], Yref[:, :L]) < tol
        assert torch.all(Y[:, L:] == complex(3.0, 1.0))   # padding rows untouched
    ctx.close()


def test_noalloc_rejects_bad_arguments(hwmod):
    w = inputs.tiny()
    ctx = hwmod.Context(0)
    L = int(ctx.setup_basis(w.geom, w.etas)[0])
    ctx.build_potential(w.atoms)
    X = torch.zeros((2, L), dtype=torch.complex128, device="cuda")
    with pytest.raises(hwmod.HwError) as e:
        hwmod.hw_apply_H_noalloc(ctx.h, 0, X.data_ptr(), X.data_ptr(), 2, L)
    assert e.value.status == hwmod.HW_EINVAL
    with pytest.raises(hwmod.HwError) as e:
        hwmod.hw_apply_H_noalloc(ctx.h, 0, X.data_ptr(), X.data_ptr() + 16, 2, L - 1)
    assert e.value.status == hwmod.HW_EINVAL
    ctx.close()
