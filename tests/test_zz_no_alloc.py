"""hw_apply_H_noalloc: the H X entry point for callers that cannot allocate device memory.

It must give the same product as hw_apply_H (same kernels and launch configuration, the
intermediates in the library's fixed 64 MiB device array instead of the context workspace).
Two calls in a row with different inputs check that the array's leftover contents never leak
into a result.  The column count is chosen per precision from the array's capacity (one
column of the tube basis needs 2 N_r n_pairs complex values: 83 columns fit per pass in FP64,
167 in mixed precision) so that both precisions take two passes, the second one short.
Collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_12252_gb300 import inputs
from _parity import assert_entrywise

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 64 << 20


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
    elem = 16 if prec == "fp64" else 8
    per_pass = SCRATCH_BYTES // (2 * w.geom.Nr * ctx.sizes["n_pairs"] * elem)
    ns = per_pass + per_pass // 5 + 1          # two passes, the second about a fifth as wide
    assert per_pass < ns < 2 * per_pass
    ld = L + 6
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
        assert_entrywise(Y[:, :L].cpu().numpy().T, Yref[:, :L].cpu().numpy().T, tol, tol * 1e-3,
                         f"noalloc {prec} call {call}")
        assert torch.all(Y[:, L:] == complex(3.0, 1.0))   # padding rows untouched
    ctx.close()


def test_noalloc_rejects_bad_arguments(hwmod):
    w = inputs.tiny()
    ctx = hwmod.Context(0)
    L = int(ctx.setup_basis(w.geom, w.etas)[0])
    ctx.build_potential(w.atoms)
    X = torch.zeros((3, L), dtype=torch.complex128, device="cuda")
    with pytest.raises(hwmod.HwError) as e:
        hwmod.hw_apply_H_noalloc(ctx.h, 0, X.data_ptr(), X.data_ptr(), 2, L)
    assert e.value.status == hwmod.HW_EINVAL
    with pytest.raises(hwmod.HwError) as e:
        hwmod.hw_apply_H_noalloc(ctx.h, 0, X.data_ptr(), X.data_ptr() + 16, 2, L - 1)
    assert e.value.status == hwmod.HW_EINVAL
    # Y starting inside X's second column: a partial overlap
    with pytest.raises(hwmod.HwError) as e:
        hwmod.hw_apply_H_noalloc(ctx.h, 0, X.data_ptr(), X[1].data_ptr(), 2, L)
    assert e.value.status == hwmod.HW_EINVAL and "overlap" in str(e.value)
    ctx.close()
