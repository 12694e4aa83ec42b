"""Thin Python binding of the C ABI in include/helicwave.h (argument marshalling only).

The module-level functions carry the C names (hw_create, hw_setup_basis, hw_apply_H, ...) and
take plain integers / pointers; `Context` wraps them for torch tensors.  Every computation runs
in libhelicwave.so; importing this module fails loudly when that library has not been built.

Block layout: a column-major complex128 block L x ns with leading dimension ld is a contiguous
torch tensor of shape (ns, ld) and dtype complex128 (row j holds column j).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhelicwave.so")

HW_OK, HW_EINVAL, HW_ENOMEM, HW_ECUDA, HW_ESTATE, HW_ENOTCONV, HW_ETIMEOUT = range(7)
HW_FP64, HW_MIXED, HW_FP64_DF = 0, 1, 2
HW_PRECOND_TPA, HW_PRECOND_LEARNED, HW_PRECOND_NONE = 0, 1, 2
STATUS_NAMES = ["HW_OK", "HW_EINVAL", "HW_ENOMEM", "HW_ECUDA", "HW_ESTATE", "HW_ENOTCONV",
                "HW_ETIMEOUT"]


class HwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class hw_basis_params(C.Structure):
    _fields_ = [("R", C.c_double), ("tau", C.c_double), ("alpha", C.c_double),
                ("ncyc", C.c_int), ("ecut", C.c_double), ("Nr", C.c_int), ("Nth1", C.c_int),
                ("Nth2", C.c_int), ("oversample", C.c_int)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "hw_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "hw_destroy": (None, [C.c_void_p]),
    "hw_last_error": (C.c_char_p, [C.c_void_p]),
    "hw_setup_basis": (C.c_int, [C.c_void_p, C.POINTER(hw_basis_params), C.c_int, _D, _D, _D,
                                 C.POINTER(C.c_int64)]),
    "hw_get_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                               C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "hw_get_grid": (C.c_int, [C.c_void_p, _D, _D]),
    "hw_get_index_map": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int32)]),
    "hw_get_kinetic": (C.c_int, [C.c_void_p, C.c_int, _D]),
    "hw_get_radial_table": (C.c_int, [C.c_void_p, C.c_int, _D]),
    "hw_get_itable": (C.c_int, [C.c_void_p, C.c_int, _D]),
    "hw_set_potential": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "hw_build_potential": (C.c_int, [C.c_void_p, C.c_int, _D, _D]),
    "hw_apply_H": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int64,
                             C.c_int]),
    "hw_apply_H_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int64,
                                     C.c_int]),
    "hw_apply_H_batched": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int,
                                     C.c_int64, C.c_int]),
    "hw_apply_precond": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                   C.c_int64, C.c_void_p, C.c_int]),
    "hw_solve_eigs": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int,
                                C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p),
                                _D, C.POINTER(C.c_void_p), C.c_int64, C.POINTER(C.c_int), _D]),
    "hw_synchronize": (C.c_int, [C.c_void_p]),
    "hw_set_option": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "hw_get_option": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_longlong)]),
    "hw_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_float), C.c_int,
                              C.POINTER(C.c_int)]),
    "hw_heev": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                          C.c_int]),
    "hw_cholesky": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_int),
                              C.c_int]),
    "hw_get_residual_history": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), _D, C.c_int,
                                         C.POINTER(C.c_int)]),
    "hw_selftest_barrier": (C.c_int, [C.c_void_p, C.c_int, C.c_longlong, C.c_int, C.POINTER(C.c_int)]),
    "hw_density": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_void_p), C.c_int, C.c_int64,
                             _D, _D, C.c_void_p, C.c_int]),
    "hw_gradient": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int64, C.c_void_p, C.c_int]),
    "hw_gram": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.c_int64,
                          C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_int64]),
    "hw_block_product": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p,
                                   C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_double,
                                   C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_int]),
    "hw_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "hw_profile_read": (C.c_int, [C.c_void_p, _D, C.POINTER(C.c_int64)]),
    "hw_profile_work": (C.c_int, [C.c_void_p, _D]),
    "hw_launch_count": (C.c_int64, [C.c_void_p]),
    "hw_set_mlp": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int64]),
    "hw_get_mlp": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int64]),
    "hw_get_potential_diagonal": (C.c_int, [C.c_void_p, C.c_int, _D]),
    "hw_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, _D, C.c_int,
                                   C.c_int64, C.c_void_p, _D, C.POINTER(C.c_float)]),
    "hw_mlp_train_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, _D, C.c_int,
                                    C.c_int64, C.c_void_p, C.c_float, _D]),
    "hw_solve_eigs_traced": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                       C.c_int, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                       C.c_void_p, C.c_void_p, _D, _D, C.c_int64, _D,
                                       C.POINTER(C.c_int)]),
}

MLP_NPARAM = 4673

PHASES = ["radial_inv", "slab", "radial_fwd", "precond", "gemm", "chol", "eig", "other", "mlp", "tridiag",
          "density", "gradient"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhelicwave.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2210_12252_gb300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return sorted(_SIGS)


def _dptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


# ----------------------------------------------------------------- C-named thin wrappers

def hw_create(device: int = 0, stream: int = 0):
    lib = load_library()
    h = C.c_void_p()
    st = lib.hw_create(C.byref(h), device, C.c_void_p(stream or None))
    if st != HW_OK:
        raise HwError(st, "hw_create failed")
    return h


def hw_destroy(h):
    load_library().hw_destroy(h)


def hw_last_error(h) -> str:
    return load_library().hw_last_error(h).decode()


def _check(h, st):
    if st != HW_OK:
        raise HwError(st, hw_last_error(h))


def hw_setup_basis(h, params: hw_basis_params, eta, nu=None, ecut_per_k=None):
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    nk = eta.size
    nu = None if nu is None else np.ascontiguousarray(nu, dtype=np.float64)
    ec = None if ecut_per_k is None else np.ascontiguousarray(ecut_per_k, dtype=np.float64)
    L = np.zeros(nk, dtype=np.int64)
    _check(h, load_library().hw_setup_basis(h, C.byref(params), nk, _dptr(eta), _dptr(nu),
                                            _dptr(ec), L.ctypes.data_as(C.POINTER(C.c_int64))))
    return L


def hw_get_sizes(h):
    M, N, K, nA = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    G = C.c_int64()
    _check(h, load_library().hw_get_sizes(h, C.byref(M), C.byref(N), C.byref(K), C.byref(G),
                                          C.byref(nA)))
    return dict(M=M.value, N=N.value, K=K.value, grid_points=G.value, n_pairs=nA.value)


def hw_get_grid(h, Nr):
    r = np.zeros(Nr)
    w = np.zeros(Nr)
    _check(h, load_library().hw_get_grid(h, _dptr(r), _dptr(w)))
    return r, w


def hw_get_index_map(h, k, L):
    out = np.zeros(3 * L, dtype=np.int32)
    _check(h, load_library().hw_get_index_map(h, k, out.ctypes.data_as(C.POINTER(C.c_int32))))
    return out.reshape(L, 3)


def hw_get_kinetic(h, k, L):
    out = np.zeros(L)
    _check(h, load_library().hw_get_kinetic(h, k, _dptr(out)))
    return out


def hw_get_radial_table(h, n, Nr, K):
    out = np.zeros(Nr * K)
    _check(h, load_library().hw_get_radial_table(h, n, _dptr(out)))
    return out.reshape(Nr, K)


def hw_get_itable(h, n, K):
    out = np.zeros(K * K)
    _check(h, load_library().hw_get_itable(h, n, _dptr(out)))
    return out.reshape(K, K)


def hw_set_potential(h, V_ptr: int, on_device: bool):
    _check(h, load_library().hw_set_potential(h, C.c_void_p(V_ptr), int(bool(on_device))))


def hw_build_potential(h, atoms, grid_points):
    atoms = np.ascontiguousarray(np.asarray(atoms, dtype=np.float64).reshape(-1, 5))
    V = np.zeros(grid_points)
    _check(h, load_library().hw_build_potential(h, atoms.shape[0], _dptr(atoms), _dptr(V)))
    return V


def hw_apply_H(h, k, X_ptr, Y_ptr, ns, ld, prec=HW_FP64):
    _check(h, load_library().hw_apply_H(h, k, C.c_void_p(X_ptr), C.c_void_p(Y_ptr), ns, ld, prec))


def hw_apply_H_noalloc(h, k, X_ptr, Y_ptr, ns, ld, prec=HW_FP64):
    """H X through the entry point that allocates nothing (fixed 64 MiB device scratch)."""
    _check(h, load_library().hw_apply_H_noalloc(h, k, C.c_void_p(X_ptr), C.c_void_p(Y_ptr), ns, ld,
                                                prec))


def hw_apply_H_batched(h, kidx, X_ptrs, Y_ptrs, ns, ld, prec=HW_FP64):
    nk = len(kidx)
    ki = (C.c_int * nk)(*kidx)
    xs = (C.c_void_p * nk)(*X_ptrs)
    ys = (C.c_void_p * nk)(*Y_ptrs)
    _check(h, load_library().hw_apply_H_batched(h, nk, ki, xs, ys, ns, ld, prec))


def hw_apply_precond(h, k, R_ptr, Z_ptr, ns, ld, ritz_ptr=0, kind=HW_PRECOND_TPA):
    _check(h, load_library().hw_apply_precond(h, k, C.c_void_p(R_ptr), C.c_void_p(Z_ptr), ns, ld,
                                              C.c_void_p(ritz_ptr or None), kind))


def hw_solve_eigs(h, kidx, n_eig, block=0, tol=1e-6, maxit=500, prec=HW_FP64,
                  precond=HW_PRECOND_TPA, X0_ptrs=None, evec_ptrs=None, ld_evecs=0):
    nk = len(kidx)
    ki = (C.c_int * nk)(*kidx)
    x0 = (C.c_void_p * nk)(*X0_ptrs) if X0_ptrs is not None else None
    ev = (C.c_void_p * nk)(*evec_ptrs) if evec_ptrs is not None else None
    evals = np.zeros(nk * n_eig)
    resid = np.zeros(nk * n_eig)
    iters = (C.c_int * nk)()
    st = load_library().hw_solve_eigs(h, nk, ki, n_eig, block, tol, maxit, prec, precond, x0,
                                      _dptr(evals), ev, ld_evecs, iters, _dptr(resid))
    if st not in (HW_OK, HW_ENOTCONV):
        _check(h, st)
    return (evals.reshape(nk, n_eig), np.array(list(iters)), resid.reshape(nk, n_eig),
            st == HW_OK)


def hw_synchronize(h):
    _check(h, load_library().hw_synchronize(h))


HW_OPT_RR_METHOD = 0
HW_OPT_RR_FALLBACKS = 1
HW_OPT_LOWP_SWITCH = 2
HW_OPT_GRAM_KERNEL = 3
HW_OPT_HYBRID = 4
HW_OPT_EIGENSOLVER = 5
HW_OPT_CHEB_DEGREE = 6
HW_OPT_CHEB_ADAPT = 7
HW_OPT_CHEB_LOCK = 8
HW_OPT_SLAB_KERNEL = 9
HW_OPT_TAIL_NO_P = 10
HW_OPT_WINDOW = 11
HW_OPT_TC_GEMM = 12
HW_OPT_RADIAL_KERNEL = 13
HW_OPT_FP64_HX = 14
HW_OPT_SMALL_GEMM = 15
HW_OPT_OVERLAP_LAUNCH = 16


def hw_set_option(h, option, value):
    _check(h, load_library().hw_set_option(h, option, value))


def hw_density(h, kidx, X, ns, ld, occ, w, rho_ptr, prec=HW_FP64):
    """rho (device pointer, N_th1*N_th2*N_r doubles) = (2/Ncyc) sum_b w[b] sum_j occ[b][j] |phi_bj|^2."""
    nk = len(kidx)
    ki = (C.c_int * nk)(*[int(k) for k in kidx])
    xp = (C.c_void_p * nk)(*[int(x) for x in X])
    occ = np.ascontiguousarray(occ, dtype=np.float64).reshape(-1)
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
    if occ.size != nk * ns or w.size != nk:
        raise ValueError("occ must hold nk*ns values and w nk")
    _check(h, load_library().hw_density(h, nk, ki, xp, ns, ld, _dptr(occ), _dptr(w), C.c_void_p(rho_ptr), prec))


def hw_gram(h, A, B):
    """C_b = A_b^H B_b for torch complex128 tensors A (nprob, m, ld) and B (nprob, n, ld) whose
    rows are the columns of the K x m / K x n blocks (K = the last dimension); returns C as
    (nprob, n, m) (row j = column j)."""
    import torch
    nprob, m, K = A.shape
    n = B.shape[1]
    C = torch.empty((nprob, n, m), dtype=torch.complex128, device=A.device)
    _check(h, load_library().hw_gram(h, m, n, K, nprob, A.data_ptr(), K, m * K, B.data_ptr(), K, n * K,
                                     C.data_ptr(), m, m * n))
    return C


def hw_get_option(h, option):
    v = C.c_longlong(0)
    _check(h, load_library().hw_get_option(h, option, C.byref(v)))
    return int(v.value)


def hw_autotune(h, k, ns):
    """Tune the H X tile shapes; returns rows (precision, theta2 chunk, pass columns, ms)."""
    buf = np.zeros(4 * 256, dtype=np.float32)
    nr = C.c_int()
    _check(h, load_library().hw_autotune(h, k, ns, buf.ctypes.data_as(C.POINTER(C.c_float)), 256,
                                         C.byref(nr)))
    return buf[: 4 * min(nr.value, 256)].reshape(-1, 4)


def hw_heev(h, A, nw, method=1):
    """A: (nprob, n, n) complex128 CUDA tensor of Hermitian matrices (row j of A[b] holds
    column j).  Returns (w, Z) as CUDA tensors: w (nprob, n), Z (nprob, n, n) with Z[b][j] the
    j-th eigenvector."""
    import torch
    nprob, n, _ = A.shape
    A = A.contiguous()
    w = torch.zeros((nprob, n), dtype=torch.float64, device=A.device)
    Z = torch.zeros_like(A)
    _check(h, load_library().hw_heev(h, n, nprob, nw, C.c_void_p(A.data_ptr()), C.c_void_p(w.data_ptr()),
                                     C.c_void_p(Z.data_ptr()), method))
    return w, Z


def hw_cholesky(h, G, prec="fp64"):
    """G: (nprob, n, n) complex128 CUDA tensor of Hermitian positive definite matrices (row j of
    G[b] holds column j; only the lower triangle of each matrix is read; G is overwritten).
    Returns (L, fail): L (nprob, n, n) with L[b][j] column j of the lower factor, fail a list of
    0 or 1 + the column of a bad pivot."""
    import torch
    nprob, n, _ = G.shape
    L = torch.zeros_like(G)
    fail = (C.c_int * nprob)()
    _check(h, load_library().hw_cholesky(h, n, nprob, C.c_void_p(G.data_ptr()), C.c_void_p(L.data_ptr()), fail,
                                         _PREC[prec]))
    return L, list(fail)


HW_HIST_FILTER_FP32, HW_HIST_FILTER_FP64, HW_HIST_LOBPCG_FP32, HW_HIST_LOBPCG_HYBRID, HW_HIST_LOBPCG_FP64 = range(5)
HIST_PHASES = ["filter_fp32", "filter_fp64", "lobpcg_fp32", "lobpcg_hybrid", "lobpcg_fp64"]


def hw_get_residual_history(h, k):
    """Residual history of the last solve at k-point k: list of (phase name, largest wanted
    residual) per filter cycle / LOBPCG iteration."""
    n = C.c_int(0)
    _check(h, load_library().hw_get_residual_history(h, k, None, None, 0, C.byref(n)))
    ph = np.zeros(max(n.value, 1), dtype=np.int32)
    res = np.zeros(max(n.value, 1))
    _check(h, load_library().hw_get_residual_history(h, k, ph.ctypes.data_as(C.POINTER(C.c_int)), _dptr(res),
                                                      n.value, C.byref(n)))
    return [(HIST_PHASES[int(p)], float(r)) for p, r in zip(ph[:n.value], res[:n.value])]


def hw_selftest_barrier(h, nblocks, spin_limit, skip_block):
    """Run the bounded grid-barrier self-test; returns the kernel's status word (HW_OK or
    HW_ETIMEOUT)."""
    ws = C.c_int(-1)
    _check(h, load_library().hw_selftest_barrier(h, nblocks, spin_limit, skip_block, C.byref(ws)))
    return int(ws.value)


def hw_block_product(h, trans_a, m, n, k, A, B, C, alpha=1.0, beta=0.0, cls=0):
    """C_b = alpha op(A_b) B_b + beta C_b on the tensor cores.  A, B, C: contiguous CUDA complex128
    tensors of shape (batch, columns, ld): block b's column c is A[b, c, :ld] (column-major
    blocks, leading dimension = the last extent).  op = conjugate transpose when trans_a
    (A_b: k x m), else none (A_b: m x k).  cls 0: FP64 class, 1: FP32 class (tensor cores);
    2, 3: the small-product kernel (every extent below 1024) in double-float and FP32."""
    for T in (A, B, C):
        assert T.is_contiguous() and T.dim() == 3
    batch = C.shape[0]
    _check(h, load_library().hw_block_product(
        h, int(trans_a), m, n, k, float(alpha), A.data_ptr(),
        A.shape[2], A.shape[1] * A.shape[2], B.data_ptr(), B.shape[2], B.shape[1] * B.shape[2], float(beta),
        C.data_ptr(), C.shape[2], C.shape[1] * C.shape[2], batch, cls))


def hw_profile(h, enable: bool):
    _check(h, load_library().hw_profile(h, int(bool(enable))))


def hw_profile_read(h):
    ms = np.zeros(len(PHASES))
    cnt = np.zeros(len(PHASES), dtype=np.int64)
    _check(h, load_library().hw_profile_read(h, _dptr(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64))))
    return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}


def hw_profile_work(h):
    work = np.zeros(len(PHASES))
    _check(h, load_library().hw_profile_work(h, _dptr(work)))
    return {p: float(work[i]) for i, p in enumerate(PHASES)}


def hw_launch_count(h) -> int:
    return int(load_library().hw_launch_count(h))


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def hw_set_mlp(h, params):
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
    _check(h, load_library().hw_set_mlp(h, _fptr(p), p.size))


def hw_get_mlp(h):
    p = np.zeros(MLP_NPARAM, dtype=np.float32)
    _check(h, load_library().hw_get_mlp(h, _fptr(p), p.size))
    return p


def hw_get_potential_diagonal(h, k, L):
    out = np.zeros(L)
    _check(h, load_library().hw_get_potential_diagonal(h, k, _dptr(out)))
    return out


def hw_mlp_loss_grad(h, k, R_ptr, E_ptr, ritz, ns, ld, vdiag_ptr=0, want_grad=True):
    ritz = np.ascontiguousarray(ritz, dtype=np.float64)
    loss = np.zeros(1)
    g = np.zeros(MLP_NPARAM, dtype=np.float32) if want_grad else None
    _check(h, load_library().hw_mlp_loss_grad(h, k, C.c_void_p(R_ptr), C.c_void_p(E_ptr), _dptr(ritz),
                                              ns, ld, C.c_void_p(vdiag_ptr or None), _dptr(loss),
                                              _fptr(g) if g is not None else None))
    return float(loss[0]), g


def hw_mlp_train_step(h, k, R_ptr, E_ptr, ritz, ns, ld, lr, vdiag_ptr=0):
    ritz = np.ascontiguousarray(ritz, dtype=np.float64)
    loss = np.zeros(1)
    _check(h, load_library().hw_mlp_train_step(h, k, C.c_void_p(R_ptr), C.c_void_p(E_ptr), _dptr(ritz),
                                               ns, ld, C.c_void_p(vdiag_ptr or None), C.c_float(lr),
                                               _dptr(loss)))
    return float(loss[0])


def hw_solve_eigs_traced(h, k, n_eig, block, tol, maxit, prec, precond, X0_ptr, rec_iters,
                         rec_R_ptr, rec_E_ptr, ld):
    n_rec = len(rec_iters)
    ri = (C.c_int * max(n_rec, 1))(*rec_iters)
    th = np.zeros(n_rec * block)
    rs = np.zeros(n_rec * block)
    ev = np.zeros(n_eig)
    it = (C.c_int * 1)()
    st = load_library().hw_solve_eigs_traced(h, k, n_eig, block, tol, maxit, prec, precond,
                                             C.c_void_p(X0_ptr or None), n_rec, ri,
                                             C.c_void_p(rec_R_ptr), C.c_void_p(rec_E_ptr),
                                             _dptr(th), _dptr(rs), ld, _dptr(ev), it)
    if st not in (HW_OK, HW_ENOTCONV):
        _check(h, st)
    return ev, int(it[0]), th.reshape(n_rec, block), rs.reshape(n_rec, block), st == HW_OK


# ----------------------------------------------------------------------------- Context

_PREC = {"fp64": HW_FP64, "mixed": HW_MIXED, "fp64_df": HW_FP64_DF}
_PRECOND = {"tpa": HW_PRECOND_TPA, "learned": HW_PRECOND_LEARNED, "none": HW_PRECOND_NONE}


class Context:
    """One library context on one device (device=-1: host-only, setup queries only)."""

    def __init__(self, device: int = 0, stream=None):
        self.device = device
        if device >= 0:
            import torch
            if stream is None:
                stream = torch.cuda.current_stream(device)
            self.stream = stream
            sp = stream.cuda_stream
        else:
            self.stream = None
            sp = 0
        self.h = hw_create(device, sp)
        self.L = None

    def close(self):
        if self.h is not None:
            hw_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup
    def setup_basis(self, geom, etas, nus=None, ecuts=None):
        self.geom = geom
        p = hw_basis_params(geom.R, geom.tau, geom.alpha, geom.ncyc, geom.ecut, geom.Nr,
                            geom.Nth1, geom.Nth2, geom.oversample)
        self.L = hw_setup_basis(self.h, p, etas, nus, ecuts)
        self.sizes = hw_get_sizes(self.h)
        return self.L

    def grid(self):
        return hw_get_grid(self.h, self.geom.Nr)

    def index_map(self, k):
        return hw_get_index_map(self.h, k, int(self.L[k]))

    def kinetic(self, k):
        return hw_get_kinetic(self.h, k, int(self.L[k]))

    def radial_table(self, n):
        return hw_get_radial_table(self.h, n, self.geom.Nr, self.sizes["K"])

    def itable(self, n):
        return hw_get_itable(self.h, n, self.sizes["K"])

    def build_potential(self, atoms):
        return hw_build_potential(self.h, atoms, self.sizes["grid_points"])

    def set_potential(self, V):
        import torch
        if isinstance(V, torch.Tensor) and V.is_cuda:
            V = V.contiguous().to(torch.float64)
            hw_set_potential(self.h, V.data_ptr(), True)
            self._vkeep = V
        else:
            V = np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(-1))
            hw_set_potential(self.h, V.ctypes.data, False)

    # -- compute
    @staticmethod
    def _blk(X):
        assert X.dtype.is_complex and X.element_size() == 16 and X.is_contiguous()
        return X.shape[0], X.shape[1]

    def apply_H(self, k, X, Y=None, prec="fp64"):
        import torch
        ns, ld = self._blk(X)
        if Y is None:
            Y = torch.zeros_like(X)
        hw_apply_H(self.h, k, X.data_ptr(), Y.data_ptr(), ns, ld, _PREC[prec])
        return Y

    def apply_H_batched(self, kidx, Xs, Ys, prec="fp64"):
        ns, ld = self._blk(Xs[0])
        hw_apply_H_batched(self.h, list(kidx), [x.data_ptr() for x in Xs],
                           [y.data_ptr() for y in Ys], ns, ld, _PREC[prec])
        return Ys

    def apply_precond(self, k, R, Z=None, ritz=None, kind="tpa"):
        import torch
        ns, ld = self._blk(R)
        if Z is None:
            Z = torch.empty_like(R)
        hw_apply_precond(self.h, k, R.data_ptr(), Z.data_ptr(), ns, ld,
                         ritz.data_ptr() if ritz is not None else 0, _PRECOND[kind])
        return Z

    def solve_eigs(self, kidx, n_eig, block=0, tol=1e-6, maxit=500, prec="fp64",
                   precond="tpa", X0=None, vectors=False):
        import torch
        evecs = None
        ptrs = None
        if vectors:
            Lmax = int(max(self.L[k] for k in kidx))
            evecs = [torch.zeros((n_eig, Lmax), dtype=torch.complex128, device=f"cuda:{self.device}")
                     for _ in kidx]
            ptrs = [e.data_ptr() for e in evecs]
        x0p = [x.data_ptr() for x in X0] if X0 is not None else None
        ev, it, res, ok = hw_solve_eigs(self.h, list(kidx), n_eig, block, tol, maxit, _PREC[prec],
                                        _PRECOND[precond], x0p, ptrs,
                                        evecs[0].shape[1] if vectors else 0)
        return dict(evals=ev, iters=it, resid=res, converged=ok, evecs=evecs)

    def synchronize(self):
        hw_synchronize(self.h)

    def gradient(self, k, X, prec="fp64"):
        """Cartesian gradient on the grid of the functions with coefficient columns X (torch
        complex128 (ns, ld) on the device) at k-point k; returns a device tensor of shape
        (ns, 3, N_th1, N_th2, N_r) (components x, y, z)."""
        import torch
        ns, ld = self._blk(X)
        g = (ns, 3, self.geom.Nth1, self.geom.Nth2, self.geom.Nr)
        D = torch.empty(g, dtype=torch.complex128, device=X.device)
        _check(self.h, load_library().hw_gradient(self.h, k, C.c_void_p(X.data_ptr()), ns, ld,
                                                   C.c_void_p(D.data_ptr()), _PREC[prec]))
        return D

    def density(self, kidx, X, occ, w, prec="fp64"):
        """Electron density from state blocks X[b] (torch complex128 (ns, ld) on the device),
        occupations occ (nk, ns) and k-point weights w (nk); returns a device tensor of shape
        (N_th1, N_th2, N_r) (the potential's order)."""
        import torch
        code = {"fp64": HW_FP64, "mixed": HW_MIXED}[prec]
        ns, ld = X[0].shape
        g = (self.geom.Nth1, self.geom.Nth2, self.geom.Nr)
        rho = torch.empty(g, dtype=torch.float64, device=X[0].device)
        hw_density(self.h, list(kidx), [x.data_ptr() for x in X], ns, ld, occ, w, rho.data_ptr(), code)
        return rho

    def set_option(self, option, value):
        hw_set_option(self.h, option, value)

    def get_option(self, option):
        return hw_get_option(self.h, option)

    def autotune(self, k=0, ns=64):
        return hw_autotune(self.h, k, ns)

    def profile(self, enable=True):
        hw_profile(self.h, enable)

    def profile_read(self):
        return hw_profile_read(self.h)

    def profile_work(self):
        return hw_profile_work(self.h)

    def launch_count(self):
        return hw_launch_count(self.h)

    # -- learned preconditioner
    def set_mlp(self, params):
        hw_set_mlp(self.h, params)

    def get_mlp(self):
        return hw_get_mlp(self.h)

    def potential_diagonal(self, k):
        return hw_get_potential_diagonal(self.h, k, int(self.L[k]))

    def mlp_loss_grad(self, k, R, E, ritz, vdiag=None, want_grad=True):
        ns, ld = self._blk(R)
        return hw_mlp_loss_grad(self.h, k, R.data_ptr(), E.data_ptr(), ritz, ns, ld,
                                vdiag.data_ptr() if vdiag is not None else 0, want_grad)

    def mlp_train_step(self, k, R, E, ritz, lr, vdiag=None):
        ns, ld = self._blk(R)
        return hw_mlp_train_step(self.h, k, R.data_ptr(), E.data_ptr(), ritz, ns, ld, lr,
                                 vdiag.data_ptr() if vdiag is not None else 0)

    def solve_traced(self, k, n_eig, block, rec_iters, tol=1e-6, maxit=500, prec="fp64",
                     precond="tpa", X0=None):
        """Solve at k-point k recording (R, E, theta, |r|) at the given iterations; returns
        evals, iterations, recorded R and E as (n_rec, block, L) tensors, theta, res, ok."""
        import torch
        L = int(self.L[k])
        n_rec = len(rec_iters)
        dev = f"cuda:{self.device}"
        R = torch.zeros((n_rec, block, L), dtype=torch.complex128, device=dev)
        E = torch.zeros_like(R)
        ev, it, th, rs, ok = hw_solve_eigs_traced(self.h, k, n_eig, block, tol, maxit, _PREC[prec],
                                                  _PRECOND[precond], X0.data_ptr() if X0 is not None else 0,
                                                  list(rec_iters), R.data_ptr(), E.data_ptr(), L)
        return dict(evals=ev, iters=it, R=R, E=E, theta=th, res=rs, converged=ok)
