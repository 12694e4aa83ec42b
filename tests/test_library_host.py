"""CPU tests of libhelicwave.so: it loads, exports every symbol of include/helicwave.h, and its
host-side setup (radial rule, tables, cutoff masks, compact order, kinetic energies, the
Gaussian-well potential) matches the CPU oracle.  No device call is made (host-only context)."""
import os
import re

import numpy as np
import pytest

from oracle import basis as B
from oracle import potential as P
from paper_2210_12252_gb300 import build as hwbuild
from paper_2210_12252_gb300 import helicwave as hw
from paper_2210_12252_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    hwbuild.build()
    return hw.load_library()


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "helicwave.h")).read()
    return sorted(set(re.findall(r"\b(hw_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", hw.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (hw_[a-z_0-9]+)", out))
    declared = header_symbols()
    assert declared, "no declarations found"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    # and the binding covers them all
    assert set(declared) <= set(hw.exported_symbols()) | {"hw_create", "hw_destroy", "hw_last_error"}


def host_ctx(geom, etas, ecuts=None):
    ctx = hw.Context(device=-1)
    L = ctx.setup_basis(geom, etas, None, ecuts)
    return ctx, L


def oracle_basis(g):
    return B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)


@pytest.mark.parametrize("geom", [inputs.GEOM_TINY, inputs.GEOM_TUBE])
def test_radial_rule_and_tables_match_oracle(lib, geom):
    ctx, _ = host_ctx(geom, [0.0])
    b = oracle_basis(geom)
    r, w = ctx.grid()
    np.testing.assert_allclose(r, b.r, rtol=0, atol=1e-13 * geom.R)
    np.testing.assert_allclose(w, b.wr, rtol=1e-11, atol=1e-15)
    s = ctx.sizes
    assert (s["M"], s["N"], s["K"]) == (b.M, b.N, b.K)
    for n in range(-b.N, b.N + 1):
        np.testing.assert_allclose(ctx.radial_table(n), b.Rtab[n], rtol=0, atol=1e-12)


def test_masks_compact_order_and_kinetic_match_oracle(lib):
    g = inputs.GEOM_TUBE
    etas = np.array([0.0, 0.37, 0.91])
    ecuts = np.array([30.0, 12.5, 21.0])
    ctx, L = host_ctx(g, etas, ecuts)
    b = oracle_basis(g)
    for k, (eta, ec) in enumerate(zip(etas, ecuts)):
        kp = B.KPoint(b, eta, 0.0, ec)
        assert L[k] == kp.L
        mnk = ctx.index_map(k)
        np.testing.assert_array_equal(mnk[:, 0], kp.m)
        np.testing.assert_array_equal(mnk[:, 1], kp.n)
        np.testing.assert_array_equal(mnk[:, 2], kp.k)
        np.testing.assert_allclose(ctx.kinetic(k), kp.ke, rtol=1e-13, atol=1e-13)


def test_no_cutoff_keeps_the_whole_box(lib):
    ctx, L = host_ctx(inputs.GEOM_TINY, [0.0])
    assert L[0] == 7 * 7 * 6


def test_gaussian_potential_matches_oracle(lib):
    w = inputs.tiny()
    ctx, _ = host_ctx(w.geom, [0.0])
    V = ctx.build_potential(w.atoms)
    Vo = P.gaussian_wells(oracle_basis(w.geom), w.atoms).ravel()
    np.testing.assert_allclose(V, Vo, rtol=1e-13, atol=1e-14)


def test_setup_rejects_bad_arguments(lib):
    ctx = hw.Context(device=-1)
    bad = [
        inputs.Geometry(R=-1.0, tau=3.0, alpha=0.1, Nr=24, Nth1=16, Nth2=16, ecut=0.0),
        inputs.Geometry(R=6.0, tau=3.0, alpha=0.1, Nr=24, Nth1=20, Nth2=16, ecut=0.0),
        inputs.Geometry(R=6.0, tau=3.0, alpha=0.1, Nr=24, Nth1=16, Nth2=16, ecut=1e-6),
        inputs.Geometry(R=6.0, tau=3.0, alpha=0.1, Nr=1, Nth1=16, Nth2=16, ecut=0.0),
    ]
    for g in bad:
        with pytest.raises(hw.HwError) as e:
            ctx.setup_basis(g, [0.0])
        assert e.value.status == hw.HW_EINVAL
    with pytest.raises(hw.HwError) as e:
        ctx.setup_basis(inputs.GEOM_TINY, [0.0], nus=[float("nan")])
    assert e.value.status == hw.HW_EINVAL


def test_device_calls_on_host_context_are_rejected(lib):
    ctx, L = host_ctx(inputs.GEOM_TINY, [0.0])
    with pytest.raises(hw.HwError) as e:
        hw.hw_apply_H(ctx.h, 0, 0, 0, 1, int(L[0]))
    assert e.value.status == hw.HW_ESTATE
    # a solve, within one block and windowed (more eigenpairs than HW_OPT_WINDOW)
    for n_eig in (8, 120):
        with pytest.raises(hw.HwError) as e:
            hw.hw_solve_eigs(ctx.h, [0], n_eig)
        assert e.value.status == hw.HW_ESTATE, n_eig
    ctx.set_option(hw.HW_OPT_WINDOW, 4)
    with pytest.raises(hw.HwError) as e:
        hw.hw_solve_eigs(ctx.h, [0], 8)
    assert e.value.status == hw.HW_ESTATE


def test_options_set_get_and_reject(lib):
    ctx = hw.Context(device=-1)
    assert ctx.get_option(hw.HW_OPT_RR_METHOD) == 0
    assert ctx.get_option(hw.HW_OPT_RR_FALLBACKS) == 0
    assert ctx.get_option(hw.HW_OPT_LOWP_SWITCH) == 5
    ctx.set_option(hw.HW_OPT_LOWP_SWITCH, 0)
    assert ctx.get_option(hw.HW_OPT_LOWP_SWITCH) == 0
    ctx.set_option(hw.HW_OPT_RR_METHOD, 1)
    assert ctx.get_option(hw.HW_OPT_RR_METHOD) == 1
    assert ctx.get_option(hw.HW_OPT_EIGENSOLVER) == 0
    assert ctx.get_option(hw.HW_OPT_CHEB_DEGREE) == 24
    assert ctx.get_option(hw.HW_OPT_CHEB_ADAPT) == 1
    assert ctx.get_option(hw.HW_OPT_CHEB_LOCK) == 1
    assert ctx.get_option(hw.HW_OPT_TAIL_NO_P) == 0
    assert ctx.get_option(hw.HW_OPT_WINDOW) == 0
    assert ctx.get_option(hw.HW_OPT_TC_GEMM) == 1
    ctx.set_option(hw.HW_OPT_TC_GEMM, 0)
    assert ctx.get_option(hw.HW_OPT_TC_GEMM) == 0
    assert ctx.get_option(hw.HW_OPT_RADIAL_KERNEL) == 1
    assert ctx.get_option(hw.HW_OPT_SLAB_KERNEL) == 2
    assert ctx.get_option(hw.HW_OPT_FP64_HX) == 1
    assert ctx.get_option(hw.HW_OPT_SMALL_GEMM) == 1
    assert ctx.get_option(hw.HW_OPT_OVERLAP_LAUNCH) == 1
    ctx.set_option(hw.HW_OPT_SLAB_KERNEL, 3)
    assert ctx.get_option(hw.HW_OPT_SLAB_KERNEL) == 3
    ctx.set_option(hw.HW_OPT_WINDOW, 24)
    assert ctx.get_option(hw.HW_OPT_WINDOW) == 24
    ctx.set_option(hw.HW_OPT_EIGENSOLVER, 1)
    ctx.set_option(hw.HW_OPT_CHEB_DEGREE, 9)
    assert (ctx.get_option(hw.HW_OPT_EIGENSOLVER), ctx.get_option(hw.HW_OPT_CHEB_DEGREE)) == (1, 9)
    for opt, val in ((hw.HW_OPT_RR_METHOD, 2), (hw.HW_OPT_RR_FALLBACKS, 0), (hw.HW_OPT_LOWP_SWITCH, 13), (99, 0),
                     (hw.HW_OPT_EIGENSOLVER, 2), (hw.HW_OPT_CHEB_DEGREE, 1), (hw.HW_OPT_CHEB_DEGREE, 65),
                     (hw.HW_OPT_CHEB_ADAPT, 2), (hw.HW_OPT_CHEB_LOCK, 3),
                     (hw.HW_OPT_TAIL_NO_P, 2), (hw.HW_OPT_WINDOW, -1), (hw.HW_OPT_WINDOW, 101),
                     (hw.HW_OPT_TC_GEMM, 3), (hw.HW_OPT_TC_GEMM, -1), (hw.HW_OPT_RADIAL_KERNEL, 2),
                     (hw.HW_OPT_SLAB_KERNEL, 4), (hw.HW_OPT_SLAB_KERNEL, -1), (hw.HW_OPT_FP64_HX, 2),
                     (hw.HW_OPT_SMALL_GEMM, 3), (hw.HW_OPT_OVERLAP_LAUNCH, 2)):
        with pytest.raises(hw.HwError) as e:
            ctx.set_option(opt, val)
        assert e.value.status == hw.HW_EINVAL
    with pytest.raises(hw.HwError):
        ctx.get_option(99)
    ctx.close()


def test_cyclic_masks_and_itable_match_oracle(lib):
    """Ncyc = 3 with nu != 0: masks, compact order and shifted kinetic energies at each (eta, nu),
    and the table I(n, k, k') of eq. I_nkk_prime (the library's Gauss-Jacobi rule against the
    oracle's Gauss-Legendre sum; for n = 0 both take the radial-rule value)."""
    g = inputs.Geometry(**{**inputs.GEOM_TUBE.__dict__, "ncyc": 3})
    etas, nus = np.array([0.1, -0.3, 0.45]), np.array([1.0, 2.0, 0.0])
    ctx = hw.Context(device=-1)
    L = ctx.setup_basis(g, etas, nus)
    b = oracle_basis(g)
    for k, (eta, nu) in enumerate(zip(etas, nus)):
        kp = B.KPoint(b, eta, nu, g.ecut)
        assert L[k] == kp.L
        mnk = ctx.index_map(k)
        np.testing.assert_array_equal(mnk[:, 0], kp.m)
        np.testing.assert_array_equal(mnk[:, 1], kp.n)
        np.testing.assert_array_equal(mnk[:, 2], kp.k)
        np.testing.assert_allclose(ctx.kinetic(k), kp.ke, rtol=1e-13, atol=1e-13)
    for n in range(-b.N, b.N + 1):
        I = b.itable(n)
        np.testing.assert_allclose(ctx.itable(n), I, rtol=0, atol=1e-12 * np.abs(I).max())


def test_binding_constants_match_the_header():
    """Every enumerator of include/helicwave.h (statuses, precisions, preconditioners, options,
    profiler phases) has the same value in the Python binding, and the binding's phase names
    follow the header's HW_PH_ order."""
    hdr = open(os.path.join(ROOT, "include", "helicwave.h")).read()
    enums = dict((k, int(v)) for k, v in re.findall(r"\b(HW_[A-Z0-9_]+)\s*=\s*(\d+)", hdr))
    assert len(enums) > 30
    for name, value in enums.items():
        if name.startswith("HW_PH_") or name == "HW_NPHASE":
            continue
        assert getattr(hw, name) == value, name
    phases = sorted((v, k) for k, v in enums.items() if k.startswith("HW_PH_"))
    assert [k[len("HW_PH_"):].lower() for _, k in phases] == hw.PHASES
    assert len(hw.PHASES) == enums["HW_NPHASE"]
