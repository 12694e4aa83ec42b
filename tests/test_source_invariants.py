"""Source-level invariants of the CUDA library that no GPU run would catch reliably.

Kernels are launched with programmatic stream serialisation (launch_dep, launch_dep_c,
launch_ex): such a kernel may start while the kernel before it in the stream still runs, so it
must wait (griddep_entry or griddep_wait) before it touches that kernel's data.  A kernel that
forgot the wait would race only sometimes.  This test reads the sources: every kernel defined in
csrc/ waits, except the cooperative kernels, which are launched without the attribute.
"""
import glob
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2210_12252_gb300", "csrc")
COOPERATIVE = {"k_jacobi", "k_barrier_selftest"}


def kernel_definitions():
    out = []
    for path in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        src = open(path).read()
        for m in re.finditer(r"__global__[^;{]*?\b(k_\w+)\s*\(", src, flags=re.S):
            brace = src.index("{", m.end())
            if ";" in src[m.end():brace]:
                continue   # a declaration
            depth, i = 0, brace
            while True:   # the body, by brace matching
                if src[i] == "{":
                    depth += 1
                elif src[i] == "}":
                    depth -= 1
                    if depth == 0:
                        break
                i += 1
            out.append((os.path.basename(path), m.group(1), src[brace:i + 1]))
    return out


def test_every_overlapped_kernel_waits_for_its_predecessor():
    kernels = kernel_definitions()
    assert len(kernels) > 50
    missing = [(f, k) for f, k, body in kernels
               if k not in COOPERATIVE and "griddep_entry()" not in body and "griddep_wait()" not in body]
    assert not missing, missing


def test_cooperative_kernels_launch_without_the_attribute():
    srcs = "".join(open(p).read() for p in glob.glob(os.path.join(CSRC, "*.cu")))
    for k in COOPERATIVE:
        assert re.search(r"cudaLaunchCooperativeKernel\(\(void\*\)" + k + r"\b", srcs), k
        assert not re.search(r"launch_dep(_c)?\([^;]*\b" + k + r"\b", srcs), k


def test_no_plain_triple_chevron_launches():
    """Every launch goes through the overlapped launchers, a cooperative launch, or (the gradient
    kernel, measured slower overlapped) cudaLaunchKernel."""
    for path in glob.glob(os.path.join(CSRC, "*.cu")):
        assert "<<<" not in open(path).read(), os.path.basename(path)


def test_entry_comes_first_where_it_is_used():
    """griddep_entry() is the kernel's first statement: nothing is read or written before it."""
    for f, k, body in kernel_definitions():
        if "griddep_entry()" in body:
            first = body[1:].strip().split(";")[0].strip()
            assert first == "griddep_entry()", (f, k, first)
