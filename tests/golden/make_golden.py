"""Writes the stored expected eigenvalues under tests/golden/ from the CPU oracle only.

    python tests/golden/make_golden.py

Every value comes from oracle.hamiltonian (dense assembly + numpy.linalg.eigh) on the seeded
workloads of paper_2210_12252_gb300.inputs; nothing here runs the CUDA library.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import basis as B, hamiltonian as Hm, potential as P  # noqa: E402
from paper_2210_12252_gb300 import inputs  # noqa: E402


def basis_of(g):
    return B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)


def write(name, header, values):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        for line in header.strip().splitlines():
            f.write("# " + line + "\n")
        for v in values:
            f.write(f"{v:.17e}\n")
    print("wrote", path)


def main(which):
    if "tiny" in which:
        for zero in (False, True):
            w = inputs.tiny(zero_potential=zero)
            b = basis_of(w.geom)
            V = P.gaussian_wells(b, w.atoms)
            kp = B.KPoint(b, 0.0, 0.0, w.geom.ecut)
            ev = np.linalg.eigvalsh(Hm.dense_H(kp, V))
            tag = "tiny_v0" if zero else "tiny"
            write(f"{tag}_eigs.txt", f"""
workload {w.name} (inputs.tiny(seed=1{', zero_potential=True' if zero else ''})), eta = 0, nu = 0
basis L = {kp.L}; all eigenvalues of the dense Hamiltonian (Algorithm 5 columns), Hartree
source: oracle.hamiltonian.dense_H + numpy.linalg.eigh""", ev)
    if "cyclic" in which:
        w = inputs.tiny_cyclic()
        b = basis_of(w.geom)
        V = P.gaussian_wells(b, w.atoms)
        for i, (eta, nu) in enumerate(zip(w.etas, w.nus)):
            kp = B.KPoint(b, eta, nu, w.geom.ecut)
            ev = np.linalg.eigvalsh(Hm.dense_H(kp, V))
            write(f"tiny_c3_k{i}_eigs.txt", f"""
workload {w.name} (inputs.tiny_cyclic(seed=1, ncyc=3)), k-point {i}: eta = {eta!r}, nu = {nu!r}
basis L = {kp.L}; all eigenvalues of the dense Hamiltonian (Algorithm 5 columns with the I_n
loop; for nu != 0 the n = 0 table is the radial-rule value), Hartree
source: oracle.hamiltonian.dense_H + numpy.linalg.eigh""", ev)
    if "tube_cyclic" in which:
        w = inputs.tube_cyclic()
        b = basis_of(w.geom)
        V = P.gaussian_wells(b, w.atoms)
        for i, (eta, nu) in enumerate(zip(w.etas, w.nus)):
            kp = B.KPoint(b, eta, nu, w.geom.ecut)
            t = time.time()
            ev = np.linalg.eigvalsh(Hm.dense_H_conv(kp, V))[:64]
            print("k-point", i, "L", kp.L, time.time() - t)
            write(f"tube_c3_k{i}_eigs.txt", f"""
workload {w.name} (inputs.tube_cyclic(seed=4, ncyc=3, nk=3)), k-point {i}: eta = {eta!r}, nu = {nu!r}
basis L = {kp.L}; lowest 64 eigenvalues of the dense Hamiltonian, Hartree
source: oracle.hamiltonian.dense_H_conv (convolution form of Algorithm 5 with the I_n loop)
+ numpy.linalg.eigh""", ev)
    if "tube" in which:
        w = inputs.tube()
        b = basis_of(w.geom)
        V = P.gaussian_wells(b, w.atoms)
        kp = B.KPoint(b, 0.0, 0.0, w.geom.ecut)
        t = time.time()
        H = Hm.dense_H_conv(kp, V)
        print("assembled", time.time() - t)
        ev = np.linalg.eigvalsh(H)[:128]
        print("diagonalised", time.time() - t)
        write("tube_eigs.txt", f"""
workload {w.name} (inputs.tube(seed=2)), eta = 0, nu = 0, cutoff 30 Ha
basis L = {kp.L}; lowest 128 eigenvalues of the dense Hamiltonian, Hartree
source: oracle.hamiltonian.dense_H_conv (convolution form of Algorithm 5) + numpy.linalg.eigh""", ev)


    if "tube32" in which:
        # the 32 k-points of the batched workload: lowest 48 eigenvalues per point
        w = inputs.tube_kpoints(nk=32)
        b = basis_of(w.geom)
        V = P.gaussian_wells(b, w.atoms)
        for i, eta in enumerate(w.etas):
            kp = B.KPoint(b, eta, 0.0, w.geom.ecut)
            t = time.time()
            ev = np.linalg.eigvalsh(Hm.dense_H_conv(kp, V))[:w.n_eig]
            print("k-point", i, "L", kp.L, time.time() - t, flush=True)
            write(f"tube32_k{i:02d}_eigs.txt", f"""
workload {w.name} (inputs.tube_kpoints(seed=3, nk=32)), k-point {i}: eta = {eta!r}, nu = 0
basis L = {kp.L}; lowest {w.n_eig} eigenvalues of the dense Hamiltonian, Hartree
source: oracle.hamiltonian.dense_H_conv (convolution form of Algorithm 5) + numpy.linalg.eigh""", ev)
    if "oracle_runs" in which:
        oracle_runs()


def oracle_runs():
    """The oracle's own LOBPCG (literal Algorithm 5 products, TPA preconditioner) run to
    convergence (every wanted residual <= 1e-6) on the tiny and tube workloads from the seeded
    start blocks the benchmark uses; records the oracle's iteration count and, per iteration,
    how many columns were still above the tolerance (each of those costs one H X column in the
    next search direction).  Its wall time here is informational: the benchmark times the
    oracle on the machine it runs on."""
    import json
    import platform
    from oracle import eigensolver as E
    out = {}
    for name, w, seed in (("tiny", inputs.tiny(), 1234), ("tube", inputs.tube(), 1234)):
        b = basis_of(w.geom)
        V = P.gaussian_wells(b, w.atoms)
        kp = B.KPoint(b, 0.0, 0.0, w.geom.ecut)
        nb = w.n_eig + max(4, w.n_eig // 8)
        X0 = inputs.random_block(kp.L, nb, seed)
        active = []   # columns still above tol at each iteration (they get a new direction)
        t = time.time()
        th, X, it, res = E.lobpcg(lambda X: Hm.apply_H(kp, V, X), kp.ke, X0, w.n_eig, tol=1e-6, maxit=500,
                                  callback=lambda i, theta, r: active.append(int((r > 1e-6).sum())))
        dt = time.time() - t
        out[name] = {"workload": w.name, "L": int(kp.L), "n_eig": int(w.n_eig), "block": int(nb),
                     "start_seed": seed, "tol": 1e-6, "iterations": int(it),
                     "active_per_iteration": active,
                     "hx_columns": int(nb + sum(active)),
                     "max_residual": float(np.max(res[: w.n_eig])), "seconds_here": round(dt, 2),
                     "cores_here": len(os.sched_getaffinity(0)), "machine_here": platform.machine()}
        print(name, out[name], flush=True)
    path = os.path.join(HERE, "oracle_lobpcg_runs.json")
    with open(path, "w") as f:
        json.dump({"source": "tests/golden/make_golden.py oracle_runs (oracle.eigensolver.lobpcg with "
                             "oracle.hamiltonian.apply_H, TPA preconditioner)", "runs": out}, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main(sys.argv[1:] or ["tiny", "cyclic", "tube", "tube_cyclic"])
