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


if __name__ == "__main__":
    main(sys.argv[1:] or ["tiny", "cyclic", "tube", "tube_cyclic"])
