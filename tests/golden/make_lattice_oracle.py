"""Write the FP64 oracle's per-dimer {E_J, E_K} for the 32-AO lattice
workloads, from host-generated inputs.  Calls only synth (inputs) and
oracle; the GPU path never touches these values.

    python tests/golden/make_lattice_oracle.py [workload ...]

Output: tests/golden/oracle_<workload>.txt, one line per dimer
"d X Y R E_J E_K" (%.17e) and a trailer with the Neumaier lattice totals.
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def _one(args):
    name, d = args
    import oracle
    import synth
    w = synth.workload(name)
    X, Y = w.pairs[d]
    mX, mY = w.monomer(X), w.monomer(Y)
    A, K = w.blocks(d)
    return d, oracle.dimer(A, K, mX.C, mX.eps, mY.C, mY.eps, mX.nocc, mY.nocc)


def main(names):
    import oracle
    import synth
    for name in names:
        w = synth.workload(name)
        E = np.empty((w.n_dimers, 2))
        with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
            for d, e in pool.imap_unordered(_one, [(name, d) for d in range(w.n_dimers)], chunksize=4):
                E[d] = e
        mon, tot = oracle.accumulate(E, [p[0] for p in w.pairs], [p[1] for p in w.pairs], w.n_monomers)
        path = os.path.join(HERE, f"oracle_{name}.txt")
        with open(path, "w") as f:
            f.write(f"# FP64 oracle (oracle/oracle.c) per-dimer first-order MCPT(2) terms, workload {name}\n")
            f.write("# written by tests/golden/make_lattice_oracle.py from host-generated synth inputs\n")
            f.write("# d X Y R_angstrom E_J E_K\n")
            for d in range(w.n_dimers):
                X, Y = w.pairs[d]
                f.write(f"{d} {X} {Y} {w.R[d]:.6f} {E[d, 0]:.17e} {E[d, 1]:.17e}\n")
            f.write(f"# total_J {tot[0]:.17e}\n# total_K {tot[1]:.17e}\n")
        print(name, w.n_dimers, tot)


def load(name):
    """(E [D,2], total [2]) from tests/golden/oracle_<name>.txt, or None."""
    path = os.path.join(HERE, f"oracle_{name}.txt")
    if not os.path.exists(path):
        return None
    rows, tot = [], [None, None]
    with open(path) as f:
        for line in f:
            if line.startswith("# total_J"):
                tot[0] = float(line.split()[2])
            elif line.startswith("# total_K"):
                tot[1] = float(line.split()[2])
            elif not line.startswith("#"):
                p = line.split()
                rows.append((float(p[4]), float(p[5])))
    return np.array(rows), np.array(tot)


if __name__ == "__main__":
    main(sys.argv[1:] or ["lattice-2x2x2", "lattice-5x5x5-cheb1"])
