"""Write the FP64 oracle's per-dimer {E_J, E_K} for the workloads whose
integral blocks are too large to build on the host (the 10x10x10 lattice,
the uneven batch, the 128-AO lattice), by the oracle's factor route:
(ia|jb) and (ib|ja) from the dimer's three-index factors B^Q, O(n^3 naux)
per dimer, equal to the four-index oracle to 1e-12 relative (pinned in
tests/test_oracle_pins.py).  Calls only synth (inputs) and oracle; the GPU
path never touches these values.

    python tests/golden/make_factor_oracle.py [--first N] [workload ...]

Output: tests/golden/oracle_<workload>.txt, one line per dimer
"d X Y R E_J E_K" (%.17e) and a trailer with the Neumaier lattice totals,
the same format as make_lattice_oracle.py (read by its load()).  With
--first N only dimers 0 .. N-1 are written and the trailer holds no totals
(the 128-AO lattice: its factor route takes ~35 s per dimer on one core).
"""
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

_W = {}


def _init():
    os.environ["OMP_NUM_THREADS"] = "1"


def _one(args):
    name, d = args
    import oracle
    import synth
    w = _W.get(name)
    if w is None:
        w = _W[name] = synth.workload(name)
    X, Y = w.pairs[d]
    mX, mY = w.monomer(X), w.monomer(Y)
    V, W = oracle.factor_route(w.factors(d), synth.scale_for_distance(w.R[d]), mX.C, mY.C, mX.nocc, mY.nocc)
    return d, oracle.energy_from_mo(V, W, mX.eps, mY.eps, mX.nocc, mY.nocc)


def main(names, first=0):
    import oracle
    import synth
    oracle.build()
    for name in names:
        w = synth.workload(name)
        if first:
            w.pairs, w.R = w.pairs[:first], w.R[:first]
        E = np.empty((w.n_dimers, 2))
        t0 = time.time()
        # costliest dimers first so the pool ends evenly
        order = sorted(range(w.n_dimers), key=lambda d: -(w.nao[w.pairs[d][0]] + w.nao[w.pairs[d][1]]))
        with mp.get_context("spawn").Pool(os.cpu_count(), initializer=_init) as pool:
            for k, (d, e) in enumerate(pool.imap_unordered(_one, [(name, d) for d in order], chunksize=8)):
                E[d] = e
                if k % 2000 == 0:
                    print(f"{name}: {k}/{w.n_dimers} dimers, {time.time() - t0:.0f} s", flush=True)
        mon, tot = oracle.accumulate(E, [p[0] for p in w.pairs], [p[1] for p in w.pairs], w.n_monomers)
        path = os.path.join(HERE, f"oracle_{name}.txt")
        what = f"dimers 0 .. {w.n_dimers - 1} of the lattice" if first else "every dimer"
        with open(path, "w") as f:
            f.write(f"# FP64 oracle (oracle/oracle.c, factor route) per-dimer first-order MCPT(2) terms, "
                    f"workload {name}\n")
            f.write(f"# written by tests/golden/make_factor_oracle.py from host-generated synth factors ({what})\n")
            f.write("# d X Y R_angstrom E_J E_K\n")
            for d in range(w.n_dimers):
                X, Y = w.pairs[d]
                f.write(f"{d} {X} {Y} {w.R[d]:.6f} {E[d, 0]:.17e} {E[d, 1]:.17e}\n")
            if not first:
                f.write(f"# total_J {tot[0]:.17e}\n# total_K {tot[1]:.17e}\n")
        print(name, w.n_dimers, tot, f"{time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    argv = sys.argv[1:]
    first = 0
    if argv[:1] == ["--first"]:
        first, argv = int(argv[1]), argv[2:]
    main(argv or ["lattice-10x10x10-cheb2", "uneven-4096", "lattice-7x7x7-cheb1-ao128"], first)
