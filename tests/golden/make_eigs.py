"""Writes tests/golden/eigs_<workload>.json with the oracle's lowest
eigenvalues and spectral norm.  Calls only the oracle (explicit CSR H,
Algorithm 1 Lanczos with full reorthogonalisation applied twice; the
extreme eigenvalues from the same Lanczos on H and -H).

Usage: python tests/golden/make_eigs.py [workload ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import basis as ob  # noqa: E402
from oracle import hamiltonian as oh  # noqa: E402
from oracle import lanczos as ol  # noqa: E402

N_KEEP = {"s12_4p4n": 120}


def main(names):
    for name in names:
        t0 = time.time()
        w, sa, sb, inter = synth.workload(name)
        B = ob.ProductBasis(sa.twom, w.nA, sb.twom, w.nB, w.twoM)
        H = oh.assemble(B, inter)
        mv = lambda x: H @ x  # noqa: E731
        v0 = synth.random_block(B.dim, 1, 4242)[:, 0]
        lo, hi = ol.extreme_eigenvalues(mv, B.dim, v0, tol=1e-14, normH_guess=1.0, max_iter=3000)
        normH = max(abs(lo), abs(hi))
        nkeep = N_KEEP.get(name, w.nev)
        th, X, res, it = ol.lanczos(mv, B.dim, nkeep, 1e-12, normH, v0, max_iter=min(B.dim, 6000))
        out = {"workload": name, "dim": B.dim, "normH": normH, "lambda_min": lo, "lambda_max": hi,
               "evals": th.tolist(), "lanczos_iterations": it,
               "max_residual_bound": float(res.max()),
               "how": "oracle Algorithm 1 Lanczos, full reorthogonalisation twice, "
                      "residual bound <= 1e-12 ||H||; ||H|| from Lanczos on H and -H"}
        path = os.path.join(HERE, "eigs_%s.json" % name)
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print(name, "dim", B.dim, "iterations", it, "time %.1fs" % (time.time() - t0))


if __name__ == "__main__":
    main(sys.argv[1:] or ["s12_4p4n"])
