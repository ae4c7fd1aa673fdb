"""Write synth/scales.json: the two-body scale of width-scaled workloads.

Test infrastructure only (see the package docstring).  Calls only the oracle.

For a width-scaled workload the Hamiltonian is H = H1 + s * H2, where H2 is
the two-body part built from unit-variance Gaussian parameters.  Because H2 is
linear in its parameters, s = 50 / (lambda_max(H2) - lambda_min(H2)) makes the
two-body part's spectral width exactly 50.  The extreme eigenvalues come from
the oracle's Algorithm 1 Lanczos on H2 and -H2.

Usage:  python -m oracle.make_scales
"""
from __future__ import annotations

import json
import os

import synth
from . import basis as ob
from . import hamiltonian as oh
from . import lanczos as ol

WIDTH = 50.0


def two_body_width(name: str) -> float:
    w = synth.WORKLOADS[name]
    sp = synth.make_space(w.shells)
    inter = synth.draw_interaction(sp, sp, w.seed, 1.0)
    inter.h1A[:] = 0.0
    inter.h1B[:] = 0.0
    B = ob.ProductBasis(sp.twom, w.nA, sp.twom, w.nB, w.twoM)
    H2 = oh.assemble(B, inter)
    v0 = synth.random_block(B.dim, 1, 12345)[:, 0]
    lo, hi = ol.extreme_eigenvalues(lambda x: H2 @ x, B.dim, v0, tol=1e-13,
                                    normH_guess=1.0, max_iter=2000)
    return hi - lo


def main():
    out = {}
    for name, w in synth.WORKLOADS.items():
        if w.width_scaled:
            width = two_body_width(name)
            out[name] = WIDTH / width
            print(name, "two-body width", width, "scale", out[name])
    path = os.path.join(os.path.dirname(synth.__file__), "scales.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
