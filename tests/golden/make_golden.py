"""Writes the stored expected values under tests/golden/ by calling only the CPU oracle.

Run from the repository root:  python tests/golden/make_golden.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from lsp_inputs import gaussian_source, make_workload  # noqa: E402


def gmres_helm2d_n32():
    v = make_workload("helm2d_n32")
    out = {}
    for pol in ("local", "paper", "mean"):
        st = O.build_stencils(v, pol)
        Q, C, P = O.sparse_matrices(st, 32, 2)
        for sig in ("1.0", "2.0", "4.0"):
            _, it, res, info = O.gmres_solve(v, gaussian_source(32, 2, float(sig)), P, C)
            assert info == 0
            out[f"{pol}/{sig}"] = it
    return {
        "what": "GMRES(40) inner iterations to rtol 1e-6 (preconditioned residual), x0 = 0, "
                "left preconditioner P^-1 C, for the 2D n=32 Helmholtz workload "
                "(omega = 2 pi 8, one centred Gaussian bump in c); key = policy/sigma_cells",
        "source": "oracle.gmres_solve (Sec. 4.1 Eq. PC, Sec. 5 solver settings)",
        "iterations": out,
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "gmres_helm2d_n32.json"), "w") as fh:
        json.dump(gmres_helm2d_n32(), fh, indent=1)
        fh.write("\n")
    print("written")
