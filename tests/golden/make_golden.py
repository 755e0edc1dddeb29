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


def gmres_multi_t_helm2d_n32():
    """Iteration counts with per-point neighbourhoods mu_j^{t_j} (Sec. 4.2): t_j from the
    nested-dissection geometry (leaf boxes of width 8, t_max = 2) and, for comparison, t = 2
    at every point."""
    v = make_workload("helm2d_n32")
    out = {}
    for pol in ("local", "paper"):
        for label, kw in (("nd8", {}), ("t2", {"t_of": 2 * O.t_choice(32, 2, 8, 1)})):
            st = O.build_stencils_multi(v, pol, **kw)
            _, it, res, info = O.gmres_solve(v, gaussian_source(32, 2, 2.0), st["P"], st["C"])
            assert info == 0
            out[f"{pol}/{label}"] = it
    return {
        "what": "GMRES(40) inner iterations to rtol 1e-6 (preconditioned residual), x0 = 0, "
                "left preconditioner P^-1 C with per-point t_j, 2D n=32 Helmholtz, sigma = 2 "
                "cells; key = policy/{nd8: t_j from leaf-8 boxes capped at 2, t2: t = 2 "
                "everywhere}",
        "source": "oracle.build_stencils_multi and oracle.gmres_solve (Sec. 4.2, Sec. 5)",
        "iterations": out,
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "gmres_helm2d_n32.json"), "w") as fh:
        json.dump(gmres_helm2d_n32(), fh, indent=1)
        fh.write("\n")
    with open(os.path.join(HERE, "gmres_multi_t_helm2d_n32.json"), "w") as fh:
        json.dump(gmres_multi_t_helm2d_n32(), fh, indent=1)
        fh.write("\n")
    print("written")
