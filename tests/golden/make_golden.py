"""Writes golden eigenvalues of a full-size workload with the FP64 oracle.

Calls only oracle/ and synthgraphs/ (never the GPU library).  Usage:
    python tests/golden/make_golden.py <workload> <eps> <out.json> [d]
<eps> is either a number or "rel:<x>" (absolute tolerance x * 2 * max degree, the relative
residual bound of the benchmark), or "abs:<x>" (the paper's absolute epsilon itself).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthgraphs as sg  # noqa: E402


def parse_eps(spec: str, normL: float) -> tuple[float, float]:
    """(absolute epsilon, relative value recorded as eps_rel) from the command-line spec."""
    if spec.startswith("abs:"):
        e = float(spec[4:])
        return e, e / normL
    rel = float(spec[4:]) if spec.startswith("rel:") else float(spec)
    return rel * normL, rel


def main():
    name, spec, out = sys.argv[1], sys.argv[2], sys.argv[3]
    d = int(sys.argv[4]) if len(sys.argv) > 4 else 10
    g = sg.workload(name)
    normL = 2.0 * float(g.degrees.max())
    eps, eps_rel = parse_eps(spec, normL)
    u0 = sg.start_vector(g.n, 1)
    t0 = time.time()
    lam, V, st = oracle.isira(g.row_ptr, g.col_idx, d, u0, eps=eps, tau_inner=1e-3)
    dt = time.time() - t0
    res = [float(np.linalg.norm(oracle.laplacian_apply(g.row_ptr, g.col_idx, V[:, j]) - lam[j] * V[:, j]) / normL)
           for j in range(d)]
    order = np.argsort(lam)
    json.dump({"workload": name, "n": g.n, "nnz": g.nnz, "d": d, "eps_rel": eps_rel, "eps_abs": eps,
               "norm_L": normL, "eigvals": [float(lam[i]) for i in order], "true_resid_rel": [res[i] for i in order],
               "oracle_stats": {k: (int(v) if isinstance(v, (int, np.integer)) else float(v)) for k, v in st.items()},
               "oracle_seconds": dt, "generator": "tests/golden/make_golden.py (oracle, FP64, 1 thread)"},
              open(out, "w"), indent=1)


if __name__ == "__main__":
    main()
