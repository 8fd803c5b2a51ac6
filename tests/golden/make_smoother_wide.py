"""Write the stored oracle values of the smoother parity test at the widest
subdomain, m = 35 (P = 32 with N_O = 1 node layer: the fine level of the
4^3, P = 32 high-order configuration).

The oracle solves each subdomain problem A_ss du_s = R_s r directly (Section
3.1, Eq. subproblem) with A_ss extracted from the 3D-assembled SIPG matrix.
At m = 35 that is a dense SPD matrix of 42,875^2 values (14.7 GB) whose
Cholesky factorisation takes minutes, too slow and too large for a test run,
so this script computes one smoothing step once and stores a seeded sample of
its output.  It calls only ``oracle/`` and the seeded input generators.

Case: periodic box 1.0 x 1.5 x 0.7 (three different element widths), 3^3
elements, P = 32 (970,299 DOFs), N_O = 1, quintic weights; u and f are
N(0, 1) draws (seeds 40, 41) rounded to FP32 so that the FP32 kernels see the
same inputs.  Stored: the correction sum_s R_s^T W_s A_ss^{-1} R_s (f - A u)
at 2048 seeded sample indices, and its max-norm and 2-norm.

    python tests/golden/make_smoother_wide.py      # ~30 GB of host memory, about 15 minutes
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle.schwarz import SchwarzSmoother, layer_delta  # noqa: E402
from oracle.sipg import Mesh, assemble  # noqa: E402
from paper_1612_04796_gb300 import inputs  # noqa: E402

CASE = {"lengths": [1.0, 1.5, 0.7], "elements": [3, 3, 3], "P": 32, "overlap_layers": 1, "profile": "quintic",
        "seed_u": 40, "seed_f": 41, "seed_sample": 42, "samples": 2048}
OUT = os.path.join(HERE, "smoother_p32_m35.json")


def main():
    t0 = time.time()
    mesh = Mesh(CASE["lengths"], CASE["elements"])
    P, n_o = CASE["P"], CASE["overlap_layers"]
    A = assemble(mesh, P)
    N = A.shape[0]
    u = inputs.gaussian(N, CASE["seed_u"]).astype(np.float32).astype(np.float64)
    f = inputs.gaussian(N, CASE["seed_f"]).astype(np.float32).astype(np.float64)
    r = f - A @ u
    sm = SchwarzSmoother(A, mesh, P, n_o, layer_delta(P, n_o), CASE["profile"], check=4, dense_limit=50000)
    corr = sm.correction(r)
    idx = np.sort(np.random.default_rng(CASE["seed_sample"]).choice(N, CASE["samples"], replace=False))
    rec = {
        "citation": "Stiller, arXiv 1612.04796, Section 3.1 (weighted additive Schwarz step with the direct "
                    "subdomain inverse A_ss^{-1}, Eq. subproblem and Eq. correction:global)",
        "written_by": "tests/golden/make_smoother_wide.py (oracle only)",
        "case": CASE, "dofs": int(N), "subdomain_width": int(round(sm.m3 ** (1 / 3))),
        "correction_max_abs": float(np.max(np.abs(corr))), "correction_norm2": float(np.linalg.norm(corr)),
        "index": [int(i) for i in idx], "value": [float(v) for v in corr[idx]],
    }
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=0)
        fh.write("\n")
    print("wrote %s (%d DOFs, m = %d) in %.0f s" % (OUT, N, rec["subdomain_width"], time.time() - t0))


if __name__ == "__main__":
    main()
