"""Write tests/golden/sigma.json: surface tension of the FP64 reference step
from the Laplace test (Sec. 3): static periodic cylinders of radius 8, 12, 16
(nz = 1), dp = P(rho_in) - P(rho_out) with P from Eq. EOS_SC, R the
equimolar radius, sigma the least-squares slope of dp against 1/R through the
origin.  Calls only the reference implementation under oracle/.

    python tests/golden/make_sigma.py
"""
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lbm_oracle as o  # noqa: E402

CASES = [("shift", -5.5, 1.0), ("guo", -5.5, 1.0)]


def laplace(G, forcing, tau):
    coex = {c["forcing"] + str(c["G"]): c for c in json.load(open(os.path.join(HERE, "coexistence.json")))["cases"]}
    c = coex[forcing + str(G)]
    rl, rv = c["rho_l"], c["rho_v"]
    p = o.Params(G=G, tau=tau, collision="srt" if forcing == "shift" else "mrt")
    pts = []
    for R, L, steps in ((8, 40, 3000), (12, 56, 4000), (16, 72, 6000)):
        yy = np.arange(L)[:, None] - (L - 1) / 2
        xx = np.arange(L)[None, :] - (L - 1) / 2
        r = np.sqrt(xx * xx + yy * yy)
        rho = (rv + 0.5 * (rl - rv) * (1 - np.tanh((r - R) / 2)))[None]
        f = o.run(o.init_populations(rho), steps, p)
        rho = f.sum(0)[0]
        rin, rout = rho[L // 2, L // 2], rho[0, 0]
        dp = o.pressure(rin, G) - o.pressure(rout, G)
        Re = math.sqrt(((rho - rout) / (rin - rout)).sum() / math.pi)
        pts.append((Re, dp))
        print(forcing, G, R, Re, dp, flush=True)
    inv = np.array([1 / R for R, _ in pts])
    dps = np.array([d for _, d in pts])
    sigma = float((inv * dps).sum() / (inv * inv).sum())
    return sigma, pts


def main():
    out = []
    for forcing, G, tau in CASES:
        s, pts = laplace(G, forcing, tau)
        out.append(dict(forcing=forcing, G=G, tau=tau, sigma=round(s, 6),
                        points=[[round(R, 6), round(d, 9)] for R, d in pts]))
    with open(os.path.join(HERE, "sigma.json"), "w") as fh:
        json.dump({"source": "tests/golden/make_sigma.py (FP64 reference, Laplace test on cylinders)",
                   "cases": out}, fh, indent=1)


if __name__ == "__main__":
    main()
