"""Write tests/golden/coexistence.json: flat-interface coexistence densities
of the FP64 reference step (steady state of a periodic liquid slab, fields
varying along z only, 64 cells), for the forcing/G/tau combinations that the
ligament inputs use.  Calls only the reference implementation under oracle/.

    python tests/golden/make_coexistence.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lbm_oracle as o  # noqa: E402

CASES = [("shift", -5.5, 1.0, 2.3068, 0.1041), ("guo", -5.5, 1.0, 2.2486, 0.0569),
         ("shift", -5.3, 1.0, 2.1617, 0.1214), ("guo", -5.3, 1.0, 2.1089, 0.0781)]


def steady_slab(G, coll, tau, rl, rv, n=64):
    z = np.arange(n) + 0.5
    d = np.abs(z - n / 2) - n / 4
    rho = (rv + 0.5 * (rl - rv) * (1 - np.tanh(d / 2.0)))[:, None, None]
    p = o.Params(G=G, tau=tau, collision=coll)
    f = o.init_populations(rho)
    prev = None
    for _ in range(200):
        f = o.run(f, 500, p)
        r = f.sum(0)[:, 0, 0]
        cur = (float(r[n // 2]), float(r[0]))
        if prev and max(abs(cur[0] - prev[0]), abs(cur[1] - prev[1])) < 1e-12:
            return cur
        prev = cur
    raise RuntimeError("no steady state")


def main():
    out = []
    for forcing, G, tau, rl, rv in CASES:
        coll = "srt" if forcing == "shift" else "mrt"
        l, v = steady_slab(G, coll, tau, rl, rv)
        out.append(dict(forcing=forcing, G=G, tau=tau, rho_l=round(l, 6), rho_v=round(v, 6)))
        print(out[-1], flush=True)
    with open(os.path.join(HERE, "coexistence.json"), "w") as fh:
        json.dump({"source": "tests/golden/make_coexistence.py (FP64 reference, 64-cell slab)",
                   "cases": out}, fh, indent=1)


if __name__ == "__main__":
    main()
