"""Write tests/golden/oracle_adsdes64.json from the oracle alone.

Regression values for the 64x64 adsorption/desorption workload (Lie,
dt = 0.1, T = 10, 8x8 cells; Section 4.1's example) at betaJ = 0 and 1:
event count, window count and a digest of the final lattice. Run:
    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import WORKLOADS  # noqa: E402


def main():
    w = WORKLOADS["adsdes64"]
    out = {}
    for bJ in (0.0, 1.0):
        init = oracle.init_bernoulli(w["lx"], w["ly"], w["seed"], w["coverage"])
        run = oracle.FSRun(w["lx"], w["ly"], *w["q"], w["model"],
                           dict(w["rates"], betaJ=bJ), init)
        run.run(w["scheme"], w["dt"], w["T"], w["seed"])
        out[str(bJ)] = dict(events=run.events, windows=run.windows, ambiguous=run.ambiguous,
                            init_sha256=hashlib.sha256(init.tobytes()).hexdigest(),
                            final_sha256=hashlib.sha256(run.lat.tobytes()).hexdigest(),
                            coverage=float(run.lat.mean()))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_adsdes64.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
