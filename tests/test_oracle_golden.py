"""The oracle reproduces its stored regression values (written by
tests/golden/make_golden.py, which calls only the oracle)."""
import hashlib
import json
import os

import oracle
from workloads import WORKLOADS


def test_golden_adsdes64():
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_adsdes64.json")
    gold = json.load(open(path))
    w = WORKLOADS["adsdes64"]
    for bJ, g in gold.items():
        init = oracle.init_bernoulli(w["lx"], w["ly"], w["seed"], w["coverage"])
        assert hashlib.sha256(init.tobytes()).hexdigest() == g["init_sha256"]
        run = oracle.FSRun(w["lx"], w["ly"], *w["q"], w["model"],
                           dict(w["rates"], betaJ=float(bJ)), init)
        run.run(w["scheme"], w["dt"], w["T"], w["seed"])
        assert run.events == g["events"] and run.windows == g["windows"]
        assert hashlib.sha256(run.lat.tobytes()).hexdigest() == g["final_sha256"]
