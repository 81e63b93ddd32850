"""Time the CPU oracle (setup, then PCG to 1e-8) on members of the 64^3 checkerboard workload
family and write tests/golden/oracle_scaling.json: per size the DoFs, setup seconds, PCG seconds
and iterations, one core.  The 64^3 row is the full-size run of make_oracle_goldens.py (taken from
hex64_checker.json).  The benchmark's CPU legs extrapolate a small sample to the full workload with
the growth exponents these rows give.  Calls only the oracle and the input generators.

Usage: python tests/golden/make_oracle_scaling.py   (about two minutes)
"""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W          # noqa: E402
from oracle import amg as O    # noqa: E402


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def time_oracle(n):
    p = W.hex_problem(n, W.fields.checkerboard(n, nb=8, hi=1e4, lo=1.0), 1e-2)
    f = W.fields.rhs(p["ndof"], 1)
    t0 = time.perf_counter()
    H = O.setup(p["A"], p["G"])
    t1 = time.perf_counter()
    _, it, _ = O.pcg(H, f, tol=1e-8, maxit=1000)
    t2 = time.perf_counter()
    return dict(n=n, ndof=p["ndof"], setup_s=t1 - t0, pcg_s=t2 - t1, iters=it)


def main():
    rows = [time_oracle(n) for n in (16, 24, 32)]
    full = json.load(open(os.path.join(HERE, "hex64_checker.json")))
    rows.append(dict(n=64, ndof=full["levels"][0]["n"], setup_s=full["oracle_seconds"]["setup"],
                     pcg_s=full["oracle_seconds"]["pcg"], iters=full["pcg"]["iterations"]))
    out = dict(workload_family="hex<n>_checker (alpha on an 8^3 checkerboard {1, 1e4}, beta 1e-2, f seed 1)",
               generator="tests/golden/make_oracle_scaling.py", cores=1, cpu=cpu_model(),
               machine=platform.machine(), rows=rows)
    json.dump(out, open(os.path.join(HERE, "oracle_scaling.json"), "w"), indent=1)
    for r in rows:
        print(r)


if __name__ == "__main__":
    main()
