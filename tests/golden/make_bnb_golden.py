"""Writes bnb_tiny_oracle.json: the FP64 oracle's Algorithm 1 results on the
seeded 10 x 8 component problems (eps = 1e-3, 128 hypercubes per
iteration).  Calls only the oracle; the GPU tests compare against it."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1812_01232_gb300 import synth  # noqa: E402


def main(seeds=(1000, 1001, 1002)):
    out = {}
    for s in seeds:
        p = synth.tiny_problem(s)
        mix = oracle.Mixtures.from_problem(p)
        r = oracle.bnb(mix, p["t_lo"], p["t_hi"], p["zeta"], p["eps"], pop=128)
        out[str(s)] = {"f": r["f"], "lb": r["lb"], "c22": r["c22"], "r": list(r["r"]), "t": list(r["t"]),
                       "nodes": r["nodes"], "status": r["status"], "eps": p["eps"]}
        print(s, out[str(s)], flush=True)
    with open(os.path.join(HERE, "bnb_tiny_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
