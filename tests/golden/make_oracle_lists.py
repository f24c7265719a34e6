"""Writes oracle_lists.json: the oracle's per-slot sliding super point lists (hosts, R_k, candidate
counts per level, accepted tuples) for two small seeded workloads, with the RHFG[0] check off and
on. It calls only the oracle and the input generator. The file pins the oracle against itself
across changes: a later change to the oracle's arithmetic must regenerate it and name, in its
commit message, the passage of the paper that justifies the change.

    python tests/golden/make_oracle_lists.py
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import trafficgen as tg  # noqa: E402

CASES = [("tiny", 8), ("paper_c1", 3)]


def compute() -> dict:
    out = {}
    for name, nslots in CASES:
        W = tg.workload(name)
        tabs = tg.hash_tables(W["hash_seed"])
        T = tg.traffic_for(W)
        for label, flags in (("literal", 0), ("verify_h0", oracle.VERIFY_H0)):
            p = oracle.params(W["params"], flags)
            pipe = oracle.Pipeline(p, tabs, T.routers)
            slots = []
            for t in range(nslots):
                r = pipe.step(T.slot(t), "pruned")
                slots.append({"ips": [int(x) for x in r["ips"]], "rk": [int(x) for x in r["rk"]],
                              "levels": [int(x) for x in r["levels"]], "raw": int(r["raw"])})
            out[f"{name}/{label}"] = slots
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_lists.json"), "w") as f:
        json.dump(compute(), f, indent=0, sort_keys=True)
        f.write("\n")
