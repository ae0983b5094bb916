"""Writes graph_hashes.json: the CSR identity (nnz, FNV-1a 64) of the seeded
synthetic graphs, so that a change of the generator, or a machine on which it
rounds differently, is caught.  Calls only the input generator."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from paper_1202_6168_gb300 import graphgen as gg  # noqa: E402

out = {}
for name, spec in [("web_10k_m8", gg.SMALL_10K), ("web_1m_m10", gg.WEB_1M)]:
    rp, col = gg.generate(spec)
    out[name] = {"n": spec.n, "mean_deg": spec.mean_deg, "window": spec.window, "seed": spec.seed,
                 "nnz": int(rp[-1]), "fnv1a64": hex(gg.csr_hash(rp, col))}
out["_about"] = ("CSR identity of the seeded synthetic graphs (generator output, not a value of "
                 "the method); written by tests/golden/make_graph_hashes.py")
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "graph_hashes.json"), "w") as f:
    json.dump(out, f, indent=1)
