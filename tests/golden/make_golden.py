"""Write the stored expected values under tests/golden/ from the oracle alone.

Usage: python tests/golden/make_golden.py
Calls only oracle/ (and the seeded input generators); nothing here runs the
CUDA library.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import algebra  # noqa: E402
from pm_inputs import rmat_edges  # noqa: E402


def rmat_s12_motifs():
    s, d = rmat_edges(12, 8, seed=1)
    g = oracle.prepare_graph(4096, s, d)
    out = {"graph": "R-MAT scale 12, edge factor 8, a=.57 b=c=.19, seed 1",
           "n": g.n, "m": g.m, "pattern_order": "algebra.connected_classes(k) masks",
           "masks": {}, "vertex_induced": {}, "edge_induced": {}}
    for k in (3, 4):
        t = time.time()
        masks = algebra.connected_classes(k)
        out["masks"][str(k)] = masks
        out["vertex_induced"][str(k)] = oracle.motif_counts_direct(g, k)
        out["edge_induced"][str(k)] = [
            oracle.count(g, algebra.Pattern.from_mask(k, m)) for m in masks]
        print(f"k={k} done in {time.time() - t:.1f}s", flush=True)
    with open(os.path.join(HERE, "rmat_s12_e8_seed1_motifs.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    rmat_s12_motifs()
