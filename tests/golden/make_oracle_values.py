"""Writes the stored oracle values of tests/golden/oracle_values.json.

Every value here comes from the FP64 CPU oracle (``oracle/``) alone, on a
seeded synthetic workload from ``workloads``; nothing is read from the CUDA
library.  They are stored because the runs are too long for a test: the
steady pored-film conductivity has a per-particle relative standard deviation
of about 10.6, so a comparison whose 3-sigma band is below 1e-3 of kappa needs
more than 1e9 oracle particles (about half an hour on 8 host cores).

Usage:  python tests/golden/make_oracle_values.py [name ...]
(no name: every entry is recomputed)
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import oracle as O  # noqa: E402

OUT = os.path.join(HERE, "oracle_values.json")


def porous_film_kappa():
    """Steady pored film of the porous-film workload (300 nm, pitch 100 nm,
    radius 30 nm, silicon-like, K_s = 40, K_e = 4096), FP64, 1.6e9 particles
    in 16 independent pieces of 1e8 (instance ids 1000 .. 1015 of the counter
    stream, seed distinct from the GPU tests'), so the samples are
    independent of every GPU run."""
    piece, n_pieces = 100_000_000, 16
    base = W.porous_film(n_particles=piece, precision="fp64", seed=0x5EED_0000_0A04)
    s1 = s2 = 0.0
    segs = parts = 0
    t0 = time.time()
    for k in range(n_pieces):
        r = O.run(W.with_run(base, instance_id=1000 + k))
        s1 += r["sum_sL"]
        s2 += r["sum_sL2"]
        segs += r["segments"]
        parts += r["particles"]
        print(f"  piece {k + 1}/{n_pieces}: {time.time() - t0:.0f} s", flush=True)
    # the oracle's own normalisation: kappa is linear in sum s L for a fixed
    # problem, so the combined estimate is the piece kappa scaled by the sums
    n = parts
    mean = s1 / n
    var = (s2 - n * mean * mean) / (n - 1)
    one = O.run(W.with_run(base, n_particles=1_000_000))
    kappa_per_sL = one["kappa"] / (one["sum_sL"] / one["particles"])
    kappa = kappa_per_sL * mean
    kappa_se = abs(kappa_per_sL) * (var / n) ** 0.5
    return {"workload": "porous_film(precision='fp64', seed=0x5EED00000A04), 16 x 1e8 particles, instances 1000-1015",
            "particles": n, "segments": segs, "kappa": kappa, "kappa_se": kappa_se,
            "seconds": time.time() - t0, "threads": os.cpu_count()}


ENTRIES = {"porous_film_kappa": porous_film_kappa}


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names or list(ENTRIES):
        print(name, flush=True)
        data[name] = ENTRIES[name]()
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
            fh.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
