"""Throughput of the CPU oracle (test infrastructure, not the product) on the
seeded workloads of the slab, film, pored-film and surface-pulse problems,
single-threaded and on every core, in segments per second.

    python oracle/time_oracle.py

The oracle is deliberately plain (one particle at a time, FP64, inverse-CDF
mode draws); these figures describe it as it stands, for comparison with the
GPU tracer, and are not a tuned CPU implementation.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

CASES = [
    ("gray slab, Kn 1, black walls, 50 bins", W.gray_slab(n_particles=2_000_000, n_bins=50)),
    ("silicon-like film 100 nm", W.silicon_film(n_particles=1_000_000, precision="fp64")),
    ("pored film, steady", W.porous_film(n_particles=400_000, precision="fp64")),
    ("pored film, surface pulse", W.porous_pulse(n_particles=20_000, precision="fp64")),
]


def main():
    ncpu = os.cpu_count() or 1
    O.build()
    print(f"| workload | threads | segments/s | sample |\n|---|---|---|---|")
    for name, prob in CASES:
        for threads in (1, ncpu):
            t0 = time.perf_counter()
            r = O.run(prob, n_threads=threads)
            dt = time.perf_counter() - t0
            n = prob["run"]["n_particles"]
            print(f"| {name} | {threads} | {r['segments'] / dt:.3e} | {n} particles, {r['segments']} segments, {dt:.2f} s |",
                  flush=True)


if __name__ == "__main__":
    main()
