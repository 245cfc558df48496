"""The checking build (-DLEMC_DEBUG) of the library on the GPU.

Every data-dependent index of the trace kernels (emission-buffer slots,
modes, queue positions, transient cells, record slots) is range-checked
there, and one out of range sets LE_MC_FLAG_DEBUG_BOUNDS in the run's device
flags instead of being trusted.  The workloads of every kernel family run
under it with no flag set, and FP64 runs trace the same histories as the
release build (the checks change no arithmetic).
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the same cases in this process (release build) and in the child (debug build)
CASES = r'''
import workloads as W
GRAY = dict(W.GRAY_UNIT, tau=2e-8, v=1.0)
CASES = {
    "film_fp32": (W.silicon_film(n_particles=1_000_000), {}),
    "film_fp64": (W.silicon_film(n_particles=100_000, precision="fp64"), {}),
    "slab_profile_fp64": (W.gray_slab(n_particles=100_000, n_bins=50), {"record_particles": True}),
    "slab_fp32": (W.gray_slab(n_particles=1_000_000, n_bins=0, precision="fp32"), {}),
    "porous_maps_fp32": (W.porous_film(n_particles=500_000, map=(8, 8)), {}),
    "porous_gray_fp64": (W.porous_film(n_particles=20_000, precision="fp64", material=GRAY, max_events=300,
                                       max_scatter=20), {"record_particles": True}),
    "pulse_fp32": (W.porous_pulse(n_particles=200_000, grid=(8, 16, 16), n_samples=40), {}),
    "initial_fp32": (W.porous_initial(n_particles=200_000), {}),
    "ttr_fp64": (W.ttr_film(n_particles=20_000, precision="fp64", n_samples=20), {}),
    "film_partial_aniso_hj_fp32": (W.silicon_film(n_particles=300_000, specularity=0.5,
                                                  material=dict(W.SILICON_LIKE, scatter_g=0.4), n_hj=8), {}),
    "porous_first_event_fp32": (W.with_run(W.porous_film(n_particles=300_000), max_events=1), {}),
    "porous_first_path_fp64": (W.with_run(W.porous_film(n_particles=20_000, precision="fp64"), max_collisions=1),
                               {"record_particles": True}),
    "film_piece_fp32": (W.with_run(W.silicon_film(n_particles=70_001), first_particle=123_457), {}),
    "film_tiny_fp32": (W.silicon_film(n_particles=33), {"record_particles": True}),
    "slab_one_fp64": (W.gray_slab(n_particles=1, n_bins=4), {}),
}
'''

CHILD = r'''
import json, sys
sys.path.insert(0, ROOT)
import paper_1206_3316_gb300 as P
assert P.LIB_PATH.endswith("libLeMC_debug.so"), P.LIB_PATH
exec(CASES)
out = {}
for name, (prob, kw) in CASES.items():
    r = P.simulate(prob, **kw)
    out[name] = {"flags": int(r["device_flags"]), "segments": int(r["segments"]), "particles": int(r["particles"])}
probs = W.batched_films(n_instances=16, n_max=1e5)
with P.Batch(probs) as bt:
    bt.launch(None)
    res = bt.results()
out["batch"] = {"flags": max(int(r["device_flags"]) for r in res), "segments": sum(int(r["segments"]) for r in res),
                "particles": sum(int(r["particles"]) for r in res)}
print(json.dumps(out))
'''


@pytest.fixture(scope="module")
def P(built_library):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return built_library


def test_debug_build_sets_no_bounds_flag(P):
    import __graft_entry__
    lib = __graft_entry__._build_module().build(debug=True)
    env = dict(os.environ, LE_MC_LIBRARY=lib)
    code = f"ROOT = {ROOT!r}\nCASES = {CASES!r}\n" + CHILD
    res = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-2000:]
    got = json.loads(res.stdout.strip().splitlines()[-1])
    ns = {}
    exec(CASES, ns)
    for name, (prob, kw) in ns["CASES"].items():
        g = got[name]
        assert g["flags"] == 0, (name, g)
        assert g["particles"] == prob["run"]["n_particles"], name
        if prob["run"].get("precision") == "fp64":
            ref = P.simulate(prob, arrays=False)
            assert g["segments"] == ref["segments"], name
    assert got["batch"]["flags"] == 0
