"""GPU tests of batches: many instances in one persistent launch.

Each instance keeps its own particle stream (seed, instance id, particle id),
so its tallies in the batch must equal those of the same instance run alone:
integer counters exactly, FP64 sums up to summation order.
"""
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(built_library):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return built_library


def _films(n, precision, seed=7):
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(n):
        L = float(np.exp(rng.uniform(np.log(10e-9), np.log(10e-6))))
        N = int(np.exp(rng.uniform(np.log(1), np.log(60_000))))
        if i == 3:
            N = 0
        if i == 5:
            N = 33
        p = W.silicon_film(n_particles=N, thickness=L, precision=precision, dTdz=(-1e6 if i % 3 else 2e5))
        p["run"]["instance_id"] = 100 + i
        probs.append(p)
    return probs


INTS = ("particles", "segments", "scatters", "wall_hits", "periodic", "truncated", "absorbed")


@pytest.mark.parametrize("precision,rtol", [("fp32", 1e-6), ("fp64", 1e-11)])
def test_batch_equals_single_runs(P, precision, rtol):
    probs = _films(24, precision)
    with P.Batch(probs) as b:
        b.launch()
        got = b.results()
    for p, g in zip(probs, got):
        alone = P.simulate(p, arrays=False)
        for k in INTS:
            assert g[k] == alone[k], (k, p["run"]["n_particles"])
        if p["run"]["n_particles"] > 1:
            assert g["kappa"] == pytest.approx(alone["kappa"], rel=rtol, abs=1e-12 * abs(alone["kappa_se"]) + 1e-300)
            assert g["kappa_se"] == pytest.approx(alone["kappa_se"], rel=1e-6)
        assert g["device_flags"] == 0


def test_batch_slabs_equal_single_runs(P):
    probs = []
    for i, kn in enumerate((0.3, 1.0, 3.0, 10.0)):
        p = W.gray_slab(n_particles=20_000 + 999 * i, n_bins=0, precision="fp64")
        p["geometry"]["L"] = 1.0 / kn  # one material (Lambda = 1), thickness sets Kn
        p["run"]["instance_id"] = i
        probs.append(p)
    with P.Batch(probs) as b:
        b.launch()
        got = b.results()
    for p, g in zip(probs, got):
        alone = P.simulate(p, arrays=False)
        for k in INTS:
            assert g[k] == alone[k]
        assert g["psi"] == pytest.approx(alone["psi"], rel=1e-12)


def test_graph_replay_and_launch_shapes_agree(P):
    probs = _films(16, "fp32", seed=11)
    results = []
    with P.Batch(probs) as b:
        for cfg in ({"use_graph": False}, {"use_graph": True},
                    {"use_graph": True, "threads_per_block": 128, "refill_min": 4, "chunk": 256}):
            b.set_config(cfg)
            for _ in range(2):  # the second launch replays the captured graph
                b.launch()
                results.append(b.results())
    ref = results[0]
    for res in results[1:]:
        for a, c in zip(ref, res):
            for k in INTS:
                assert a[k] == c[k]
            assert a["kappa"] == pytest.approx(c["kappa"], rel=1e-6, abs=1e-9)


def test_autotune_and_cache(P, tmp_path):
    probs = _films(8, "fp32", seed=3)
    cache = str(tmp_path / "tune.txt")
    with P.Batch(probs) as b:
        best = b.autotune(cache_path=cache)
        assert best["threads_per_block"] in (128, 256, 512) and best["ms"] > 0
        assert os.path.exists(cache)
        again = b.autotune(cache_path=cache)  # served from the cache
        assert {k: again[k] for k in ("threads_per_block", "refill_min", "chunk")} == \
               {k: best[k] for k in ("threads_per_block", "refill_min", "chunk")}
        b.launch()
        assert sum(r["particles"] for r in b.results()) == sum(p["run"]["n_particles"] for p in probs)
    assert len(open(cache).read().strip().splitlines()) == 1


def test_batch_rejects_mixed_families(P):
    a = W.silicon_film(n_particles=10)
    b = W.silicon_film(n_particles=10, seed=99)
    with pytest.raises(P.LeMcError):
        P.Batch([a, b])
    c = W.silicon_film(n_particles=10, n_hj=4)
    with pytest.raises(P.LeMcError):
        P.Batch([c])
    d = W.porous_film(n_particles=10)
    with pytest.raises(P.LeMcError):
        P.Batch([d])


def test_batched_films_each_instance_against_its_pin(P, oracle, analytic):
    # config 3: 256 films of uneven thickness and size in one launch; every
    # instance matches the Fuchs-Sondheimer value for its thickness, and the
    # small instances match the FP64 oracle
    probs = W.batched_films(256)
    with P.Batch(probs) as b:
        b.launch()
        got = b.results()
    from scipy import stats
    zs = []
    for p, g in zip(probs, got):
        pin = analytic.kappa_film(W.SILICON_LIKE, p["geometry"]["L"])
        zs.append((g["kappa"] - pin) / g["kappa_se"])
        assert g["particles"] == p["run"]["n_particles"] and g["device_flags"] == 0
    zs = np.array(zs)
    # the 256 instances are independent: sum z^2 is chi-square with 256
    # degrees of freedom under the pins
    p_all = stats.chi2.sf(np.sum(zs ** 2), zs.size)
    print(f"\n256 batched films against Fuchs-Sondheimer: sum z^2 = {np.sum(zs ** 2):.1f}, p = {p_all:.3g}, "
          f"max |z| = {np.abs(zs).max():.2f}")
    assert p_all > 1e-3
    small = [i for i, p in enumerate(probs) if p["run"]["n_particles"] <= 100_000][:24]
    for i in small:
        o = oracle.run(W.with_run(probs[i], precision="fp64"))
        z = abs(got[i]["kappa"] - o["kappa"]) / np.hypot(got[i]["kappa_se"], o["kappa_se"])
        assert z < 4.5, (i, z)
