"""GPU tests of the request server (continuous batching in one resident
kernel).

A request's epochs depend only on its own statistics, so the particles it
traces, and its result, are the same whether it runs alone or among other
requests: integer counters exactly, FP64 sums up to summation order.  The
resident kernel traces the same particles as le_mc_run for the request.
"""
import numpy as np
import pytest

import workloads as W
from tests.tolerances import sum_order_rtol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P(built_library):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return built_library


def _mix():
    reqs = []
    f = W.silicon_film(n_particles=20_000_000, thickness=100e-9)
    reqs.append((f, 0.01))
    f2 = W.silicon_film(n_particles=20_000_000, thickness=1e-6)
    f2["material"]["T_eq"] = 150.0
    f2["run"]["instance_id"] = 1
    reqs.append((f2, 0.01))
    s = W.gray_slab(n_particles=5_000_000, kn=2.0, n_bins=0, precision="fp32")
    s["run"]["instance_id"] = 2
    reqs.append((s, 0.003))
    p = W.porous_film(n_particles=20_000_000, pitch=150e-9, radius=40e-9)
    p["material"]["T_eq"] = 250.0
    p["run"]["instance_id"] = 3
    reqs.append((p, 0.01))
    small = W.silicon_film(n_particles=70_000, thickness=30e-9)
    small["run"]["instance_id"] = 4
    reqs.append((small, 1e-4))  # budget-limited
    return reqs


INTS = ("particles", "segments", "scatters", "wall_hits", "periodic", "truncated", "absorbed")


def test_results_same_alone_and_in_mix(P):
    reqs = _mix()
    alone = []
    with P.Server(max_slots=4) as srv:
        for prob, target in reqs:
            rid = srv.submit(prob, target)
            srv.wait_all(300)
            alone.append(srv.poll(rid))
    with P.Server(max_slots=4) as srv:
        ids = [srv.submit(prob, target) for prob, target in reqs]
        srv.wait_all(300)
        mixed = [srv.poll(i) for i in ids]
        stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    # the requests were interleaved inside the resident kernel: submitted
    # together, they were all traced by one launch of it
    assert stats["kernel_launches"] == 1, stats
    for (prob, target), a, m in zip(reqs, alone, mixed):
        assert a["state"] == m["state"] == "done"
        for k in INTS:
            assert a[k] == m[k], k
        assert a["epochs"] == m["epochs"]
        key = "psi" if prob["source"]["kind"] == "walls" else "kappa"
        assert m[key] == pytest.approx(a[key], rel=sum_order_rtol(a, prob["run"]["precision"], key))
        assert m["rel_err"] <= target or m["particles"] == prob["run"]["n_particles"]


def test_served_results_match_le_mc_run(P):
    # the resident kernel traces the particles le_mc_run traces for the same
    # request (same ids, random words, frames and rules, FP32 trajectories):
    # over the particles a served request used, the two agree in their
    # counters and estimates up to the rare histories that rounding parts
    reqs = [r for r in _mix()[:4]]
    with P.Server(max_slots=4) as srv:
        ids = [srv.submit(prob, target) for prob, target in reqs]
        srv.wait_all(300)
        served = [srv.poll(i) for i in ids]
    for (prob, target), s in zip(reqs, served):
        n = int(s["particles"])
        g = P.simulate(W.with_run(prob, n_particles=n), arrays=False)
        key = "psi" if prob["source"]["kind"] == "walls" else "kappa"
        for k in ("segments", "scatters", "wall_hits", "periodic"):
            assert abs(s[k] - g[k]) <= 1e-3 * max(g[k], 1), (k, s[k], g[k])
        # (histories parted by rounding are independent samples: with a fraction
        # f of them the difference has a standard deviation of sqrt(2 f) sigma)
        assert abs(s[key] - g[key]) < 1.5 * g[key + "_se"], (key, s[key], g[key], g[key + "_se"])
        assert s["device_flags"] == 0


def test_served_film_matches_pin(P, analytic):
    prob = W.silicon_film(n_particles=50_000_000, thickness=100e-9)
    with P.Server() as srv:
        rid = srv.submit(prob, 0.003)
        srv.wait_all(300)
        r = srv.poll(rid)
    pin = analytic.kappa_film(W.SILICON_LIKE, 100e-9)
    assert r["state"] == "done" and r["rel_err"] <= 0.003
    assert abs(r["kappa"] - pin) < 3.0 * r["kappa_se"]


def test_cancel_and_invalid(P):
    with P.Server(max_slots=2, max_epoch_particles=1 << 16) as srv:
        big = srv.submit(W.silicon_film(n_particles=4_000_000_000 - 1), 1e-9)
        queued = [srv.submit(W.silicon_film(n_particles=3_000_000, thickness=1e-6 * (i + 1)), 1e-9) for i in range(3)]
        srv.cancel(big)
        for q in queued:
            srv.cancel(q)
        srv.wait_all(120)
        assert srv.poll(big)["state"] == "failed"
        assert all(srv.poll(q)["state"] == "failed" for q in queued)
        ok = srv.submit(W.gray_slab(n_particles=100_000, n_bins=0, precision="fp32"), 0.05)
        srv.wait_all(120)
        assert srv.poll(ok)["state"] == "done"
        with pytest.raises(P.LeMcError):
            srv.submit(W.gray_slab(n_particles=100, n_bins=10, precision="fp32"), 0.01)  # arrays are not served
        with pytest.raises(P.LeMcError):
            srv.submit(W.gray_slab(n_particles=100, n_bins=0, precision="fp64"), 0.01)  # FP32 trajectories only
        with pytest.raises(P.LeMcError):
            srv.submit(W.silicon_film(n_particles=100, specularity=0.5), 0.01)  # partially specular walls
        with pytest.raises(P.LeMcError):
            srv.submit(W.gray_slab(n_particles=100, n_bins=0), 0.0)
        with pytest.raises(P.LeMcError):
            srv.poll(10 ** 9)


def test_resident_kernel_relaunch_gives_the_same_results(P):
    # With a 1 ms idle timeout the resident kernel leaves between requests
    # submitted one after another and is launched again for each; the
    # results equal those of a server whose kernel stays up (the particle
    # set of a request does not depend on which launch traces it).
    import time
    reqs = _mix()[:4]
    out = {}
    for idle_ms in (1, 60000):
        res = []
        with P.Server(max_slots=2, idle_exit_ms=idle_ms) as srv:
            for prob, target in reqs:
                rid = srv.submit(prob, target)
                srv.wait_all(300)
                res.append(srv.poll(rid))
                time.sleep(0.05)  # longer than the short idle timeout
            launches = srv.stats()["kernel_launches"]
        out[idle_ms] = (res, launches)
    (short, n_short), (long_, n_long) = out[1], out[60000]
    assert n_long == 1 and n_short >= len(reqs), (n_short, n_long)
    for (prob, target), a, b in zip(reqs, short, long_):
        assert a["state"] == b["state"] == "done"
        for k in INTS:
            assert a[k] == b[k], k
        key = "psi" if prob["source"]["kind"] == "walls" else "kappa"
        assert a[key] == pytest.approx(b[key], rel=sum_order_rtol(b, prob["run"]["precision"], key))


def test_unreachable_target_runs_to_its_budget(P):
    # A target far below what the budget can reach: after the pilot epoch the
    # particles the target asks for exceed what a 64-bit integer holds; the
    # request must still run in epochs to its budget and finish (its epochs
    # are bounded in floating point before any conversion).
    prob = W.silicon_film(n_particles=300_000, thickness=100e-9)
    with P.Server(max_slots=2) as srv:
        rid = srv.submit(prob, 1e-12)
        try:
            srv.wait_all(120)
        except P.LeMcError:
            srv.cancel(rid)  # (so that closing the server does not wait on it)
            raise
        r = srv.poll(rid)
    assert r["state"] == "done" and r["particles"] == 300_000, r
    assert r["rel_err"] > 1e-12 and r["epochs"] >= 2
