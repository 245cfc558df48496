"""Failure handling on the GPU without a GPU fault.

Device allocations are made to fail through the library's test hook
(``le_mc_test_fail_allocation``): the call that needed the memory reports
LE_MC_ERR_NOMEM and releases what it had allocated, and the library stays
usable: the next call succeeds and gives the result it gives without the
failure.  In the request server the request that met the failure ends FAILED
while the next one completes.
"""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

NOMEM = 2


@pytest.fixture(scope="module")
def P(built_library):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    yield built_library
    built_library.le_mc_test_fail_allocation(-1)


def test_material_allocation_failure(P):
    desc = P.material_desc(W.SILICON_LIKE)
    for after in range(5):  # each of the material's five device tables in turn
        P.le_mc_test_fail_allocation(after)
        with pytest.raises(P.LeMcError) as e:
            P.le_mc_create_material(desc)
        assert e.value.status == NOMEM, after
    m = P.le_mc_create_material(desc)  # the hook disarmed itself when it fired
    P.le_mc_destroy_material(m)


def test_run_allocation_failure_then_same_result(P):
    prob = W.silicon_film(n_particles=200_000)
    ref = P.simulate(prob, arrays=False)
    mat = P.le_mc_create_material(P.material_desc(prob["material"]))
    geo = P.le_mc_create_geometry(P.geometry_desc(prob["geometry"]))
    try:
        P.le_mc_test_fail_allocation(0)
        with pytest.raises(P.LeMcError) as e:
            P.le_mc_run(mat, geo, P.run_desc(prob["source"], prob["run"]), None)
        assert e.value.status == NOMEM
        h = P.le_mc_run(mat, geo, P.run_desc(prob["source"], prob["run"]), None)
        t = P.le_mc_read_tallies(h)
        P.le_mc_destroy_run(h)
        for k in ("particles", "segments", "scatters", "wall_hits"):
            assert t[k] == ref[k]
        assert t["device_flags"] == 0
    finally:
        P.le_mc_destroy_geometry(geo)
        P.le_mc_destroy_material(mat)


def test_batch_allocation_failure(P):
    probs = W.batched_films(n_instances=8, n_max=1e5)
    P.le_mc_test_fail_allocation(5)  # after the shared material's five tables: the batch's own memory
    with pytest.raises(P.LeMcError) as e:
        P.Batch(probs)
    assert e.value.status == NOMEM
    with P.Batch(probs) as bt:
        bt.launch(None)
        res = bt.results()
    assert [r["particles"] for r in res] == [p["run"]["n_particles"] for p in probs]


def test_server_request_allocation_failure(P):
    with P.Server(max_slots=2) as srv:
        P.le_mc_test_fail_allocation(0)  # the first request's material
        bad = srv.submit(W.silicon_film(n_particles=200_000), 0.05)
        srv.wait_all(120)
        good = srv.submit(W.silicon_film(n_particles=200_000), 0.05)
        srv.wait_all(120)
        assert srv.poll(bad)["state"] == "failed"
        r = srv.poll(good)
        assert r["state"] == "done" and r["particles"] > 0
        assert srv.stats()["failed"] == 1
