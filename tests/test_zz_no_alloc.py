"""le_mc_run_noalloc, the entry point for callers that may not allocate GPU
memory (e.g. inside host callbacks or regions owned by another allocator):
it must give the same sums and counters as le_mc_run, call after call, while
its kernel scratch lives in a fixed array inside the library.  Problems above
its size limit are traced in pieces (first_particle), which must add up to
the whole run.

Collected last on purpose: if it fails, a stop-at-first-failure run has
already run every other test.  It also passes alone in a fresh process.
"""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

INTS = ("particles", "segments", "scatters", "wall_hits", "periodic", "truncated", "absorbed")


@pytest.fixture(scope="module")
def P(built_library):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return built_library


def _reference(P, prob):
    return P.simulate(prob, arrays=False)


def test_noalloc_matches_run_twice_in_a_row(P):
    import torch
    dev = torch.device("cuda", 0)
    # the caller owns (and here allocates, ahead of time) the result buffers
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    counters = torch.zeros(7, dtype=torch.int64, device=dev)
    cases = [W.silicon_film(n_particles=300_000, precision="fp32"),
             W.silicon_film(n_particles=100_003, thickness=1e-6, precision="fp32", dTdz=2e5),
             W.gray_slab(n_particles=50_000, n_bins=0, precision="fp64")]
    for prob in cases:
        mat = P.le_mc_create_material(P.material_desc(prob["material"]))
        geo = P.le_mc_create_geometry(P.geometry_desc(prob["geometry"]))
        try:
            ref = _reference(P, prob)
            for _ in range(2):  # two calls in a row reuse the same scratch
                P.le_mc_run_noalloc(mat, geo, P.run_desc(prob["source"], prob["run"]),
                                    sums.data_ptr(), counters.data_ptr(), torch.cuda.current_stream(dev))
                torch.cuda.synchronize(dev)
                s = sums.cpu().tolist()
                c = counters.cpu().tolist()
                for k, v in zip(INTS, c):
                    assert v == ref[k], k
                assert s[0] == pytest.approx(ref["sum_sL"], rel=1e-6, abs=1e-12 * abs(ref["sum_sL2"]) ** 0.5)
                assert s[1] == pytest.approx(ref["sum_sL2"], rel=1e-6)
        finally:
            P.le_mc_destroy_geometry(geo)
            P.le_mc_destroy_material(mat)


def test_noalloc_rejects_oversize_and_arrays(P):
    import torch
    dev = torch.device("cuda", 0)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    counters = torch.zeros(7, dtype=torch.int64, device=dev)
    prob = W.silicon_film(n_particles=P.NOALLOC_MAX_PARTICLES + 1)
    mat = P.le_mc_create_material(P.material_desc(prob["material"]))
    geo = P.le_mc_create_geometry(P.geometry_desc(prob["geometry"]))
    try:
        with pytest.raises(P.LeMcError) as e:
            P.le_mc_run_noalloc(mat, geo, P.run_desc(prob["source"], prob["run"]), sums.data_ptr(),
                                counters.data_ptr())
        assert e.value.status == 1 and "LE_MC_NOALLOC_MAX_PARTICLES" in str(e.value)
        with_hj = W.with_run(prob, n_particles=1000, n_hj=4)
        with pytest.raises(P.LeMcError):
            P.le_mc_run_noalloc(mat, geo, P.run_desc(with_hj["source"], with_hj["run"]), sums.data_ptr(),
                                counters.data_ptr())
    finally:
        P.le_mc_destroy_geometry(geo)
        P.le_mc_destroy_material(mat)


def test_noalloc_pieces_of_a_pored_film_add_up(P):
    """Two pieces (particle ids [0, k) and [k, N)) of a pored film, traced
    through the no-allocation entry point, give le_mc_run's counters over the
    whole range exactly and its sums to summation order; the device flags of
    each piece are readable and clear.  The material is destroyed while the
    second piece may still run: its release must wait for that work."""
    import torch
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    N, k = 600_000, 250_000
    prob = W.porous_film(n_particles=N, precision="fp32")
    ref = _reference(P, prob)
    sums = torch.zeros(2, 2, dtype=torch.float64, device=dev)
    counters = torch.zeros(2, 7, dtype=torch.int64, device=dev)
    mat = P.le_mc_create_material(P.material_desc(prob["material"]))
    geo = P.le_mc_create_geometry(P.geometry_desc(prob["geometry"]))
    try:
        for i, (first, n) in enumerate(((0, k), (k, N - k))):
            piece = W.with_run(prob, n_particles=n, first_particle=first)
            P.le_mc_run_noalloc(mat, geo, P.run_desc(piece["source"], piece["run"]),
                                sums[i].data_ptr(), counters[i].data_ptr(), stream)
            if i == 0:
                assert P.le_mc_noalloc_flags(stream) == 0
    finally:
        P.le_mc_destroy_material(mat)  # the second piece may still be in flight
        P.le_mc_destroy_geometry(geo)
    assert P.le_mc_noalloc_flags(stream) == ref["device_flags"] == 0
    torch.cuda.synchronize(dev)
    c = counters.sum(dim=0).cpu().tolist()
    s = sums.sum(dim=0).cpu().tolist()
    for name, v in zip(INTS, c):
        assert v == ref[name], name
    assert c[0] == N and c[4] > 0  # every particle traced, periodic faces crossed
    # FP32 per-particle lengths are the same bits; only the grouping of the
    # compensated lane sums differs (bound: FP32 rounding of sum |s L|)
    scale = (N * ref["sum_sL2"]) ** 0.5
    assert s[0] == pytest.approx(ref["sum_sL"], rel=1e-6, abs=1e-7 * scale)
    assert s[1] == pytest.approx(ref["sum_sL2"], rel=1e-6)
