"""Input generators: determinism and the level-by-level FP32 variant."""
import numpy as np

from paper_2009_12849_gb300 import workloads as W


def test_f32_generator_matches_full_draw():
    g = W.make_grid(24, 20, 7, 25.0, 25.0, W.geometric_dz(7, 10.0, 60.0))
    for mode in (False, True):
        a = W.random_fields(g, 4, mode)
        b = W.random_fields_f32(g, 4, mode)
        for x, y in zip(a, b):
            assert y.dtype == np.float32
            assert np.array_equal(x.astype(np.float32), y)


def test_boundary_faces_zero_and_profiles():
    g, seed, mode = W.workload_256()
    assert abs(g.dz[0] - 10.0) < 1e-12 and abs(g.dz[-1] - 100.0) < 1e-9
    assert np.all(np.diff(g.rho_f) < 0)
    u, v, w = W.random_fields(W.make_grid(8, 8, 4, 1, 1, W.uniform_dz(4, 1)), 0, True)
    assert np.all(w[0] == 0) and np.all(w[-1] == 0)


def test_serving_and_batch_recipes():
    reqs = W.serving_requests(200)
    assert all(128 <= r["n"] <= 512 and 64 <= r["nz"] <= 192 for r in reqs)
    assert all(W.nearest_smooth(r["n"]) == r["n"] for r in reqs)
    t = [r["t"] for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    inst = W.batch_instances(64)
    assert len(inst) == 64
    assert {g.nx for g, _ in inst} <= {64, 96, 128, 192, 256}


def test_serving_request_objects():
    from paper_2009_12849_gb300 import serve as S
    reqs = S.requests_from_recipe(50, 2000.0, 4)
    assert len(reqs) == 50 and all(r.points == r.n * r.n * r.nz for r in reqs)
    assert S.field_bytes(10, 3) == 4 * 10 * 10 * 10
