"""Autotuner of the RAS smoother (tile shape, k, overlap) by time to
E_v <= 1e-8: bucketing and the JSON cache on the CPU; one small tuning run
through the library on the GPU."""
import math

import numpy as np
import pytest

from paper_2509_19061_gb300 import autotune, inputs


def test_buckets():
    assert autotune.bucket(1024, 1024, 1e6, "f64") == "n10_f64_c6"
    assert autotune.bucket(64, 64, 1e2, "f32") == "n6_f32_c2"
    assert autotune.bucket(8192, 8192, 0.5, "f32") == "n13_f32_c0"
    # log2(sqrt(nx ny)) for non-square grids
    assert autotune.bucket(2048, 512, 10.0, "f64") == "n10_f64_c1"
    ec, en = np.full((4, 4), 2.0), np.full((5, 5), 3.0)
    en[1, 1] = 3000.0
    assert math.isclose(autotune.contrast_of(ec, en), 1500.0)


def test_cache_round_trip_and_nearest_lookup(tmp_path):
    path = str(tmp_path / "tune.json")
    c = autotune.Cache(path)
    assert c.lookup(512, 512, 1e4, "f64") == autotune.DEFAULT
    c.record(512, 512, 1e4, "f64", autotune.Choice(16, 16, 2, 1, 0.5, 30))
    c.record(4096, 4096, 1e4, "f64", autotune.Choice(32, 32, 8, 7, 2.0, 40))
    c.save()
    d = autotune.Cache(path)
    assert d.lookup(512, 512, 1e4, "f64") == autotune.Choice(16, 16, 2, 1, 0.5, 30)
    # nearest size bucket with the same dtype and contrast bucket
    assert d.lookup(1024, 1024, 1e4, "f64").k == 2
    assert d.lookup(8192, 8192, 1e4, "f64").k == 8
    # another contrast or dtype: the default
    assert d.lookup(512, 512, 1e2, "f64") == autotune.DEFAULT
    assert d.lookup(512, 512, 1e4, "f32") == autotune.DEFAULT


def test_candidates_are_valid_schedules():
    assert len(autotune.DEFAULT_CANDIDATES) >= 12
    for ti, tj, k, o in autotune.DEFAULT_CANDIDATES:
        assert k >= 1 and o in (0, k - 1)
        assert autotune.feasible(ti, tj, k, o, 1024, 1024)
    assert not autotune.feasible(64, 32, 4, 3, 48, 48)


@pytest.mark.gpu
def test_tuning_run_picks_the_fastest_converging_schedule(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19061_gb300 import api, build
    build.build()
    prob = inputs.sinker_problem(128, eta_in=1e4)
    cands = [(16, 16, 2, 1), (32, 32, 4, 3), (32, 32, 4, 0), (16, 16, 1, 0)]
    win, table = autotune.tune(api, prob, candidates=cands, tol=1e-8)
    assert len(table) == 4
    assert all(math.isfinite(c.seconds) and c.cycles > 0 for c in table)
    assert win.seconds == min(c.seconds for c in table)
    cache = autotune.Cache(str(tmp_path / "t.json"))
    cache.record(prob.nx, prob.ny, autotune.contrast_of(prob.eta_c, prob.eta_n), "f64", win)
    cache.save()
    got = autotune.Cache(str(tmp_path / "t.json")).lookup(128, 128, 1e4, "f64")
    assert (got.tile_i, got.tile_j, got.k, got.overlap) == (win.tile_i, win.tile_j, win.k, win.overlap)
    ctx = api.StokesContext(128, 128, 1.0, 1.0, "f64")
    ctx.set_problem(prob)
    vx, vy = ctx.field(), ctx.field()
    st, e, c = ctx.vcycle(vx, vy, None, inner="f32", tol=1e-8, max_cycles=300, nu_max=40, **got.smoother())
    assert st == api.STOKES_OK and e <= 1e-8
    ctx.close()


def test_shipped_cache_covers_the_tuned_buckets():
    c = autotune.Cache(autotune.SHIPPED)
    assert len(c.entries) >= 9
    for key, ch in c.entries.items():
        assert math.isfinite(ch.seconds) and ch.cycles > 0, key
        assert autotune.feasible(ch.tile_i, ch.tile_j, ch.k, ch.overlap, 256, 256)
    kw = autotune.tuned_smoother(1024, 1024, np.ones((2, 2)), np.full((3, 3), 1e4))
    assert kw["variant"] == "ras" and kw["k"] >= 1


@pytest.mark.gpu
def test_tuner_keeps_only_register_layout_shapes():
    """Launch shapes whose window fits no register layout run the general
    shared-memory tile kernel (3 to 5 times slower per sweep); the tuner
    leaves them out, so no tuned schedule falls off that cliff."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19061_gb300 import api, build
    build.build()
    assert not autotune.fast_layout(api, 4096, 4096, 56, 32, 7, "f32")   # 72-column window
    assert autotune.fast_layout(api, 4096, 4096, 48, 64, 7, "f32")       # 64 x 80: pair layout
    assert not autotune.fast_layout(api, 1024, 1024, 32, 32, 7, "f64")   # 48 x 48: 576 threads
    assert autotune.fast_layout(api, 1024, 1024, 24, 24, 7, "f64")       # 40 x 40
    for dtype, n in (("f32", 4096), ("f64", 1024)):
        kept = [c for c in autotune.DEFAULT_CANDIDATES if autotune.fast_layout(api, n, n, c[0], c[1], c[3], dtype)]
        assert len(kept) >= 12
        for ti, tj, k, o in kept:
            assert api.stokes_tile_kernel_plan(n, n, (ti, tj), o, dtype)[0] in ("tma", "pair", "global")
