"""GPU parity of the batched path (many instances of different sizes in one
launch per step, the batched V-cycle as one CUDA graph) against one context
per instance, through the C ABI.

Every instance follows the schedule of its own context, so the smoothing
results and the V-cycle / defect-correction iterates must agree bit for bit;
the flexible-CG solve sums its inner products in another order and is
compared to rounding.  The single-context path is itself pinned to the FP64
oracle by the other GPU tests.
"""
import numpy as np
import pytest

from paper_2509_19061_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19061_gb300 import api as a, build
    build.build()
    return a


def problems(sizes, seed):
    out = []
    for q, (nx, ny) in enumerate(sizes):
        ec, en = inputs.random_viscosity(nx, ny, seed + q, (-2.0, 2.0))
        prob = inputs.sinker_problem(nx, ny, eta_in=1e3, lx=1.0, ly=ny / nx)
        prob.eta_c, prob.eta_n = ec, en
        out.append(prob)
    return out


def single_results(api, probs, dtype, v0, p, fn):
    """Run fn(ctx, vx, vy, pt) on one context per instance; natural-shape v."""
    import torch
    res = []
    for q, prob in enumerate(probs):
        ctx = api.StokesContext(prob.nx, prob.ny, prob.lx, prob.ly, dtype)
        ctx.set_problem(prob)
        vx, vy = ctx.pack(v0[q][0], "vx"), ctx.pack(v0[q][1], "vy")
        pt = None if p is None else ctx.pack(p[q], "p")
        out = fn(ctx, vx, vy, pt)
        torch.cuda.synchronize()
        res.append((ctx.unpack(vx, "vx"), ctx.unpack(vy, "vy"), out))
        ctx.close()
    return res


def batch_context(api, probs, dtype):
    b = api.BatchContext([q.nx for q in probs], [q.ny for q in probs], [q.lx for q in probs],
                         [q.ly for q in probs], dtype)
    b.set_problems(probs)
    return b


SIZES = [(40, 24), (64, 64), (100, 70), (33, 50), (8, 12)]


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("kw", [
    dict(variant="ras", sweeps=9, tile=(32, 32), k=4, overlap=3, seed=5),
    dict(variant="ras", sweeps=7, tile=(16, 12), k=3, overlap=1, seed=11),
    dict(variant="ras", sweeps=6, tile=(8, 8), k=2, overlap=0, shifts=[[1, 2], [7, 0], [3, 3]]),
    dict(variant="jacobi", sweeps=5),
    dict(variant="fused", sweeps=6),
    dict(variant="blocked", sweeps=3, tile=(16, 16)),
    dict(variant="ras", sweeps=9, tile=(56, 32), k=4, overlap=3, seed=5),    # 64-column windows: FP32 pair layout
    dict(variant="ras", sweeps=17, tile=(48, 64), k=8, overlap=7, seed=3),   # 64 x 80 windows, 20 warps
])
@pytest.mark.parametrize("tma", [True, False])
def test_batched_smoothing_is_bitwise_the_single_context(api, dtype, kw, tma):
    import torch
    if dtype == "f64" and kw.get("tile") == (48, 64):
        pytest.skip("an FP64 64 x 80 window exceeds shared memory (STOKES_ERR_ARG in every path)")
    probs = problems(SIZES, 10)
    v0 = [inputs.random_velocity(q.nx, q.ny, 100 + i) for i, q in enumerate(probs)]
    p = [inputs.random_pressure(q.nx, q.ny, 200 + i, 0.5) for i, q in enumerate(probs)]
    ref = single_results(api, probs, dtype, v0, p, lambda c, vx, vy, pt: c.smooth(vx, vy, pt, **kw))
    b = batch_context(api, probs, dtype)
    b.set_option(api.STOKES_OPT_USE_TMA, 1 if tma else 0)
    vx, vy = b.pack([v[0] for v in v0], "vx"), b.pack([v[1] for v in v0], "vy")
    pt = b.pack(p, "p")
    b.smooth(vx, vy, pt, **kw)
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert np.array_equal(b.unpack(vx, "vx", i), ref[i][0]), (i, "vx")
        assert np.array_equal(b.unpack(vy, "vy", i), ref[i][1]), (i, "vy")
    # a second call reuses the cached plan and continues from the result
    b.smooth(vx, vy, pt, **kw)
    ref2 = single_results(api, probs, dtype, [(r[0], r[1]) for r in ref], p,
                          lambda c, x, y, q: c.smooth(x, y, q, **kw))
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert np.array_equal(b.unpack(vx, "vx", i), ref2[i][0])
        assert np.array_equal(b.unpack(vy, "vy", i), ref2[i][1])
    b.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batched_energy_matches_the_single_context(api, dtype):
    probs = problems(SIZES, 20)
    v0 = [inputs.random_velocity(q.nx, q.ny, 300 + i) for i, q in enumerate(probs)]
    p = [inputs.random_pressure(q.nx, q.ny, 400 + i, 0.5) for i, q in enumerate(probs)]
    ref = single_results(api, probs, dtype, v0, p, lambda c, vx, vy, pt: c.energy(vx, vy, pt))
    b = batch_context(api, probs, dtype)
    vx, vy = b.pack([v[0] for v in v0], "vx"), b.pack([v[1] for v in v0], "vy")
    e = b.energy(vx, vy, b.pack(p, "p"))
    for i in range(len(probs)):
        rv, _, ff = ref[i][2]
        assert abs(e[i, 0] - rv) <= 1e-12 * rv and abs(e[i, 1] - ff) <= 1e-12 * ff
    b.close()


SQUARE_SIZES = [(64, 64), (100, 100), (48, 48), (130, 130), (7, 7)]


@pytest.mark.parametrize("kw", [
    dict(variant="ras", sweeps=9, tile=(56, 32), k=4, overlap=3, seed=5),
    dict(variant="ras", sweeps=17, tile=(48, 64), k=8, overlap=7, seed=3),
    dict(variant="ras", sweeps=10, tile=(62, 56), k=8, overlap=0, seed=8),
])
def test_batched_pair_layout_square_cells(api, kw):
    """A batch whose instances all have square cells runs the pair layout in
    its square-cell form; every instance equals its own context (which takes
    the same form) value for value, and the exact-Jacobi schedules equal
    global fused Jacobi."""
    import torch
    probs = problems(SQUARE_SIZES, 60)
    assert all(q.lx / q.nx == q.ly / q.ny for q in probs)
    v0 = [inputs.random_velocity(q.nx, q.ny, 600 + i) for i, q in enumerate(probs)]
    ref = single_results(api, probs, "f32", v0, None, lambda c, vx, vy, pt: c.smooth(vx, vy, pt, **kw))
    b = batch_context(api, probs, "f32")
    vx, vy = b.pack([v[0] for v in v0], "vx"), b.pack([v[1] for v in v0], "vy")
    b.smooth(vx, vy, None, **kw)
    torch.cuda.synchronize()
    for i in range(len(probs)):
        assert np.array_equal(b.unpack(vx, "vx", i), ref[i][0]), (i, "vx")
        assert np.array_equal(b.unpack(vy, "vy", i), ref[i][1]), (i, "vy")
    if kw["overlap"] >= kw["k"] - 1:
        jac = single_results(api, probs, "f32", v0, None,
                             lambda c, vx, vy, pt: c.smooth(vx, vy, pt, variant="fused", sweeps=kw["sweeps"]))
        for i in range(len(probs)):
            assert np.array_equal(b.unpack(vx, "vx", i), jac[i][0]), (i, "vx")
            assert np.array_equal(b.unpack(vy, "vy", i), jac[i][1]), (i, "vy")
    b.close()


def test_batched_pair_wait_timeout_is_reported(api):
    """The batched pair kernel's bounded staging wait: a limit below zero
    gives up at once, the timeout is reported, and the batch recovers."""
    import torch
    probs = problems([(64, 64), (100, 100)], 70)
    b = batch_context(api, probs, "f32")
    vx, vy = b.slab(), b.slab()
    b.set_option(api.STOKES_OPT_WAIT_LIMIT_CYCLES, -1)
    b.smooth(vx, vy, variant="ras", sweeps=4, tile=(56, 32), k=4, overlap=3)
    with pytest.raises(api.StokesError) as ex:
        b.energy(vx, vy)
    assert ex.value.status == api.STOKES_ERR_TIMEOUT
    b.set_option(api.STOKES_OPT_WAIT_LIMIT_CYCLES, 2000000000)
    vx.zero_()
    vy.zero_()
    b.smooth(vx, vy, variant="ras", sweeps=4, tile=(56, 32), k=4, overlap=3)
    e = b.energy(vx, vy)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(e)) and np.all(e[:, 0] < e[:, 1])
    b.close()


MG_SIZES = [(64, 64), (96, 64), (80, 48), (128, 128), (32, 32)]


@pytest.mark.parametrize("dtype,inner", [("f64", "f64"), ("f64", "f32"), ("f32", "f32")])
@pytest.mark.parametrize("sm", [
    dict(variant="ras", tile=(32, 32), k=4, overlap=3, seed=1, nu_max=12),
    dict(variant="ras", tile=(16, 8), k=2, overlap=0, seed=9, nu_max=10),
    dict(variant="jacobi", nu_max=9),
    dict(variant="mixed", tile=(16, 16), k=4, overlap=0, seed=6, nu_max=10),
    dict(variant="ras", tile=(56, 32), k=4, overlap=3, seed=2, nu_max=12),   # pair layout on the 64+ levels
])
def test_batched_defect_correction_is_bitwise_the_single_context(api, dtype, inner, sm):
    """Three defect-correction cycles: every iterate is v += B(b - M v), with
    no inner products on the path, so the batched V-cycle graph must
    reproduce each instance's own context bit for bit."""
    import torch
    probs = [inputs.sinker_problem(nx, ny, eta_in=10.0 ** (1 + 0.5 * i), lx=1.0, ly=ny / nx)
             for i, (nx, ny) in enumerate(MG_SIZES)]
    v0 = [(np.zeros((q.ny, q.nx + 1)), np.zeros((q.ny + 1, q.nx))) for q in probs]
    kw = dict(sm, inner=inner, krylov=False, tol=0.0, max_cycles=3)
    ref = single_results(api, probs, dtype, v0, None, lambda c, vx, vy, pt: c.vcycle(vx, vy, pt, **kw))
    b = batch_context(api, probs, dtype)
    vx, vy = b.slab(), b.slab()
    st, e, cyc, sts = b.solve(vx, vy, None, **kw)
    torch.cuda.synchronize()
    assert st == api.STOKES_ERR_NOT_CONVERGED and list(cyc) == [3] * len(probs)
    for i in range(len(probs)):
        assert np.array_equal(b.unpack(vx, "vx", i), ref[i][0]), i
        assert np.array_equal(b.unpack(vy, "vy", i), ref[i][1]), i
        assert abs(e[i] - ref[i][2][1]) <= 1e-12 * ref[i][2][1]
    assert b.kernels() > 0
    b.close()


def test_batched_fcg_reaches_1e8_like_the_single_contexts(api):
    """Flexible CG to E_v <= 1e-8 on sinkers of uneven sizes and contrasts
    1e2..1e6 (the batched workload's recipe): every instance converges, in
    the cycles its own context needs (rounding of the inner products aside),
    to the same solution."""
    import torch
    specs = inputs.batch_specs(seed=5, count=6)
    probs = [inputs.batch_problem(sp) for sp in specs]
    kw = dict(variant="ras", tile=(32, 32), k=4, overlap=3, seed=1, nu_max=40, inner="f32", krylov=True,
              tol=1e-8, max_cycles=200)
    v0 = [(np.zeros((q.ny, q.nx + 1)), np.zeros((q.ny + 1, q.nx))) for q in probs]
    ref = single_results(api, probs, "f64", v0, None, lambda c, vx, vy, pt: c.vcycle(vx, vy, pt, **kw))
    b = batch_context(api, probs, "f64")
    vx, vy = b.slab(), b.slab()
    st, e, cyc, sts = b.solve(vx, vy, None, **kw)
    torch.cuda.synchronize()
    assert st == api.STOKES_OK and all(s == api.STOKES_OK for s in sts)
    for i, q in enumerate(probs):
        rst, re, rc = ref[i][2]
        assert rst == api.STOKES_OK and e[i] <= 1e-8
        assert abs(int(cyc[i]) - rc) <= 2, (i, cyc[i], rc)
        dx = b.unpack(vx, "vx", i) - ref[i][0]
        dy = b.unpack(vy, "vy", i) - ref[i][1]
        num = np.sum(dx ** 2) + np.sum(dy ** 2)
        den = np.sum(ref[i][0] ** 2) + np.sum(ref[i][1] ** 2)
        assert np.sqrt(num / den) <= 1e-6, i
    b.close()


def test_batched_errors(api):
    import torch
    probs = problems([(32, 32), (40, 40)], 30)
    b = batch_context(api, probs, "f64")
    vx, vy = b.slab(), b.slab()
    with pytest.raises(api.StokesError) as ex:
        b.smooth(vx, vy, variant="rbgs", sweeps=2)
    assert ex.value.status == api.STOKES_ERR_ARG
    with pytest.raises(api.StokesError) as ex:
        b.smooth(vx, vy, variant="ras", sweeps=2, k=0)
    assert ex.value.status == api.STOKES_ERR_ARG
    b.close()
    # an instance whose coarsest level is too large for the dense solve
    b = batch_context(api, problems([(32, 32), (126, 126)], 40), "f64")
    with pytest.raises(api.StokesError) as ex:
        b.solve(b.slab(), b.slab(), variant="ras", inner="f64")
    assert ex.value.status == api.STOKES_ERR_ARG
    b.close()
    # solve before the problem is set
    b = api.BatchContext([32], [32], dtype="f64")
    with pytest.raises(api.StokesError) as ex:
        b.solve(b.slab(), b.slab(), variant="ras")
    assert ex.value.status == api.STOKES_ERR_STATE
    b.close()
    torch.cuda.synchronize()


def test_batched_wait_timeout_is_reported_and_recoverable(api):
    """A bounded wait that gives up (limit below zero: at once) is recorded on
    the device and reported by the next synchronising call; the batch keeps
    working once the limit is restored."""
    import torch
    probs = problems([(64, 64), (40, 72)], 50)
    b = batch_context(api, probs, "f32")
    vx, vy = b.slab(), b.slab()
    b.set_option(api.STOKES_OPT_WAIT_LIMIT_CYCLES, -1)
    b.smooth(vx, vy, variant="ras", sweeps=4, tile=(32, 32), k=4, overlap=3)
    with pytest.raises(api.StokesError) as ex:
        b.energy(vx, vy)
    assert ex.value.status == api.STOKES_ERR_TIMEOUT
    b.set_option(api.STOKES_OPT_WAIT_LIMIT_CYCLES, 2000000000)
    vx.zero_()
    vy.zero_()
    b.smooth(vx, vy, variant="ras", sweeps=4, tile=(32, 32), k=4, overlap=3)
    e = b.energy(vx, vy)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(e)) and np.all(e[:, 0] < e[:, 1])
    b.close()


@pytest.mark.parametrize("tile,k,o", [((48, 64), 8, 7),   # the benchmark's (autotuned) schedule: pair layout
                                      ((48, 32), 8, 7),   # the smaller pair-kernel instance
                                      ((32, 32), 4, 3)])  # one-column TMA layout
def test_full_batched_workload_samples_match_single_contexts(api, tile, k, o):
    """The batched workload at full size (256 seeded instances, sides 64 to
    1024, 4.85e7 cells) in the benchmark's launch configuration (FP32 RAS,
    the autotuned 48 x 64, k = 8, overlap 7 on the pair layout, TMA staging),
    with 48 x 32 tiles and in the one-column layout: eight sweeps; sampled
    instances (the smallest, the largest and two others) equal their own
    contexts bit for bit."""
    import torch
    specs = inputs.batch_specs(seed=5, count=256)
    probs = [inputs.batch_problem(sp) for sp in specs]
    kw = dict(variant="ras", sweeps=8, tile=tile, k=k, overlap=o, seed=1)
    b = batch_context(api, probs, "f32")
    vx, vy = b.slab(), b.slab()
    b.smooth(vx, vy, None, **kw)
    torch.cuda.synchronize()
    sizes = [q.nx for q in probs]
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 200})
    v0 = [(np.zeros((probs[i].ny, probs[i].nx + 1)), np.zeros((probs[i].ny + 1, probs[i].nx))) for i in sample]
    ref = single_results(api, [probs[i] for i in sample], "f32", v0, None,
                         lambda c, x, y, pt: c.smooth(x, y, pt, **kw))
    for r, i in zip(ref, sample):
        assert np.array_equal(b.unpack(vx, "vx", i), r[0]), i
        assert np.array_equal(b.unpack(vy, "vy", i), r[1]), i
    b.close()
