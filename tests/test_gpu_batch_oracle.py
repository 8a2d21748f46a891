"""The batched path checked directly against the FP64 oracle, through the C ABI.

Each instance of a batch (instances of uneven sizes, one launch per step
for all of them, per-instance tensor maps, persistent tile assignment,
segment-mapped element-wise kernels) must reproduce, instance by instance,
the oracle's RAS-Jacobi (Algorithm 2) and its multigrid solves (Sec. 3.2,
configuration of Sec. 6.2).  FP64: relative 1e-12 normwise and, element by
element, max |v_gpu - v_oracle| <= 1e-12 max |v_oracle|; FP32: the energy-norm
gate of the single-context tests (1e-5) against the oracle run on the
FP32-rounded inputs.
"""
import numpy as np
import pytest

import oracle as ora
from paper_2509_19061_gb300 import inputs

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
FP32_ENERGY_TOL = 1e-5


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19061_gb300 import api as a, build
    build.build()
    return a


def ogrid(prob, cast=None):
    c = (lambda a: a) if cast is None else cast
    return ora.Grid(prob.nx, prob.ny, prob.hx, prob.hy, c(prob.eta_c), c(prob.eta_n))


def rel(a, b):
    """The larger of the normwise relative error ||a - b||_2 / ||b||_2 and the
    element-wise one max |a - b| / max |b| over every entry of all components
    (the second catches an error confined to a few unknowns, e.g. next to a
    wall, that the norm would average away)."""
    num = sum(np.sum((x - y) ** 2) for x, y in zip(a, b))
    den = sum(np.sum(y ** 2) for y in b)
    emax = max(float(np.max(np.abs(x - y))) for x, y in zip(a, b))
    bmax = max(float(np.max(np.abs(y))) for y in b)
    return max(float(np.sqrt(num / den)), emax / bmax)


def max_rel(a, b):
    """max |a - b| over every entry of both components / max |b|."""
    num = max(float(np.max(np.abs(x - y))) for x, y in zip(a, b))
    den = max(float(np.max(np.abs(y))) for y in b)
    return num / den


def energy_rel(g, a, b):
    dx, dy = ora.diag_M(g)
    num = np.sum(-dx * (a[0] - b[0]) ** 2) + np.sum(-dy * (a[1] - b[1]) ** 2)
    den = np.sum(-dx * b[0] ** 2) + np.sum(-dy * b[1] ** 2)
    return float(np.sqrt(num / den))


def f32(a):
    return None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)


# uneven instances: a non-square one with hx != hy, one of 512^2 cells, a
# ragged one smaller than a tile, different contrasts
SIZES = [(96, 40, 1.0, 0.7, 1e2), (512, 512, 1.0, 1.0, 1e4), (37, 53, 0.8, 1.1, 1e3), (130, 66, 1.3, 0.9, 1e6)]


def uneven_problems():
    probs = []
    for q, (nx, ny, lx, ly, contrast) in enumerate(SIZES):
        prob = inputs.sinker_problem(nx, ny, eta_in=contrast, lx=lx, ly=ly, radius=0.15)
        probs.append(prob)
    return probs


def batch_context(api, probs, dtype):
    b = api.BatchContext([q.nx for q in probs], [q.ny for q in probs], [q.lx for q in probs],
                         [q.ly for q in probs], dtype)
    b.set_problems(probs)
    return b


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("kw", [
    dict(variant="ras", sweeps=10, tile=(32, 32), k=4, overlap=3, seed=7),   # exact Jacobi (o = k - 1)
    dict(variant="ras", sweeps=9, tile=(24, 16), k=4, overlap=0, seed=3),    # ring-only tiles (o = 0)
    dict(variant="ras", sweeps=11, tile=(16, 16), k=3, overlap=1, seed=12),  # 0 < o < k - 1, remainder pass
    dict(variant="ras", sweeps=12, tile=(56, 32), k=4, overlap=3, seed=5),   # FP32 pair layout (64-column windows)
])
def test_batched_ras_matches_the_oracle(api, dtype, kw):
    """RAS smoothing of four uneven instances in one batched call, from a
    random state with a non-zero pressure: every instance equals the oracle's
    RAS with the same tiles, k, overlap and SplitMix64 shift seed."""
    import torch
    probs = uneven_problems()
    v0 = [inputs.random_velocity(q.nx, q.ny, 500 + i, 1e-2) for i, q in enumerate(probs)]
    p = [inputs.random_pressure(q.nx, q.ny, 600 + i, 0.3) for i, q in enumerate(probs)]
    b = batch_context(api, probs, dtype)
    vx, vy = b.pack([v[0] for v in v0], "vx"), b.pack([v[1] for v in v0], "vy")
    b.smooth(vx, vy, b.pack(p, "p"), **kw)
    torch.cuda.synchronize()
    cast = f32 if dtype == "f32" else (lambda a: a)
    for i, q in enumerate(probs):
        g = ogrid(q, cast)
        bx, by = ora.rhs(g, cast(q.fx), cast(q.fy), cast(p[i]))
        ref = ora.ras(g, bx, by, 0.3, kw["sweeps"], kw["tile"][0], kw["tile"][1], kw["k"], kw["overlap"],
                      shift_mode=1, seed=kw["seed"], vx=cast(v0[i][0]), vy=cast(v0[i][1]))
        got = (b.unpack(vx, "vx", i), b.unpack(vy, "vy", i))
        if dtype == "f64":
            assert rel(got, ref) <= F64_TOL, (i, rel(got, ref))
        else:
            err = energy_rel(g, got, ref)
            assert err <= FP32_ENERGY_TOL, (i, err)
            assert max_rel(got, ref) <= 10 * FP32_ENERGY_TOL, (i, max_rel(got, ref))
    b.close()


@pytest.mark.parametrize("kw", [
    dict(variant="jacobi", sweeps=6),
    dict(variant="fused", sweeps=7),
    dict(variant="blocked", sweeps=5, tile=(16, 16)),
])
def test_batched_jacobi_schedules_match_the_oracle(api, kw):
    """Plain, fused and blocked fused Jacobi (one map, Sec. 5 (ii)-(iv)) in
    one batched call: every instance equals the oracle's Jacobi."""
    import torch
    probs = uneven_problems()
    v0 = [inputs.random_velocity(q.nx, q.ny, 700 + i, 1e-2) for i, q in enumerate(probs)]
    p = [inputs.random_pressure(q.nx, q.ny, 800 + i, 0.3) for i, q in enumerate(probs)]
    b = batch_context(api, probs, "f64")
    vx, vy = b.pack([v[0] for v in v0], "vx"), b.pack([v[1] for v in v0], "vy")
    b.smooth(vx, vy, b.pack(p, "p"), **kw)
    torch.cuda.synchronize()
    for i, q in enumerate(probs):
        g = ogrid(q)
        bx, by = ora.rhs(g, q.fx, q.fy, p[i])
        ref = ora.jacobi(g, bx, by, 0.3, kw["sweeps"], v0[i][0], v0[i][1])
        got = (b.unpack(vx, "vx", i), b.unpack(vy, "vy", i))
        assert rel(got, ref) <= F64_TOL, (i, rel(got, ref))
    b.close()


def test_batched_energy_matches_the_oracle(api):
    """Per-instance energy sums (Sec. 6.4) of the batch against the oracle."""
    probs = uneven_problems()
    v0 = [inputs.random_velocity(q.nx, q.ny, 900 + i, 1e-3) for i, q in enumerate(probs)]
    p = [inputs.random_pressure(q.nx, q.ny, 950 + i, 0.3) for i, q in enumerate(probs)]
    b = batch_context(api, probs, "f64")
    vx, vy = b.pack([v[0] for v in v0], "vx"), b.pack([v[1] for v in v0], "vy")
    e = b.energy(vx, vy, b.pack(p, "p"))
    for i, q in enumerate(probs):
        rv, _, ff = ora.energy(ogrid(q), q.fx, q.fy, p[i], v0[i][0], v0[i][1])
        assert abs(e[i, 0] - rv) <= F64_TOL * rv and abs(e[i, 1] - ff) <= F64_TOL * ff, (i, e[i], rv, ff)
    b.close()


MG_SIZES = [(64, 64, 1.0, 1.0), (96, 64, 1.0, 64 / 96), (80, 48, 1.2, 0.6), (128, 128, 1.0, 1.0),
            (512, 384, 1.0, 0.7)]
VARIANT_CODE = {"jacobi": 0, "fused": 1, "blocked": 2, "rbgs": 3, "ras": 4, "mixed": 5}


def oracle_mg(sm):
    tile = sm.get("tile", (32, 32))
    k = sm.get("k", 4)
    return ora.MG(variant=VARIANT_CODE[sm["variant"]], ti=tile[0], tj=tile[1], k=k, overlap=sm.get("overlap", k - 1),
                  seed=sm.get("seed", 0), nu_max=sm.get("nu_max", 0))


@pytest.mark.parametrize("krylov", [False, True])
@pytest.mark.parametrize("sm", [
    dict(variant="ras", tile=(32, 32), k=4, overlap=3, seed=1, nu_max=12),
    dict(variant="ras", tile=(16, 8), k=2, overlap=0, seed=9, nu_max=10),
    dict(variant="mixed", tile=(16, 16), k=4, overlap=0, seed=6, nu_max=10),
])
def test_batched_solve_matches_the_oracle(api, krylov, sm):
    """Two outer iterations of the batched FP64 solve (one V-cycle graph for
    every instance; defect correction or flexible CG), instance by instance
    against the oracle's mg_solve / mg_fcg, with a non-zero pressure.  Defect
    correction has no inner products on the path (1e-12); flexible CG sums
    its inner products in another order (1e-10, as for one context)."""
    import torch
    probs = [inputs.sinker_problem(nx, ny, eta_in=10.0 ** (2 + 0.5 * i), lx=lx, ly=ly)
             for i, (nx, ny, lx, ly) in enumerate(MG_SIZES)]
    p = [inputs.random_pressure(q.nx, q.ny, 40 + i, 0.1) for i, q in enumerate(probs)]
    b = batch_context(api, probs, "f64")
    vx, vy = b.slab(), b.slab()
    st, e, cyc, sts = b.solve(vx, vy, b.pack(p, "p"), inner="f64", krylov=krylov, tol=0.0, max_cycles=2, **sm)
    torch.cuda.synchronize()
    assert st == api.STOKES_ERR_NOT_CONVERGED and list(cyc) == [2] * len(probs)
    solve = ora.mg_fcg if krylov else ora.mg_solve
    tol = 1e-10 if krylov else F64_TOL
    for i, q in enumerate(probs):
        rx, ry, rc, re, _ = solve(ogrid(q), q.fx, q.fy, p[i], oracle_mg(sm), 0.0, 2)
        got = (b.unpack(vx, "vx", i), b.unpack(vy, "vy", i))
        assert rel(got, (rx, ry)) <= tol, (i, rel(got, (rx, ry)))
        assert abs(e[i] - re) <= 1e-9 * re, (i, e[i], re)
    b.close()
