"""GPU parity of the multigrid V-cycle and the defect-correction solve
(Sec. 3.2, configuration of Sec. 6.2) against the FP64 oracle, through the C
ABI.  FP64 inner cycles must match the oracle to 1e-12 (normwise, relative);
FP32 inner cycles with FP64 defect correction must reach the same converged
solution as the all-FP64 path.
"""
import numpy as np
import pytest

import oracle as ora
from paper_2509_19061_gb300 import inputs

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19061_gb300 import api as a, build
    build.build()
    return a


def ogrid(prob):
    return ora.Grid(prob.nx, prob.ny, prob.hx, prob.hy, prob.eta_c, prob.eta_n)


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


VARIANT_CODE = {"jacobi": 0, "fused": 1, "blocked": 2, "rbgs": 3, "ras": 4, "mixed": 5}


def run_solve(api, prob, dtype, cycles, tol=0.0, p=None, **mg):
    import torch
    ctx = api.StokesContext(prob.nx, prob.ny, prob.lx, prob.ly, dtype)
    ctx.set_problem(prob)
    vx, vy = ctx.field(), ctx.field()
    pt = None if p is None else ctx.pack(p, "p")
    st, e, c = ctx.vcycle(vx, vy, pt, tol=tol, max_cycles=cycles, **mg)
    torch.cuda.synchronize()
    v = (ctx.unpack(vx, "vx"), ctx.unpack(vy, "vy"))
    ctx.close()
    return st, e, c, v


def oracle_solve(prob, cycles, tol=0.0, p=None, krylov=False, **mg):
    kw = dict(mg)
    variant = kw.pop("variant", "ras")
    tile = kw.pop("tile", (32, 32))
    k = kw.pop("k", 4)
    overlap = kw.pop("overlap", k - 1)
    m = ora.MG(max_levels=kw.pop("levels", 16), coarsest=kw.pop("coarsest", 16), nu_pre=kw.pop("nu_pre", 5),
               nu_post=kw.pop("nu_post", 5), growth=kw.pop("nu_growth", 2.5), nu_max=kw.pop("nu_max", 0),
               variant=VARIANT_CODE[variant], omega=kw.pop("omega", 0.3), ti=tile[0], tj=tile[1], k=k,
               overlap=overlap, seed=kw.pop("seed", 0))
    kw.pop("inner", None)
    assert not kw, kw
    solve = ora.mg_fcg if krylov else ora.mg_solve
    return solve(ogrid(prob), prob.fx, prob.fy, p, m, tol, cycles)


@pytest.mark.parametrize("case", [
    dict(n=(32, 32), variant="fused"),
    dict(n=(64, 48), variant="jacobi", nu_max=7),
    dict(n=(64, 64), variant="ras", tile=(8, 8), k=2, overlap=0, seed=3),
    dict(n=(96, 64), variant="ras", tile=(16, 12), k=3, overlap=1, seed=9, nu_max=20),
    dict(n=(64, 64), variant="rbgs", nu_max=10),
    dict(n=(48, 40), variant="blocked", tile=(16, 16)),
    dict(n=(128, 96), variant="mixed", tile=(16, 16), k=4, overlap=0, seed=4, nu_max=16),
])
@pytest.mark.parametrize("krylov", [False, True])
def test_vcycle_f64_matches_oracle(api, case, krylov):
    """Two outer iterations (defect correction or flexible CG) with an FP64
    V-cycle (levels down to 16, dense coarsest solve) match the oracle."""
    case = dict(case)
    nx, ny = case.pop("n")
    prob = inputs.sinker_problem(nx, ny, eta_in=1e2, lx=1.0, ly=ny / nx)
    p = inputs.random_pressure(nx, ny, 4, 0.1)
    st, e, c, v = run_solve(api, prob, "f64", 2, p=p, inner="f64", krylov=krylov, **case)
    assert st == api.STOKES_ERR_NOT_CONVERGED and c == 2
    ref = oracle_solve(prob, 2, p=p, krylov=krylov, **case)
    # flexible CG adds inner products, whose summation order differs
    tol = 1e-10 if krylov else F64_TOL
    assert rel(v, ref[:2]) <= tol
    assert abs(e - ref[3]) <= 1e-9 * ref[3]


@pytest.mark.parametrize("n,variant", [((512, 384), "ras"), ((512, 384), "mixed"), ((1024, 1024), "ras")])
@pytest.mark.parametrize("krylov", [False, True])
def test_vcycle_f64_matches_oracle_at_depth(api, n, variant, krylov):
    """The paper's uncapped sweep schedule (Sec. 6.2: 5, 13, 32, 79, 196, 489
    sweeps from the finest level down) on hierarchies of 6 and 7 levels, with
    the coarse levels small enough to run as one whole-level tile and the
    dense solve at the bottom: two outer iterations against the oracle."""
    nx, ny = n
    prob = inputs.sinker_problem(nx, ny, eta_in=1e3, lx=1.0, ly=0.7 * ny / nx)
    p = inputs.random_pressure(nx, ny, 5, 0.1)
    case = dict(variant=variant, tile=(32, 32), k=4, overlap=3 if variant == "ras" else 0, seed=2)
    assert ora.mg_levels(nx, ny, 16, 16) >= 6
    st, e, c, v = run_solve(api, prob, "f64", 2, p=p, inner="f64", krylov=krylov, **case)
    assert st == api.STOKES_ERR_NOT_CONVERGED and c == 2
    ref = oracle_solve(prob, 2, p=p, krylov=krylov, **case)
    tol = 1e-10 if krylov else F64_TOL
    assert rel(v, ref[:2]) <= tol, rel(v, ref[:2])
    assert abs(e - ref[3]) <= 1e-9 * ref[3]


def test_single_level_is_the_dense_solve(api):
    prob = inputs.sinker_problem(16, 12, eta_in=1e3, ly=0.75)
    st, e, c, v = run_solve(api, prob, "f64", 1, inner="f64", levels=1, variant="fused")
    dx, dy = ora.dense_solve(ogrid(prob), prob.fx, prob.fy)
    assert rel(v, (dx, dy)) <= 1e-11


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_solve_to_1e8_fp32_inner_reaches_the_fp64_solution(api, inner):
    """Flexible CG in FP64 around the V-cycle reaches E_v <= 1e-8 on the
    1e6-contrast multi-sinker with an FP32 or FP64 inner cycle; both land on
    the oracle's converged solution."""
    prob = inputs.multi_sinker(128, seed=3)
    kw = dict(variant="ras", tile=(32, 32), k=4, overlap=3, nu_max=40, seed=1)
    st, e, c, v = run_solve(api, prob, "f64", 80, tol=1e-8, inner=inner, krylov=True, **kw)
    assert st == api.STOKES_OK and e <= 1e-8, (st, e, c)
    ref = oracle_solve(prob, 120, tol=1e-10, krylov=True, **kw)
    assert ref[3] <= 1e-10
    g = ogrid(prob)
    dx, dy = ora.diag_M(g)
    num = np.sum(-dx * (v[0] - ref[0]) ** 2) + np.sum(-dy * (v[1] - ref[1]) ** 2)
    den = np.sum(-dx * ref[0] ** 2) + np.sum(-dy * ref[1] ** 2)
    err = float(np.sqrt(num / den))
    print("inner %s: %d cycles, E_v %.2e, energy error vs converged oracle %.2e" % (inner, c, e, err))
    assert err <= 1e-6


def test_multigrid_errors(api):
    prob = inputs.sinker_problem(64)
    with pytest.raises(api.StokesError) as ex:
        run_solve(api, prob, "f64", 1, inner="f64", levels=1, variant="fused")  # 64^2 dense: too large
    assert ex.value.status == api.STOKES_ERR_ARG
    ctx = api.StokesContext(32, 32, 1.0, 1.0, "f64")
    vx, vy = ctx.field(), ctx.field()
    with pytest.raises(api.StokesError) as ex:
        ctx.vcycle(vx, vy, variant="fused")
    assert ex.value.status == api.STOKES_ERR_STATE
    ctx.close()


def test_refinement_f64_matches_the_oracle(api):
    """krylov = 2 with an FP64 inner precision: two outer defect-correction
    steps, each three flexible-CG iterations preconditioned by the V-cycle,
    match the oracle's refinement loop."""
    prob = inputs.sinker_problem(96, 64, eta_in=1e3, lx=1.0, ly=64 / 96)
    kw = dict(variant="ras", tile=(16, 16), k=4, overlap=3, seed=3, nu_max=20)
    st, e, c, v = run_solve(api, prob, "f64", 6, inner="f64", krylov=2, inner_its=3, **kw)
    assert st == api.STOKES_ERR_NOT_CONVERGED and c == 6
    m = ora.MG(variant=4, ti=16, tj=16, k=4, overlap=3, seed=3, nu_max=20)
    rx, ry, rc, re, rh = ora.mg_refine(ogrid(prob), prob.fx, prob.fy, None, m, 0.0, 6, 3)
    assert rel(v, (rx, ry)) <= 1e-10
    assert abs(e - re) <= 1e-8 * re


def test_refinement_fp32_inner_reaches_1e8(api):
    """FP32 inner flexible CG (operator, updates and the V-cycle in FP32)
    inside FP64 defect correction reaches E_v <= 1e-8 on the 1e6-contrast
    multi-sinker and lands on the oracle's converged solution."""
    prob = inputs.multi_sinker(128, seed=3)
    kw = dict(variant="ras", tile=(32, 32), k=4, overlap=3, nu_max=40, seed=1)
    st, e, c, v = run_solve(api, prob, "f64", 120, tol=1e-8, inner="f32", krylov=2, inner_its=8, **kw)
    assert st == api.STOKES_OK and e <= 1e-8, (st, e, c)
    ref = oracle_solve(prob, 120, tol=1e-10, krylov=True, **kw)
    g = ogrid(prob)
    dx, dy = ora.diag_M(g)
    num = np.sum(-dx * (v[0] - ref[0]) ** 2) + np.sum(-dy * (v[1] - ref[1]) ** 2)
    den = np.sum(-dx * ref[0] ** 2) + np.sum(-dy * ref[1] ** 2)
    print("refinement, fp32 inner: %d V-cycles, E_v %.2e, energy error %.2e" % (c, e, np.sqrt(num / den)))
    assert np.sqrt(num / den) <= 1e-6


def test_nan_viscosity_is_reported_as_diverged(api):
    """A NaN planted in eta on the host reaches the residual: the solve stops
    with STOKES_ERR_DIVERGED instead of running on."""
    prob = inputs.sinker_problem(64, eta_in=1e3)
    prob.eta_c = prob.eta_c.copy()
    prob.eta_c[20, 30] = np.nan
    ctx = api.StokesContext(64, 64, 1.0, 1.0, "f64")
    ctx.set_problem(prob)
    vx, vy = ctx.field(), ctx.field()
    with pytest.raises(api.StokesError) as e:
        ctx.vcycle(vx, vy, None, variant="ras", tile=(32, 32), k=4, overlap=3, inner="f32", tol=1e-8, max_cycles=20)
    assert e.value.status == api.STOKES_ERR_DIVERGED
    ctx.close()
