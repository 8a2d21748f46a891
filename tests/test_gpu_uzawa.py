"""GPU parity of the inexact Uzawa iteration (Sec. 3.1-3.2, configuration of
Sec. 6.2) against the FP64 oracle, through the C ABI: lithostatic start,
pressure update with zero mean, viscosity continuation, and the full
relative energy residual after every cycle."""
import numpy as np
import pytest

import oracle as ora
from paper_2509_19061_gb300 import inputs

pytestmark = pytest.mark.gpu

VARIANT_CODE = {"jacobi": 0, "fused": 1, "blocked": 2, "rbgs": 3, "ras": 4, "mixed": 5}


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


def gpu_uzawa(api, prob, dtype="f64", p0=None, **kw):
    import torch
    ctx = api.StokesContext(prob.nx, prob.ny, prob.lx, prob.ly, dtype)
    ctx.set_problem(prob)
    vx, vy = ctx.field(), ctx.field()
    p = ctx.field() if p0 is None else ctx.pack(p0, "p")
    st, hist, cyc, e = ctx.uzawa(vx, vy, p, **kw)
    torch.cuda.synchronize()
    out = (ctx.unpack(vx, "vx"), ctx.unpack(vy, "vy"), ctx.unpack(p, "p"))
    ctx.close()
    return st, hist, cyc, e, out


def oracle_mg(sm):
    kw = dict(sm)
    variant = kw.pop("variant", "ras")
    tile = kw.pop("tile", (32, 32))
    k = kw.pop("k", 4)
    overlap = kw.pop("overlap", k - 1)
    return ora.MG(max_levels=kw.pop("levels", 16), coarsest=kw.pop("coarsest", 16), nu_pre=kw.pop("nu_pre", 5),
                  nu_post=kw.pop("nu_post", 5), growth=kw.pop("nu_growth", 2.5), nu_max=kw.pop("nu_max", 0),
                  variant=VARIANT_CODE[variant], omega=kw.pop("omega", 0.3), ti=tile[0], tj=tile[1], k=k,
                  overlap=overlap, seed=kw.pop("seed", 0))


def test_lithostatic_start_matches_the_oracle(api):
    prob = inputs.sinker_problem(48, 40, eta_in=1e3, ly=40 / 48)
    st, hist, cyc, e, (vx, vy, p) = gpu_uzawa(api, prob, cycles=0, variant="fused")
    assert cyc == 0
    want = ora.lithostatic(ogrid(prob), prob.fy)
    np.testing.assert_allclose(p, want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_hydrostatic_state_is_a_fixed_point(api):
    """Uniform density: v = 0 and the lithostatic pressure solve the system,
    so the iteration stays there (up to the rounding of G p against f)."""
    nx = ny = 64
    ec, en = inputs.random_viscosity(nx, ny, 31, (-2.0, 2.0))
    prob = inputs.sinker_problem(nx, eta_in=1.0, rho_in=1.0)
    prob.eta_c, prob.eta_n = ec, en
    st, hist, cyc, e, (vx, vy, p) = gpu_uzawa(api, prob, cycles=3, theta_interval=0, variant="ras", tile=(16, 16),
                                              k=2, inner="f64")
    assert np.abs(vx).max() <= 1e-12 and np.abs(vy).max() <= 1e-12
    np.testing.assert_allclose(p, ora.lithostatic(ogrid(prob), prob.fy), rtol=0, atol=1e-11)
    assert np.all(hist <= 1e-12)


@pytest.mark.parametrize("case", [
    dict(n=(64, 48), krylov=True, vel_its=1, theta_interval=8, sm=dict(variant="ras", tile=(8, 8), k=2, overlap=1,
                                                                        seed=5, nu_max=12)),
    dict(n=(64, 64), krylov=True, vel_its=2, theta_interval=0, sm=dict(variant="jacobi", nu_max=10)),
    dict(n=(48, 40), krylov=False, vel_its=1, theta_interval=5, sm=dict(variant="fused", nu_max=10)),
    dict(n=(96, 64), krylov=True, vel_its=1, theta_interval=6, sm=dict(variant="mixed", tile=(16, 16), k=4,
                                                                        overlap=0, seed=2, nu_max=16)),
])
def test_uzawa_f64_matches_the_oracle(api, case):
    """Thirty Uzawa cycles with an FP64 V-cycle: velocity, pressure and the
    residual history match the oracle (the CG inner products and the
    pressure mean are summed in another order, hence 1e-9)."""
    nx, ny = case["n"]
    prob = inputs.sinker_problem(nx, ny, eta_in=1e2, ly=ny / nx)
    sm = case["sm"]
    st, hist, cyc, e, v = gpu_uzawa(api, prob, cycles=30, theta_interval=case["theta_interval"], inner="f64",
                                    krylov=case["krylov"], vel_its=case["vel_its"], **sm)
    assert cyc == 30
    rx, ry, rp, rh = ora.uzawa(ogrid(prob), prob.fx, prob.fy, oracle_mg(sm), 30,
                               theta_interval=case["theta_interval"], krylov=case["krylov"],
                               vel_its=case["vel_its"])
    assert rel(v[:2], (rx, ry)) <= 1e-9
    assert rel((v[2],), (rp,)) <= 1e-9
    np.testing.assert_allclose(hist, rh, rtol=1e-8)
    assert abs(v[2].mean()) <= 1e-12 * np.abs(v[2]).max()


def test_uzawa_fp32_context_follows_the_oracle(api):
    """An FP32 context (FP32 fields, sweeps, energy sums with the continuation's
    viscosity and 1/diag formed from it): thirty Uzawa cycles with
    continuation follow the oracle's residual history to FP32 accuracy (each
    cycle adds rounding of order 1e-7 relative to the iterate, which the
    iteration carries along: measured 1.6e-5, bound 2e-4)."""
    nx, ny = 96, 72
    prob = inputs.sinker_problem(nx, ny, eta_in=1e2, ly=ny / nx)
    sm = dict(variant="ras", tile=(16, 16), k=2, overlap=1, seed=3, nu_max=12)
    st, hist, cyc, e, v = gpu_uzawa(api, prob, dtype="f32", cycles=30, theta_interval=8, inner="f32", **sm)
    rx, ry, rp, rh = ora.uzawa(ogrid(prob), prob.fx, prob.fy, oracle_mg(sm), 30, theta_interval=8)
    dev = float(np.max(np.abs(hist - rh) / rh))
    print("fp32 context: max relative deviation of the residual history %.2e" % dev)
    assert cyc == 30 and dev <= 2e-4


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_uzawa_with_continuation_converges_at_contrast_1e6(api, inner):
    """The configuration of Sec. 6.2 on the 128^2 sinker at contrast 1e6:
    continuation in five stages of 25 cycles, one CG step preconditioned by
    one V-cycle per Uzawa cycle; the full energy residual falls by orders of
    magnitude, with FP32 or FP64 sweeps."""
    prob = inputs.sinker_problem(128, eta_in=1e6)
    st, hist, cyc, e, v = gpu_uzawa(api, prob, cycles=300, theta_interval=25, inner=inner, variant="ras",
                                    tile=(32, 32), k=4, overlap=3, seed=1, nu_max=40)
    print("inner %s: E %.2e -> %.2e after %d cycles" % (inner, hist[:10].max(), hist[-1], cyc))
    assert hist[-1] <= 1e-4 * hist[:10].max()


def test_uzawa_errors(api):
    prob = inputs.sinker_problem(32)
    with pytest.raises(api.StokesError) as ex:
        gpu_uzawa(api, prob, cycles=3, omega_p=0.0, variant="fused")
    assert ex.value.status == api.STOKES_ERR_ARG
    ctx = api.StokesContext(32, 32, 1.0, 1.0, "f64")
    vx, vy, p = ctx.field(), ctx.field(), ctx.field()
    with pytest.raises(api.StokesError) as ex:
        ctx.uzawa(vx, vy, p, cycles=3, variant="fused")
    assert ex.value.status == api.STOKES_ERR_STATE
    ctx.close()


@pytest.mark.parametrize("depth", [2, 5])
def test_anderson_uzawa_f64_matches_the_oracle(api, depth):
    """Algorithm 1 over the Uzawa map with an FP64 V-cycle: v, p and the
    residual history follow the oracle (the least-squares weights come from
    inner products summed in another order, hence the looser bound)."""
    prob = inputs.sinker_problem(64, 48, eta_in=1e2, ly=48 / 64)
    sm = dict(variant="ras", tile=(8, 8), k=2, overlap=1, seed=5, nu_max=12)
    st, hist, cyc, e, v = gpu_uzawa(api, prob, cycles=30, theta_interval=8, inner="f64", anderson=depth, **sm)
    rx, ry, rp, rh = ora.anderson_uzawa(ogrid(prob), prob.fx, prob.fy, oracle_mg(sm), 30, depth=depth,
                                        theta_interval=8)
    assert rel(v[:2], (rx, ry)) <= 1e-7
    assert rel((v[2],), (rp,)) <= 1e-7
    np.testing.assert_allclose(hist, rh, rtol=1e-6)


def test_anderson_needs_fewer_uzawa_cycles(api):
    prob = inputs.sinker_problem(128, eta_in=1e6)
    kw = dict(cycles=300, theta_interval=25, tol=1e-8, inner="f32", variant="ras", tile=(32, 32), k=4, overlap=3,
              seed=1, nu_max=40)
    st0, h0, c0, e0, _ = gpu_uzawa(api, prob, **kw)
    st1, h1, c1, e1, _ = gpu_uzawa(api, prob, anderson=5, **kw)
    print("plain %d cycles, Anderson(5) %d cycles" % (c0, c1))
    assert st1 == api.STOKES_OK and e1 <= 1e-8
    assert c1 < c0
