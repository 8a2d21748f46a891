"""The slab decomposition on the GPU (stokes_slabs_*, all slabs on one
device), through the C ABI: RAS-Jacobi (Algorithm 2) with the grid split into
horizontal slabs that exchange halo rows after every outer iteration must
equal the oracle's RAS on the whole grid (FP64: 1e-12 normwise and element
by element) and the single-context smoothing bit for bit (FP32 and FP64)."""
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


def rel(a, b):
    num = sum(np.sum((x - y) ** 2) for x, y in zip(a, b))
    den = sum(np.sum(y ** 2) for y in b)
    emax = max(float(np.max(np.abs(x - y))) for x, y in zip(a, b))
    bmax = max(float(np.max(np.abs(y))) for y in b)
    return max(float(np.sqrt(num / den)), emax / bmax)


def problem(nx, ny, seed, lx=1.2, ly=1.7):
    prob = inputs.sinker_problem(nx, ny, eta_in=1e3, lx=lx, ly=ly)
    prob.eta_c, prob.eta_n = inputs.random_viscosity(nx, ny, seed, (-2.0, 2.0))
    return prob


def slab_run(api, prob, dtype, nslabs, v0, p, **kw):
    import torch
    ctx = api.StokesContext(prob.nx, prob.ny, prob.lx, prob.ly, dtype)  # layout and packing only
    s = api.SlabContext(prob.nx, prob.ny, prob.lx, prob.ly, dtype, nslabs)
    s.set_viscosity_dev(ctx.pack(prob.eta_c, "eta_c"), ctx.pack(prob.eta_n, "eta_n"))
    s.set_rhs_dev(ctx.pack(prob.fx, "fx"), ctx.pack(prob.fy, "fy"))
    vx, vy = ctx.pack(v0[0], "vx"), ctx.pack(v0[1], "vy")
    pt = None if p is None else ctx.pack(p, "p")
    s.smooth(vx, vy, pt, **kw)
    torch.cuda.synchronize()
    out = (ctx.unpack(vx, "vx"), ctx.unpack(vy, "vy"))
    copies = s.exchanges()
    s.close()
    ctx.close()
    return out, copies


def single_run(api, prob, dtype, v0, p, **kw):
    import torch
    ctx = api.StokesContext(prob.nx, prob.ny, prob.lx, prob.ly, dtype)
    ctx.set_problem(prob)
    vx, vy = ctx.pack(v0[0], "vx"), ctx.pack(v0[1], "vy")
    pt = None if p is None else ctx.pack(p, "p")
    ctx.smooth(vx, vy, pt, **kw)
    torch.cuda.synchronize()
    out = (ctx.unpack(vx, "vx"), ctx.unpack(vy, "vy"))
    ctx.close()
    return out


@pytest.mark.parametrize("nslabs", [2, 3, 5])
@pytest.mark.parametrize("kw", [
    dict(sweeps=9, tile=(16, 12), k=4, overlap=0, seed=3),    # ring-only tiles
    dict(sweeps=10, tile=(32, 16), k=4, overlap=3, seed=7),   # exact Jacobi
    dict(sweeps=7, tile=(24, 8), k=3, overlap=1, seed=21),    # 0 < o < k - 1, remainder pass
    dict(sweeps=12, tile=(56, 32), k=4, overlap=3, seed=5),   # 64-column windows (FP32 pair layout)
])
def test_slab_ras_matches_oracle_and_single_context(api, nslabs, kw):
    nx, ny = 150, 241
    prob = problem(nx, ny, 31)
    v0 = inputs.random_velocity(nx, ny, 32, 0.1)
    p = inputs.random_pressure(nx, ny, 33, 0.2)
    H = kw["tile"][1] + kw["overlap"] + 1
    if ny // nslabs < H + 1:
        pytest.skip("slabs thinner than the halo (rejected by design)")
    got, (copies, nbytes) = slab_run(api, prob, "f64", nslabs, v0, p, **kw)
    n_outer = (kw["sweeps"] + kw["k"] - 1) // kw["k"]
    assert copies == n_outer * 4 * (nslabs - 1) and nbytes > 0
    g = ora.Grid(nx, ny, prob.hx, prob.hy, prob.eta_c, prob.eta_n)
    bx, by = ora.rhs(g, prob.fx, prob.fy, p)
    ref = ora.ras(g, bx, by, 0.3, kw["sweeps"], kw["tile"][0], kw["tile"][1], kw["k"], kw["overlap"], shift_mode=1,
                  seed=kw["seed"], vx=v0[0], vy=v0[1])
    assert rel(got, ref) <= F64_TOL, rel(got, ref)
    one = single_run(api, prob, "f64", v0, p, variant="ras", **kw)
    assert np.array_equal(got[0], one[0]) and np.array_equal(got[1], one[1])


@pytest.mark.parametrize("kw", [dict(sweeps=17, tile=(48, 64), k=8, overlap=7, seed=3),
                                dict(sweeps=16, tile=(62, 56), k=8, overlap=0, seed=8),
                                dict(sweeps=12, tile=(32, 32), k=4, overlap=3, seed=1)])
def test_slab_ras_fp32_is_bitwise_the_single_context(api, kw):
    """FP32, the benchmark's tile shapes on a 1024^2 layered sinker split into
    four slabs: the slab result equals the single-grid smoothing bit for bit."""
    n = 1024
    prob = inputs.layered_sinker(n, seed=4)
    v0 = inputs.random_velocity(n, n, 41, 1e-3)
    got, _ = slab_run(api, prob, "f32", 4, v0, None, **kw)
    one = single_run(api, prob, "f32", v0, None, variant="ras", **kw)
    assert np.array_equal(got[0], one[0]) and np.array_equal(got[1], one[1])


def test_slab_errors(api):
    import torch
    prob = problem(64, 60, 50)
    s = api.SlabContext(64, 60, 1.2, 1.7, "f64", 2)
    ctx = api.StokesContext(64, 60, 1.2, 1.7, "f64")
    vx, vy = ctx.field(), ctx.field()
    with pytest.raises(api.StokesError) as e:
        s.smooth(vx, vy, sweeps=4, tile=(8, 8), k=2, overlap=1)
    assert e.value.status == api.STOKES_ERR_STATE
    s.set_viscosity_dev(ctx.pack(prob.eta_c, "eta_c"), ctx.pack(prob.eta_n, "eta_n"))
    s.set_rhs_dev(ctx.pack(prob.fx, "fx"), ctx.pack(prob.fy, "fy"))
    with pytest.raises(api.StokesError) as e:
        s.smooth(vx, vy, variant="fused", sweeps=4)
    assert e.value.status == api.STOKES_ERR_ARG
    with pytest.raises(api.StokesError) as e:  # 30-row slabs, halo 32 + 3 + 1
        s.smooth(vx, vy, sweeps=4, tile=(32, 32), k=4, overlap=3)
    assert e.value.status == api.STOKES_ERR_ARG
    s.smooth(vx, vy, sweeps=4, tile=(8, 8), k=2, overlap=1)
    torch.cuda.synchronize()
    s.close()
    ctx.close()
