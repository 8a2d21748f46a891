"""stokes_energy_norm_noalloc: the energy-norm entry point for callers that
cannot allocate device memory (no context, scratch in a static device
array).  It must give the same sums as stokes_residual_energy_norm.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It also passes on its own in
a fresh process.
"""
import numpy as np
import pytest

from paper_2509_19061_gb300 import inputs

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12  # the tolerance of the FP64 parity tests


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_19061_gb300 import api as a, build
    build.build()
    return a


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_context_energy_norm_twice(api, dtype):
    import torch
    nx, ny, lx, ly = 183, 127, 1.3, 0.9
    prob = inputs.sinker_problem(nx, ny, lx=lx, ly=ly, eta_in=1e3)
    ctx = api.StokesContext(nx, ny, lx, ly, dtype)
    ec, en = ctx.pack(prob.eta_c, "eta_c"), ctx.pack(prob.eta_n, "eta_n")
    fx, fy = ctx.pack(prob.fx, "fx"), ctx.pack(prob.fy, "fy")
    ctx.set_viscosity_dev(ec, en)
    ctx.set_rhs_dev(fx, fy)
    p = ctx.pack(inputs.random_pressure(nx, ny, 2), "p")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((5, 6)):  # two calls in a row, different states
        v = inputs.random_velocity(nx, ny, seed, 0.01)
        vx, vy = ctx.pack(v[0], "vx"), ctx.pack(v[1], "vy")
        want = ctx.energy(vx, vy, p)
        out.fill_(-1.0)
        api.stokes_energy_norm_noalloc(nx, ny, lx, ly, ctx.dtype_code, ctx.pitch, ec, en, fx, fy, p, vx, vy, out,
                                       stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for a, b in zip(got, want):
            assert abs(a - b) <= REL_TOL * abs(b), (call, got, want)
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_without_pressure_matches_context(api, dtype):
    """p = NULL means p = 0: the sums equal the context's without a pressure."""
    import torch
    nx, ny, lx, ly = 97, 64, 1.0, 0.8
    prob = inputs.sinker_problem(nx, ny, lx=lx, ly=ly, eta_in=1e4)
    ctx = api.StokesContext(nx, ny, lx, ly, dtype)
    ec, en = ctx.pack(prob.eta_c, "eta_c"), ctx.pack(prob.eta_n, "eta_n")
    fx, fy = ctx.pack(prob.fx, "fx"), ctx.pack(prob.fy, "fy")
    ctx.set_viscosity_dev(ec, en)
    ctx.set_rhs_dev(fx, fy)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (8, 9):
        v = inputs.random_velocity(nx, ny, seed, 0.01)
        vx, vy = ctx.pack(v[0], "vx"), ctx.pack(v[1], "vy")
        want = ctx.energy(vx, vy, None)
        assert want[1] > 0.0
        api.stokes_energy_norm_noalloc(nx, ny, lx, ly, ctx.dtype_code, ctx.pitch, ec, en, fx, fy, None, vx, vy, out,
                                       stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for a, b in zip(got, want):
            assert abs(a - b) <= REL_TOL * abs(b), (got, want)
    ctx.close()


def test_noalloc_rejects_grids_beyond_its_limits(api):
    import torch
    t = torch.zeros(8, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for nx, ny, pitch in ((46341, 8, 46400), (8, 1, 32), (8, 8, 8)):
        with pytest.raises(api.StokesError) as e:
            api.stokes_energy_norm_noalloc(nx, ny, 1.0, 1.0, api.STOKES_F32, pitch, t, t, t, t, None, t, t, out)
        assert e.value.status == api.STOKES_ERR_ARG
