"""GPU parity of the 3D path (stokes3d_*: the operator, fused Jacobi,
RAS-Jacobi on 3D tiles and the energy norm; the 3D extension of Sec. 9)
against the 3D FP64 oracle, through the C ABI.  FP64: relative 1e-12,
normwise and element by element; FP32: the energy-norm gate of the 2D tests
(1e-5) against the oracle on the FP32-rounded inputs."""
import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3d
    oracle3d.lib()
    return oracle3d


def rel(a, b):
    num = sum(np.sum((x - y) ** 2) for x, y in zip(a, b))
    den = sum(np.sum(y ** 2) for y in b)
    emax = max(float(np.max(np.abs(x - y))) for x, y in zip(a, b))
    bmax = max(float(np.max(np.abs(y))) for y in b)
    return max(float(np.sqrt(num / den)), emax / bmax)


def problem(nx, ny, nz, seed, l=(1.1, 0.8, 1.3)):
    prob = inputs.sinker3d_problem(nx, ny, nz, eta_in=1e2, lx=l[0], ly=l[1], lz=l[2])
    prob.eta_c, prob.eta_xy, prob.eta_xz, prob.eta_yz = inputs.random_viscosity3d(nx, ny, nz, seed, (-2.0, 2.0))
    return prob


def ogrid(o3, prob, cast=lambda a: a):
    return o3.Grid3(prob.nx, prob.ny, prob.nz, prob.hx, prob.hy, prob.hz, cast(prob.eta_c), cast(prob.eta_xy),
                    cast(prob.eta_xz), cast(prob.eta_yz))


def f32(a):
    return None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)


class Run3:
    def __init__(self, api, prob, dtype, v0=None, p=None):
        self.ctx = api.Stokes3DContext(prob.nx, prob.ny, prob.nz, prob.lx, prob.ly, prob.lz, dtype)
        self.ctx.set_problem(prob)
        if v0 is None:
            v0 = (np.zeros(self.ctx.shape["vx"]), np.zeros(self.ctx.shape["vy"]), np.zeros(self.ctx.shape["vz"]))
        self.v = [self.ctx.pack(a, n) for a, n in zip(v0, ("vx", "vy", "vz"))]
        self.p = None if p is None else self.ctx.pack(p, "p")

    def smooth(self, **kw):
        self.ctx.smooth(*self.v, self.p, **kw)

    def get(self):
        import torch
        torch.cuda.synchronize()
        return tuple(self.ctx.unpack(t, n) for t, n in zip(self.v, ("vx", "vy", "vz")))


@pytest.mark.parametrize("n", [(13, 9, 7), (2, 2, 2), (3, 5, 4), (33, 17, 9)])
def test_operator3d_f64(api, o3, n):
    prob = problem(*n, 1)
    v = inputs.random_velocity3d(*n, 2)
    p = inputs.random_pressure3d(*n, 3)
    r = Run3(api, prob, "f64", v, p)
    out = r.ctx.apply(*r.v, r.p)
    got = tuple(r.ctx.unpack(t, nm) for t, nm in zip(out, ("vx", "vy", "vz")))
    g = ogrid(o3, prob)
    m = o3.apply_M(g, *v)
    # G p = -grad p at the unknowns: the oracle's rhs of f = 0 is -G p
    gp = o3.rhs(g, *g.zeros(), -p)
    want = tuple(a + b for a, b in zip(m, gp))
    assert rel(got, want) <= F64_TOL, rel(got, want)
    # walls zero, padding untouched (zero)
    assert np.all(got[0][:, :, 0] == 0) and np.all(got[0][:, :, n[0]] == 0)
    assert np.all(out[0][n[2]:].cpu().numpy() == 0) and np.all(out[0][:, :, n[0] + 1:].cpu().numpy() == 0)


@pytest.mark.parametrize("with_p", [False, True])
def test_energy3d_f64(api, o3, with_p):
    n = (11, 8, 6)
    prob = problem(*n, 4)
    v = inputs.random_velocity3d(*n, 5, 1e-2)
    p = inputs.random_pressure3d(*n, 6) if with_p else None
    r = Run3(api, prob, "f64", v, p)
    got = r.ctx.energy(*r.v, r.p)
    want = o3.energy(ogrid(o3, prob), (prob.fx, prob.fy, prob.fz), p, v)
    for a, b in zip(got, want):
        assert abs(a - b) <= F64_TOL * abs(b), (got, want)
    assert r.ctx.energy(*r.v, r.p) == got  # fixed summation order


def test_jacobi3d_every_sweep_f64(api, o3):
    n = (12, 10, 9)
    prob = problem(*n, 7)
    v0 = inputs.random_velocity3d(*n, 8, 0.1)
    p = inputs.random_pressure3d(*n, 9, 0.2)
    g = ogrid(o3, prob)
    b = o3.rhs(g, prob.fx, prob.fy, prob.fz, p)
    for s in (1, 2, 5):
        r = Run3(api, prob, "f64", v0, p)
        r.smooth(variant="fused", sweeps=s)
        want = o3.jacobi(g, b, 0.3, s, v0)
        assert rel(r.get(), want) <= F64_TOL, (s, rel(r.get(), want))


@pytest.mark.parametrize("n", [(70, 13, 9), (97, 18, 12)])
def test_jacobi3d_interior_blocks_f64(api, o3, n):
    """Grids large enough that the fused Jacobi has blocks whose points and
    neighbours all lie inside every extent (taken without extent tests) next
    to boundary blocks: every sweep count matches the oracle, and RAS with
    overlap k - 1 equals it bit for bit in FP64 and FP32."""
    prob = problem(*n, 17)
    v0 = inputs.random_velocity3d(*n, 18, 0.1)
    p = inputs.random_pressure3d(*n, 19, 0.2)
    g = ogrid(o3, prob)
    b = o3.rhs(g, prob.fx, prob.fy, prob.fz, p)
    for s in (1, 3):
        r = Run3(api, prob, "f64", v0, p)
        r.smooth(variant="fused", sweeps=s)
        want = o3.jacobi(g, b, 0.3, s, v0)
        assert rel(r.get(), want) <= F64_TOL, (s, rel(r.get(), want))
    for dtype in ("f64", "f32"):
        a = Run3(api, prob, dtype, v0, p)
        a.smooth(variant="ras", sweeps=4, tile=(8, 8, 8), k=2, overlap=1, seed=4)
        f = Run3(api, prob, dtype, v0, p)
        f.smooth(variant="fused", sweeps=4)
        for x, y in zip(a.get(), f.get()):
            assert np.array_equal(x, y), dtype


@pytest.mark.parametrize("n,tile,k,o", [((12, 10, 9), (4, 4, 4), 2, 1), ((12, 10, 9), (5, 3, 4), 3, 0),
                                         ((12, 10, 9), (4, 5, 3), 3, 2), ((20, 20, 20), (8, 8, 8), 2, 1),
                                         ((9, 7, 5), (16, 16, 16), 2, 0), ((17, 6, 11), (4, 4, 4), 4, 3),
                                         ((10, 10, 10), (3, 3, 3), 2, 3)])
def test_ras3d_f64(api, o3, n, tile, k, o):
    prob = problem(*n, 10)
    v0 = inputs.random_velocity3d(*n, 11, 0.1)
    p = inputs.random_pressure3d(*n, 12, 0.2)
    g = ogrid(o3, prob)
    b = o3.rhs(g, prob.fx, prob.fy, prob.fz, p)
    sweeps = 2 * k + 1
    r = Run3(api, prob, "f64", v0, p)
    r.smooth(variant="ras", sweeps=sweeps, tile=tile, k=k, overlap=o, seed=2024)
    want = o3.ras(g, b, 0.3, sweeps, tile, k, o, shift_mode=1, seed=2024, v=v0)
    assert rel(r.get(), want) <= F64_TOL, rel(r.get(), want)


def test_ras3d_explicit_shifts_and_exact_overlap(api, o3):
    """An explicit shift list gives the oracle's RAS; overlap k - 1 gives
    global Jacobi, bit for bit (one per-point arithmetic in both kernels)."""
    n = (14, 11, 9)
    prob = problem(*n, 13)
    v0 = inputs.random_velocity3d(*n, 14, 0.1)
    g = ogrid(o3, prob)
    b = o3.rhs(g, prob.fx, prob.fy, prob.fz)
    sh = [[1, 2, 0], [3, 0, 2], [0, 1, 1]]
    r = Run3(api, prob, "f64", v0)
    r.smooth(variant="ras", sweeps=6, tile=(4, 3, 3), k=2, overlap=0, shifts=sh)
    want = o3.ras(g, b, 0.3, 6, (4, 3, 3), 2, 0, shift_mode=2, shifts=sh, v=v0)
    assert rel(r.get(), want) <= F64_TOL
    for dtype in ("f64", "f32"):
        a = Run3(api, prob, dtype, v0)
        a.smooth(variant="ras", sweeps=7, tile=(5, 4, 3), k=3, overlap=2, seed=9)
        c = Run3(api, prob, dtype, v0)
        c.smooth(variant="fused", sweeps=7)
        for x, y in zip(a.get(), c.get()):
            assert np.array_equal(x, y), dtype


# tiles whose window (tile + 2 (overlap + 1) per axis) spans 16 to 32 lanes in x
# and fits the column kernel's rows and depth (FP64: 8 rows, 8 levels; FP32:
# 16 rows with 8 levels, 12 with 12), on grids with ragged edge tiles
COL_F64 = [((45, 21, 17), (14, 4, 4), 2, 1), ((37, 9, 13), (28, 2, 2), 3, 1), ((50, 14, 11), (20, 6, 6), 4, 0),
           ((33, 17, 9), (24, 3, 5), 2, 0), ((21, 8, 8), (18, 2, 2), 4, 2)]


@pytest.mark.parametrize("n,tile,k,o", COL_F64)
def test_ras3d_column_kernel_f64(api, o3, n, tile, k, o):
    """RAS on tiles of the column kernel (lane = x, warp = y, the z column in
    registers, each flux formed once) against the oracle: seeded shifts,
    a ragged last pass, and overlaps 0 .. k - 1."""
    prob = problem(*n, 21)
    v0 = inputs.random_velocity3d(*n, 22, 0.1)
    p = inputs.random_pressure3d(*n, 23, 0.2)
    g = ogrid(o3, prob)
    b = o3.rhs(g, prob.fx, prob.fy, prob.fz, p)
    sweeps = 2 * k + 1
    r = Run3(api, prob, "f64", v0, p)
    r.smooth(variant="ras", sweeps=sweeps, tile=tile, k=k, overlap=o, seed=77)
    want = o3.ras(g, b, 0.3, sweeps, tile, k, o, shift_mode=1, seed=77, v=v0)
    assert rel(r.get(), want) <= F64_TOL, rel(r.get(), want)


def test_ras3d_column_kernel_explicit_shifts(api, o3):
    n = (40, 12, 10)
    prob = problem(*n, 24)
    v0 = inputs.random_velocity3d(*n, 25, 0.1)
    g = ogrid(o3, prob)
    b = o3.rhs(g, prob.fx, prob.fy, prob.fz)
    sh = [[0, 0, 0], [13, 3, 5], [27, 1, 2], [5, 5, 1]]
    r = Run3(api, prob, "f64", v0)
    r.smooth(variant="ras", sweeps=8, tile=(28, 6, 6), k=2, overlap=0, shifts=sh)
    want = o3.ras(g, b, 0.3, 8, (28, 6, 6), 2, 0, shift_mode=2, shifts=sh, v=v0)
    assert rel(r.get(), want) <= F64_TOL


@pytest.mark.parametrize("tile,k", [((28, 8, 8), 2), ((28, 4, 4), 2), ((26, 6, 6), 3), ((14, 2, 2), 2),
                                    ((28, 4, 8), 2), ((28, 8, 4), 2), ((28, 12, 4), 2)])
def test_ras3d_column_kernel_exact_overlap_is_jacobi(api, o3, tile, k):
    """Overlap k - 1 on column-kernel tiles equals global fused Jacobi bit for
    bit in FP64 and FP32: every FP32 window shape instantiated (8 levels with
    8, 12 or 16 rows, 12 levels with 8 or 12 rows) and the FP64 one."""
    n = (61, 27, 22)
    prob = problem(*n, 26)
    v0 = inputs.random_velocity3d(*n, 27, 0.1)
    p = inputs.random_pressure3d(*n, 28, 0.2)
    for dtype in ("f64", "f32"):
        h = k
        if dtype == "f64" and (tile[1] + 2 * h > 8 or tile[2] + 2 * h > 8):
            continue
        a = Run3(api, prob, dtype, v0, p)
        a.smooth(variant="ras", sweeps=2 * k + 1, tile=tile, k=k, overlap=k - 1, seed=5)
        c = Run3(api, prob, dtype, v0, p)
        c.smooth(variant="fused", sweeps=2 * k + 1)
        for x, y in zip(a.get(), c.get()):
            assert np.array_equal(x, y), dtype


@pytest.mark.parametrize("tile,k,o", [((30, 10, 10), 4, 0), ((28, 8, 8), 2, 1), ((30, 14, 6), 4, 0)])
def test_ras3d_column_kernel_fp32_energy_error(api, o3, tile, k, o):
    """FP32 column-kernel tiles that FP64 cannot take (12 levels, 16 rows):
    the energy-norm error against the oracle on the FP32-rounded inputs."""
    n = (64, 40, 36)
    prob = inputs.sinker3d_problem(*n, eta_in=1e3)
    g = ogrid(o3, prob, f32)
    b = o3.rhs(g, f32(prob.fx), f32(prob.fy), f32(prob.fz))
    r = Run3(api, prob, "f32")
    r.smooth(variant="ras", sweeps=12, tile=tile, k=k, overlap=o, seed=8)
    want = o3.ras(g, b, 0.3, 12, tile, k, o, shift_mode=1, seed=8)
    got = r.get()
    d = o3.diag_M(g)
    num = sum(np.sum(-dd * (x - y) ** 2) for dd, x, y in zip(d, got, want))
    den = sum(np.sum(-dd * y ** 2) for dd, y in zip(d, want))
    err = float(np.sqrt(num / den))
    print("3d fp32 column %s k%d o%d: energy error %.2e" % (tile, k, o, err))
    assert err <= FP32_ENERGY_TOL


@pytest.mark.parametrize("variant,kw", [("fused", {}), ("ras", dict(tile=(8, 8, 8), k=2, overlap=1)),
                                        ("ras", dict(tile=(8, 8, 4), k=4, overlap=0))])
def test_fp32_energy_error_3d(api, o3, variant, kw):
    n = (24, 24, 24)
    prob = inputs.sinker3d_problem(*n, eta_in=1e3)
    g = ogrid(o3, prob, f32)
    b = o3.rhs(g, f32(prob.fx), f32(prob.fy), f32(prob.fz))
    r = Run3(api, prob, "f32")
    r.smooth(variant=variant, sweeps=20, seed=3, **kw)
    if variant == "fused":
        want = o3.jacobi(g, b, 0.3, 20, g.zeros())
    else:
        want = o3.ras(g, b, 0.3, 20, kw["tile"], kw["k"], kw["overlap"], shift_mode=1, seed=3)
    got = r.get()
    d = o3.diag_M(g)
    num = sum(np.sum(-dd * (x - y) ** 2) for dd, x, y in zip(d, got, want))
    den = sum(np.sum(-dd * y ** 2) for dd, y in zip(d, want))
    err = float(np.sqrt(num / den))
    print("3d fp32 %s %s: energy error %.2e" % (variant, kw, err))
    assert err <= FP32_ENERGY_TOL


def test_smoothers3d_ignore_layout_padding(api, o3):
    """NaN in every padding entry of the caller's velocity changes nothing."""
    import torch
    n = (10, 7, 6)
    prob = problem(*n, 15)
    v0 = inputs.random_velocity3d(*n, 16, 0.1)
    outs = []
    for poison in (False, True):
        r = Run3(api, prob, "f64", v0)
        if poison:
            for t, nm in zip(r.v, ("vx", "vy", "vz")):
                sh = r.ctx.shape[nm]
                mask = torch.ones_like(t, dtype=torch.bool)
                mask[:sh[0], :sh[1], :sh[2]] = False
                t[mask] = float("nan")
        r.smooth(variant="ras", sweeps=5, tile=(4, 4, 3), k=2, overlap=1, seed=1)
        outs.append(r.get())
        r2 = Run3(api, prob, "f64", v0)
        r2.smooth(variant="fused", sweeps=3)
        outs.append(r2.get())
    for x, y in zip(outs[0], outs[2]):
        assert np.array_equal(x, y)
    for x, y in zip(outs[1], outs[3]):
        assert np.array_equal(x, y)


def test_3d_errors(api):
    import torch
    ctx = api.Stokes3DContext(8, 8, 8, dtype="f64")
    v = [ctx.field() for _ in range(3)]
    with pytest.raises(api.StokesError) as e:
        ctx.smooth(*v, variant="fused", sweeps=1)
    assert e.value.status == api.STOKES_ERR_STATE
    ctx.set_problem(inputs.sinker3d_problem(8))
    with pytest.raises(api.StokesError) as e:
        ctx.smooth(*v, variant="rbgs", sweeps=1)
    assert e.value.status == api.STOKES_ERR_ARG
    with pytest.raises(api.StokesError) as e:  # an FP64 window of 16^3 cells x 10 fields does not fit
        ctx.smooth(*v, variant="ras", sweeps=1, tile=(32, 32, 32), k=4, overlap=3)
    assert e.value.status == api.STOKES_ERR_ARG
    with pytest.raises(api.StokesError) as e:
        ctx.smooth(*v, variant="ras", sweeps=2, tile=(4, 4, 4), k=2, shifts=[[4, 0, 0]])
    assert e.value.status == api.STOKES_ERR_ARG
    torch.cuda.synchronize()
    ctx.close()
