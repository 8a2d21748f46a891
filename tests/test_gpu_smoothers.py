"""GPU parity of libstokes against the FP64 oracle, through the C ABI.

FP64: normwise relative error ||v_gpu - v_oracle||_2 / ||v_oracle||_2 <= 1e-12
after every sweep count tested.  FP32: the error of the FP32 result against
the FP64 oracle in the diag(-M)-weighted energy norm, relative to the same
norm of the FP64 result, is below FP32_ENERGY_TOL (derived in the design
notes: each sweep adds a few units of FP32 roundoff relative to |v|).
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


def energy_rel(g, a, b):
    """sqrt(sum (-d) (a-b)^2 / sum (-d) b^2) over the unknowns."""
    dx, dy = ora.diag_M(g)
    num = np.sum(-dx * (a[0] - b[0]) ** 2) + np.sum(-dy * (a[1] - b[1]) ** 2)
    den = np.sum(-dx * b[0] ** 2) + np.sum(-dy * b[1] ** 2)
    return float(np.sqrt(num / den))


def rand_problem(nx, ny, seed, lx=1.3, ly=0.9):
    prob = inputs.sinker_problem(nx, ny, lx=lx, ly=ly, eta_in=1e3)
    ec, en = inputs.random_viscosity(nx, ny, seed, (-2.0, 2.0))
    prob.eta_c, prob.eta_n = ec, en
    return prob


class Run:
    """A context holding one problem and a velocity state on the GPU."""

    def __init__(self, api, prob, dtype, v0=None, p=None):
        self.api, self.prob = api, prob
        self.ctx = api.StokesContext(prob.nx, prob.ny, prob.lx, prob.ly, dtype)
        self.ctx.set_problem(prob)
        if v0 is None:
            v0 = (np.zeros((prob.ny, prob.nx + 1)), np.zeros((prob.ny + 1, prob.nx)))
        self.vx, self.vy = self.ctx.pack(v0[0], "vx"), self.ctx.pack(v0[1], "vy")
        self.p = None if p is None else self.ctx.pack(p, "p")

    def smooth(self, **kw):
        self.ctx.smooth(self.vx, self.vy, self.p, **kw)

    def v(self):
        import torch
        torch.cuda.synchronize()
        return self.ctx.unpack(self.vx, "vx"), self.ctx.unpack(self.vy, "vy")


# ---------------------------------------------------------------------------
# operator and energy norm
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny", [(61, 47), (2, 2), (3, 5), (130, 33)])
def test_apply_operator_f64(api, nx, ny):
    prob = rand_problem(nx, ny, 1)
    vx, vy = inputs.random_velocity(nx, ny, 2)
    p = inputs.random_pressure(nx, ny, 3)
    r = Run(api, prob, "f64", (vx, vy), p)
    ox, oy = r.ctx.apply(r.vx, r.vy, r.p)
    g = ogrid(prob)
    mx, my = ora.apply_M(g, vx, vy)
    gx, gy = ora.apply_G(g, p)
    want = (mx + gx, my + gy)
    got = (r.ctx.unpack(ox, "vx"), r.ctx.unpack(oy, "vy"))
    assert rel(got, want) <= F64_TOL
    # walls and padding of the output are zero
    assert np.all(got[0][:, 0] == 0) and np.all(got[0][:, nx] == 0)
    ox_h, oy_h = ox.cpu().numpy(), oy.cpu().numpy()
    assert np.all(ox_h[ny, :] == 0) and np.all(ox_h[:, nx + 1:] == 0)
    assert np.all(oy_h[:, nx:] == 0)


@pytest.mark.parametrize("with_p", [False, True])
def test_energy_norm_f64(api, with_p):
    nx, ny = 77, 53
    prob = rand_problem(nx, ny, 4)
    vx, vy = inputs.random_velocity(nx, ny, 5, 1e-3)
    p = inputs.random_pressure(nx, ny, 6) if with_p else None
    r = Run(api, prob, "f64", (vx, vy), p)
    got = r.ctx.energy(r.vx, r.vy, r.p)
    want = ora.energy(ogrid(prob), prob.fx, prob.fy, p, vx, vy)
    for a, b in zip(got, want):
        assert abs(a - b) <= F64_TOL * abs(b)
    again = r.ctx.energy(r.vx, r.vy, r.p)
    assert again == got  # fixed summation order


@pytest.mark.parametrize("with_p", [False, True])
def test_energy_norm_f32(api, with_p):
    """FP32 context: each term is formed in FP32 and summed in FP64.  Against
    the oracle on the FP32-rounded inputs the sums agree to the FP32
    rounding of the residual and the coefficients (1e-5 relative)."""
    nx, ny = 77, 53
    prob = rand_problem(nx, ny, 4)
    vx, vy = inputs.random_velocity(nx, ny, 5, 1e-3)
    p = inputs.random_pressure(nx, ny, 6) if with_p else None
    r = Run(api, prob, "f32", (vx, vy), p)
    got = r.ctx.energy(r.vx, r.vy, r.p)
    f32 = lambda a: None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)
    g32 = ora.Grid(nx, ny, prob.hx, prob.hy, f32(prob.eta_c), f32(prob.eta_n))
    want = ora.energy(g32, f32(prob.fx), f32(prob.fy), f32(p), f32(vx), f32(vy))
    for a, b in zip(got, want):
        assert abs(a - b) <= 1e-5 * abs(b), (a, b)
    assert r.ctx.energy(r.vx, r.vy, r.p) == got


@pytest.mark.parametrize("n,l,with_p", [((1000, 1000), (1.0, 1.0), False), ((1000, 1000), (1.0, 1.0), True),
                                        ((513, 301), (1.3, 0.9), True)])
def test_energy_norm_f32_many_strips(api, n, l, with_p):
    """The FP32 energy sums on grids of many column strips and row bands, on
    square cells (the square-cell shear form) and on hx != hy, with and
    without pressure: against the oracle on the FP32-rounded inputs (1e-5
    relative) and repeatable bit for bit."""
    nx, ny = n
    prob = rand_problem(nx, ny, 7, lx=l[0], ly=l[1])
    vx, vy = inputs.random_velocity(nx, ny, 8, 1e-3)
    p = inputs.random_pressure(nx, ny, 9) if with_p else None
    r = Run(api, prob, "f32", (vx, vy), p)
    got = r.ctx.energy(r.vx, r.vy, r.p)
    f32 = lambda a: None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)
    g32 = ora.Grid(nx, ny, prob.hx, prob.hy, f32(prob.eta_c), f32(prob.eta_n))
    want = ora.energy(g32, f32(prob.fx), f32(prob.fy), f32(p), f32(vx), f32(vy))
    for a, b in zip(got, want):
        assert abs(a - b) <= 1e-5 * abs(b), (a, b)
    assert r.ctx.energy(r.vx, r.vy, r.p) == got


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_entry_points_reject_buffers_off_16_byte_boundaries(api, dtype):
    """The kernels read rows as 16-byte vectors and stage windows by tensor
    copies, so a velocity or pressure buffer that does not start on a
    16-byte boundary is refused (STOKES_ERR_ARG) before any kernel runs."""
    prob = inputs.sinker_problem(64)
    r = Run(api, prob, dtype)
    off = r.vx.view(-1)[1:]  # one element past the allocation's start
    for call in (lambda: r.ctx.smooth(off, r.vy, None, variant="fused", sweeps=1),
                 lambda: r.ctx.smooth(r.vx, r.vy, off, variant="ras", sweeps=2, tile=(16, 16), k=2, overlap=1),
                 lambda: r.ctx.energy(r.vx, off),
                 lambda: r.ctx.energy(r.vx, r.vy, off),
                 lambda: r.ctx.vcycle(off, r.vy, None, variant="fused", max_cycles=1)):
        with pytest.raises(api.StokesError) as e:
            call()
        assert e.value.status == api.STOKES_ERR_ARG
    rv, rp, ff = r.ctx.energy(r.vx, r.vy)  # the context stays usable
    assert rp == 0.0 and ff > 0.0


def test_energy_norm_is_one_at_zero_state(api):
    prob = inputs.sinker_problem(64)
    r = Run(api, prob, "f64")
    rv, rp, ff = r.ctx.energy(r.vx, r.vy)
    assert rp == 0.0 and abs(rv - ff) <= 1e-14 * ff


# ---------------------------------------------------------------------------
# the sinker smoothing case: 64^2, contrast 1e3, 10 sweeps, parity every sweep
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("variant", ["jacobi", "fused", "blocked", "rbgs"])
def test_sinker_64_every_sweep_f64(api, variant):
    prob = inputs.sinker_problem(64, eta_in=1e3, eta_out=1.0, rho_in=2.0, rho_out=1.0, radius=0.1)
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    r = Run(api, prob, "f64")
    ref = (g.zeros_vx(), g.zeros_vy())
    for s in range(10):
        r.smooth(variant=variant, sweeps=1, tile=(16, 8))
        if variant == "rbgs":
            ref = ora.rbgs(g, bx, by, 0.3, 1, *ref)
        else:
            ref = ora.jacobi(g, bx, by, 0.3, 1, *ref)
        assert rel(r.v(), ref) <= F64_TOL, "sweep %d" % (s + 1)


def test_sinker_64_ras_every_sweep_f64(api):
    """8x8 tiles, k = 2, overlap 1, SplitMix64 shifts with seed 1: one call per
    sweep count 1..10 from the zero state (odd counts end on a partial outer
    iteration)."""
    prob = inputs.sinker_problem(64, eta_in=1e3, eta_out=1.0, rho_in=2.0, rho_out=1.0, radius=0.1)
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    for n in range(1, 11):
        r = Run(api, prob, "f64")
        r.smooth(variant="ras", sweeps=n, tile=(8, 8), k=2, overlap=1, seed=1)
        ref = ora.ras(g, bx, by, 0.3, n, 8, 8, 2, 1, shift_mode=1, seed=1)
        assert rel(r.v(), ref) <= F64_TOL, "sweeps %d" % n


# ---------------------------------------------------------------------------
# the 1024^2 sinker at contrast 1e4 in FP64, 100 sweeps per smoother: the
# benchmark's smoother table (every smoother, RAS tiles of 16^2 to 64 x 32)
# against the oracle on the whole field
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kw", [
    dict(variant="jacobi"), dict(variant="fused"), dict(variant="rbgs"),
    dict(variant="blocked", tile=(32, 32)),
    dict(variant="ras", tile=(32, 32), k=2, overlap=1),
    dict(variant="ras", tile=(16, 16), k=4, overlap=3),
    dict(variant="ras", tile=(64, 32), k=4, overlap=3),
])
def test_sinker_1024_contrast1e4_100_sweeps_f64(api, kw):
    n, sweeps = 1024, 100
    prob = inputs.sinker_problem(n, eta_in=1e4)
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    r = Run(api, prob, "f64")
    r.smooth(sweeps=sweeps, seed=1, **kw)
    if kw["variant"] == "ras":
        ref = ora.ras(g, bx, by, 0.3, sweeps, kw["tile"][0], kw["tile"][1], kw["k"], kw["overlap"], shift_mode=1,
                      seed=1)
    else:
        fn = ora.rbgs if kw["variant"] == "rbgs" else ora.jacobi
        ref = fn(g, bx, by, 0.3, sweeps, g.zeros_vx(), g.zeros_vy())
    assert rel(r.v(), ref) <= F64_TOL


# ---------------------------------------------------------------------------
# ragged grids, several tiles, hx != hy, non-zero pressure
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("variant", ["jacobi", "fused", "blocked", "rbgs"])
def test_ragged_f64(api, variant):
    nx, ny = 97, 61
    prob = rand_problem(nx, ny, 7)
    v0 = inputs.random_velocity(nx, ny, 8, 0.1)
    p = inputs.random_pressure(nx, ny, 9)
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, p)
    r = Run(api, prob, "f64", v0, p)
    r.smooth(variant=variant, sweeps=7, tile=(32, 16), omega=0.25)
    fn = ora.rbgs if variant == "rbgs" else ora.jacobi
    ref = fn(g, bx, by, 0.25, 7, *v0)
    assert rel(r.v(), ref) <= F64_TOL


@pytest.mark.parametrize("tile,k,o", [((16, 12), 1, 0), ((16, 12), 3, 0), ((16, 12), 3, 1), ((16, 12), 3, 2),
                                      ((7, 9), 2, 0), ((7, 9), 4, 3), ((5, 5), 3, 6), ((128, 20), 4, 0), ((60, 40), 2, 1)])
def test_ras_ragged_f64(api, tile, k, o):
    nx, ny = 100, 75
    prob = rand_problem(nx, ny, 10)
    v0 = inputs.random_velocity(nx, ny, 11, 0.1)
    p = inputs.random_pressure(nx, ny, 12)
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, p)
    r = Run(api, prob, "f64", v0, p)
    r.smooth(variant="ras", sweeps=7, tile=tile, k=k, overlap=o, seed=2024)
    ref = ora.ras(g, bx, by, 0.3, 7, tile[0], tile[1], k, o, shift_mode=1, seed=2024, vx=v0[0], vy=v0[1])
    assert rel(r.v(), ref) <= F64_TOL


def test_ras_explicit_shift_list_f64(api):
    nx, ny = 90, 70
    prob = rand_problem(nx, ny, 13)
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    shifts = inputs.random_shifts(4, 12, 10, 99)
    r = Run(api, prob, "f64")
    r.smooth(variant="ras", sweeps=8, tile=(12, 10), k=2, overlap=0, shifts=shifts)
    ref = ora.ras(g, bx, by, 0.3, 8, 12, 10, 2, 0, shift_mode=2, shifts=shifts)
    assert rel(r.v(), ref) <= F64_TOL


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_ras_exact_overlap_is_bitwise_jacobi(api, dtype):
    """o >= k-1 reproduces global Jacobi; the tiled and the global kernels round
    identically, so the fields agree bit for bit."""
    nx, ny = 150, 110
    prob = inputs.sinker_problem(nx, ny, eta_in=1e4)
    a = Run(api, prob, dtype)
    b = Run(api, prob, dtype)
    a.smooth(variant="ras", sweeps=12, tile=(32, 24), k=4, overlap=3, seed=5)
    b.smooth(variant="fused", sweeps=12)
    va, vb = a.v(), b.v()
    assert np.array_equal(va[0], vb[0]) and np.array_equal(va[1], vb[1])


def test_run_twice_bitwise(api):
    prob = inputs.sinker_problem(200, 150, eta_in=1e4)
    outs = []
    for _ in range(2):
        r = Run(api, prob, "f32")
        r.smooth(variant="ras", sweeps=9, tile=(32, 32), k=4, overlap=0, seed=3)
        outs.append(r.v())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


# ---------------------------------------------------------------------------
# FP32 against the FP64 oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("variant,kw", [("jacobi", {}), ("fused", {}), ("blocked", {}), ("rbgs", {}),
                                        ("ras", dict(tile=(32, 32), k=4, overlap=0)),
                                        ("ras", dict(tile=(32, 32), k=4, overlap=3))])
def test_fp32_energy_error(api, variant, kw):
    n = 192
    prob = inputs.sinker_problem(n, eta_in=1e4)
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    r = Run(api, prob, "f32")
    r.smooth(variant=variant, sweeps=100, seed=7, **kw)
    if variant == "rbgs":
        ref = ora.rbgs(g, bx, by, 0.3, 100, g.zeros_vx(), g.zeros_vy())
    elif variant == "ras":
        ref = ora.ras(g, bx, by, 0.3, 100, 32, 32, 4, kw["overlap"], shift_mode=1, seed=7)
    else:
        ref = ora.jacobi(g, bx, by, 0.3, 100, g.zeros_vx(), g.zeros_vy())
    err = energy_rel(g, r.v(), ref)
    print("fp32 %s %s: relative energy error %.3e" % (variant, kw, err))
    assert err <= FP32_ENERGY_TOL


# ---------------------------------------------------------------------------
# edge cases and errors
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny", [(2, 2), (2, 3), (3, 2), (5, 4)])
def test_tiny_grids_all_variants(api, nx, ny):
    prob = rand_problem(nx, ny, 20, 1.0, 1.0)
    v0 = inputs.random_velocity(nx, ny, 21)
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    for variant in ("jacobi", "fused", "blocked", "rbgs", "ras"):
        r = Run(api, prob, "f64", v0)
        r.smooth(variant=variant, sweeps=3, tile=(2, 2), k=2, overlap=0, seed=1)
        if variant == "rbgs":
            ref = ora.rbgs(g, bx, by, 0.3, 3, *v0)
        elif variant == "ras":
            ref = ora.ras(g, bx, by, 0.3, 3, 2, 2, 2, 0, shift_mode=1, seed=1, vx=v0[0], vy=v0[1])
        else:
            ref = ora.jacobi(g, bx, by, 0.3, 3, *v0)
        assert rel(r.v(), ref) <= F64_TOL, variant


def test_zero_sweeps_is_identity_and_walls_kept(api):
    nx, ny = 40, 30
    prob = rand_problem(nx, ny, 22)
    vx, vy = inputs.random_velocity(nx, ny, 23)
    vx[:, 0] = 0.5  # Dirichlet wall data is read, never written
    r = Run(api, prob, "f64", (vx, vy))
    r.smooth(variant="ras", sweeps=0, k=4)
    got = r.v()
    assert np.array_equal(got[0], vx) and np.array_equal(got[1], vy)
    r.smooth(variant="ras", sweeps=5, tile=(8, 8), k=2, overlap=1, seed=4)
    got = r.v()
    assert np.all(got[0][:, 0] == 0.5) and np.all(got[0][:, nx] == 0.0)
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    ref = ora.ras(g, bx, by, 0.3, 5, 8, 8, 2, 1, shift_mode=1, seed=4, vx=vx, vy=vy)
    assert rel(got, ref) <= F64_TOL


def test_argument_and_state_errors(api):
    import torch
    ctx = api.StokesContext(32, 32, 1.0, 1.0, "f64")
    vx, vy = ctx.field(), ctx.field()
    with pytest.raises(api.StokesError) as e:
        ctx.smooth(vx, vy, variant="fused", sweeps=1)
    assert e.value.status == api.STOKES_ERR_STATE
    ctx.set_problem(inputs.sinker_problem(32))
    with pytest.raises(api.StokesError) as e:
        ctx.smooth(vx, vy, variant="ras", sweeps=4, tile=(32, 32), k=4, overlap=100)
    assert e.value.status == api.STOKES_ERR_ARG
    with pytest.raises(api.StokesError) as e:
        ctx.smooth(vx, vy, variant="ras", sweeps=4, tile=(8, 8), k=2, shifts=[[9, 0], [0, 0]])
    assert e.value.status == api.STOKES_ERR_ARG
    with pytest.raises(api.StokesError) as e:
        ctx.smooth(vx, vy, variant="ras", sweeps=4, k=0)
    assert e.value.status == api.STOKES_ERR_ARG
    torch.cuda.synchronize()
    ctx.close()


# ---------------------------------------------------------------------------
# full size: 8192^2 layered sinker (contrast 1e6), the benchmark's launch
# configuration; sampled tiles of one outer iteration against the oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype,tile,k,o", [("f32", (48, 64), 8, 7),   # the benchmark's schedule
                                            ("f32", (62, 56), 8, 0),   # ring-only tiles, pair kernel
                                            ("f32", (32, 32), 4, 3), ("f64", (32, 32), 4, 3),
                                            ("f32", (32, 32), 4, 0)])
def test_full_size_sampled_tiles(api, dtype, tile, k, o):
    n = 8192
    prob = inputs.layered_sinker(n, seed=4)
    v0 = inputs.random_velocity(n, n, 31, 1e-3)
    si, sj = 13, 27
    r = Run(api, prob, dtype, v0)
    r.smooth(variant="ras", sweeps=k, tile=tile, k=k, overlap=o, shifts=[[si, sj]])
    got = r.v()
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    ntx, nty = ora.tile_count(n, tile[0], si), ora.tile_count(n, tile[1], sj)
    rng = np.random.default_rng(5)
    tiles = [(0, 0), (ntx - 1, nty - 1), (0, nty - 1), (ntx - 1, 0)]
    tiles += [(int(a), int(b)) for a, b in zip(rng.integers(0, ntx, 12), rng.integers(0, nty, 12))]
    ref = ora.ras_tiles(g, bx, by, 0.3, tile[0], tile[1], k, o, si, sj, tiles, v0[0], v0[1], v0[0], v0[1])
    # compare the unknowns owned by the sampled tiles' cells
    cuts_x = [0] + [c for c in range(si, n, tile[0]) if c > 0] + [n]
    cuts_y = [0] + [c for c in range(sj, n, tile[1]) if c > 0] + [n]
    for (a, b) in tiles:
        x0, x1, y0, y1 = cuts_x[a], cuts_x[a + 1], cuts_y[b], cuts_y[b + 1]
        gx = (got[0][y0:y1, x0:x1], got[1][y0:y1, x0:x1])
        rx = (ref[0][y0:y1, x0:x1], ref[1][y0:y1, x0:x1])
        if dtype == "f64":
            assert rel(gx, rx) <= F64_TOL, (a, b)
        else:
            assert rel(gx, rx) <= FP32_ENERGY_TOL, (a, b)


# ---------------------------------------------------------------------------
# the benchmark's whole launch sequence on the whole field: the layered
# sinker (contrast 1e6, seed 4) at 1024^2, 100 sweeps from zero in one call,
# exactly as one benchmark step runs them (13 or 25 tile launches: the odd
# pass count routes the intermediate passes through the second scratch pair;
# the last launch runs the remainder sweeps), then the energy sums
# ---------------------------------------------------------------------------
def _f32(a):
    return None if a is None else np.asarray(a, dtype=np.float32).astype(np.float64)


def energy_sums_fsum(g, fx, fy, vx, vy):
    """The oracle's velocity energy sums (Sec. 6.4) with every term from the
    oracle's residual and diagonal, added with an exactly rounded sum
    (math.fsum): over a million terms spanning six orders of magnitude the
    oracle's own left-to-right loop carries a rounding error of order
    N u = 1e-10, which would hide a 1e-12 comparison."""
    import math
    bx, by = ora.rhs(g, fx, fy, None)
    mx, my = ora.apply_M(g, vx, vy)
    dx, dy = ora.diag_M(g)
    nx, ny = g.nx, g.ny
    rx, ry = (bx - mx)[:, 1:nx], (by - my)[1:ny, :]
    wx, wy = -dx[:, 1:nx], -dy[1:ny, :]
    fxu, fyu = np.asarray(fx)[:, 1:nx], np.asarray(fy)[1:ny, :]
    rv = math.fsum((rx * rx / wx).ravel()) + math.fsum((ry * ry / wy).ravel())
    ff = math.fsum((fxu * fxu / wx).ravel()) + math.fsum((fyu * fyu / wy).ravel())
    return rv, ff


@pytest.mark.parametrize("dtype,tile,k,o,kernel", [
    ("f32", (48, 64), 8, 7, "pair"),    # the benchmark's schedule (square-cell pair form, 512 threads)
    ("f32", (62, 56), 8, 0, "pair"),    # ring-only tiles, pair layout
    ("f32", (32, 32), 4, 3, "tma"),     # one-column layout, 25 passes
    ("f64", (32, 32), 4, 3, "tma"),     # FP64, 25 passes
    ("f64", (32, 32), 8, 0, "tma"),     # FP64, ring-only, 13 passes
])
def test_benchmark_sequence_whole_field(api, dtype, tile, k, o, kernel):
    n, sweeps, seed = 1024, 100, 1
    assert api.stokes_tile_kernel_plan(n, n, tile, o, dtype)[0] == kernel
    prob = inputs.layered_sinker(n, seed=4)
    r = Run(api, prob, dtype)
    r.smooth(variant="ras", sweeps=sweeps, tile=tile, k=k, overlap=o, seed=seed)
    got = r.v()
    e = r.ctx.energy(r.vx, r.vy)
    cast = _f32 if dtype == "f32" else (lambda a: a)
    g = ora.Grid(n, n, prob.hx, prob.hy, cast(prob.eta_c), cast(prob.eta_n))
    bx, by = ora.rhs(g, cast(prob.fx), cast(prob.fy), None)
    ref = ora.ras(g, bx, by, 0.3, sweeps, tile[0], tile[1], k, o, shift_mode=1, seed=seed)
    rv, ff = energy_sums_fsum(g, cast(prob.fx), cast(prob.fy), got[0], got[1])
    want = (rv, ora.energy(g, cast(prob.fx), cast(prob.fy), None, got[0], got[1])[1], ff)
    if dtype == "f64":
        assert rel(got, ref) <= F64_TOL, rel(got, ref)
        for a, b in zip(e, want):
            assert abs(a - b) <= F64_TOL * abs(b), (e, want)
    else:
        err = energy_rel(g, got, ref)
        emax = max(float(np.max(np.abs(x - y))) for x, y in zip(got, ref)) / max(float(np.max(np.abs(y)))
                                                                                 for y in ref)
        print("fp32 %s k=%d o=%d: energy error %.2e, max element error %.2e (of max |v|)" % (tile, k, o, err, emax))
        assert err <= FP32_ENERGY_TOL
        assert emax <= 10 * FP32_ENERGY_TOL
        # the FP32 energy sums of the same state (terms in FP32, sums in FP64)
        for a, b in zip(e, want):
            assert abs(a - b) <= FP32_ENERGY_TOL * abs(b), (e, want)


# ---------------------------------------------------------------------------
# the three tile-kernel paths give the same bits; failure detection
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("tile,k,o", [((32, 32), 4, 3), ((32, 32), 4, 0), ((24, 16), 3, 1), ((40, 40), 1, 0),
                                      ((13, 7), 2, 5)])
def test_tma_and_global_staging_agree(api, dtype, tile, k, o):
    nx, ny = 301, 207
    prob = rand_problem(nx, ny, 40)
    v0 = inputs.random_velocity(nx, ny, 41, 0.1)
    outs = []
    for use_tma in (1, 0):
        r = Run(api, prob, dtype, v0)
        r.ctx.set_option(api.STOKES_OPT_USE_TMA, use_tma)
        r.smooth(variant="ras", sweeps=9, tile=tile, k=k, overlap=o, seed=77)
        outs.append(r.v())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    if dtype == "f64":
        g = ogrid(prob)
        bx, by = ora.rhs(g, prob.fx, prob.fy, None)
        ref = ora.ras(g, bx, by, 0.3, 9, tile[0], tile[1], k, o, shift_mode=1, seed=77, vx=v0[0], vy=v0[1])
        assert rel(outs[0], ref) <= F64_TOL


def test_staging_wait_timeout_is_reported_and_context_recovers(api):
    """A staged-window wait that gives up records STOKES_ERR_TIMEOUT on the
    device (after letting its copy land); the host reads it at the next check
    and the context keeps working."""
    nx, ny = 128, 96
    prob = rand_problem(nx, ny, 42)
    g = ogrid(prob)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    r = Run(api, prob, "f64")
    r.ctx.set_option(api.STOKES_OPT_WAIT_LIMIT_CYCLES, -1)
    r.smooth(variant="ras", sweeps=4, tile=(32, 32), k=4, overlap=3, seed=1)
    with pytest.raises(api.StokesError) as e:
        r.ctx.synchronize()
    assert e.value.status == api.STOKES_ERR_TIMEOUT
    r.ctx.synchronize()  # cleared
    r.ctx.set_option(api.STOKES_OPT_WAIT_LIMIT_CYCLES, 2_000_000_000)
    r2 = Run(api, prob, "f64")
    r2.smooth(variant="ras", sweeps=4, tile=(32, 32), k=4, overlap=3, seed=1)
    ref = ora.ras(g, bx, by, 0.3, 4, 32, 32, 4, 3, shift_mode=1, seed=1)
    assert rel(r2.v(), ref) <= F64_TOL
    r.smooth(variant="ras", sweeps=4, tile=(32, 32), k=4, overlap=3, seed=1)
    r.ctx.synchronize()


# ---------------------------------------------------------------------------
# the packed-pair FP32 kernel (two columns per thread) gives the bits of the
# one-column-per-thread kernel
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny,tile,k,o", [
    (301, 207, (56, 32), 4, 3),   # 64-column window, the benchmark's shape
    (301, 207, (32, 32), 4, 3),   # 40-column window: idle lanes
    (301, 207, (60, 20), 2, 1),
    (301, 207, (62, 64), 1, 0),   # 66 window rows: 17 strips
    (301, 207, (48, 40), 8, 7),
    (301, 207, (48, 64), 8, 7),   # 80 window rows: 20 strips, the largest CTA
    (301, 207, (13, 7), 2, 5),
    (70, 45, (56, 32), 4, 0),     # ragged last tiles, overlap 0
    (5, 3, (56, 32), 3, 2),       # grid smaller than the tile
    (2, 2, (8, 8), 2, 1),
])
def test_pair_kernel_matches_the_column_kernel(api, nx, ny, tile, k, o):
    """Mode 2 sends every window of at most 64 columns to the pair kernel;
    its fields equal those of the one-column kernel (and, for o >= k - 1, of
    global fused Jacobi) value for value."""
    name, threads, smem = api.stokes_tile_kernel_plan(nx, ny, tile, o, "f32", pair_mode=2)
    assert name == "pair", (name, threads)
    assert api.stokes_tile_kernel_plan(nx, ny, tile, o, "f32", pair_mode=0)[0] != "pair"
    prob = rand_problem(nx, ny, 43)
    v0 = inputs.random_velocity(nx, ny, 44, 0.1)
    outs = []
    for pair in (2, 0):
        r = Run(api, prob, "f32", v0)
        r.ctx.set_option(api.STOKES_OPT_PAIRED, pair)
        r.smooth(variant="ras", sweeps=9, tile=tile, k=k, overlap=o, seed=78)
        outs.append(r.v())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    if o >= k - 1:
        r = Run(api, prob, "f32", v0)
        r.smooth(variant="fused", sweeps=9)
        jac = r.v()
        assert np.array_equal(outs[0][0], jac[0]) and np.array_equal(outs[0][1], jac[1])


@pytest.mark.parametrize("tile,k,o", [((48, 64), 8, 7), ((56, 32), 4, 3), ((62, 56), 8, 0), ((48, 32), 3, 2)])
def test_pair_kernel_square_cells(api, tile, k, o):
    """Square cells (hx = hy bit for bit: 300 x 200 cells on 1.5 x 1.0) take
    the pair kernel's square-cell form, which keeps one coefficient for Txx
    and Tyy and one scaled shear; its fields equal those of the one-column
    kernel value for value, and those of global fused Jacobi for o >= k - 1."""
    nx, ny = 300, 200
    prob = rand_problem(nx, ny, 47, lx=1.5, ly=1.0)
    assert prob.lx / nx == prob.ly / ny
    v0 = inputs.random_velocity(nx, ny, 48, 0.1)
    outs = []
    for pair in (1, 0):
        r = Run(api, prob, "f32", v0)
        r.ctx.set_option(api.STOKES_OPT_PAIRED, pair)
        r.smooth(variant="ras", sweeps=11, tile=tile, k=k, overlap=o, seed=79)
        outs.append(r.v())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    if o >= k - 1:
        r = Run(api, prob, "f32", v0)
        r.smooth(variant="fused", sweeps=11)
        jac = r.v()
        assert np.array_equal(outs[0][0], jac[0]) and np.array_equal(outs[0][1], jac[1])


def test_pair_kernel_selection(api):
    plan = api.stokes_tile_kernel_plan
    assert plan(1024, 1024, (56, 32), 3, "f32")[0] == "pair"       # 64-column window: default mode
    assert plan(1024, 1024, (62, 32), 0, "f32")[0] == "pair"
    assert plan(1024, 1024, (40, 32), 3, "f32")[0] != "pair"       # 48 columns: one-column kernel
    assert plan(1024, 1024, (40, 32), 3, "f32", pair_mode=2)[0] == "pair"
    assert plan(1024, 1024, (64, 32), 3, "f32", pair_mode=2)[0] != "pair"  # 72 columns
    assert plan(1024, 1024, (56, 32), 3, "f64")[0] != "pair"
    assert plan(1024, 1024, (56, 32), 3, "f32", use_tma=False)[0] != "pair"
    with pytest.raises(api.StokesError):
        plan(1024, 1024, (56, 32), 3, "f32", pair_mode=3)
    ctx = api.StokesContext(16, 16, 1.0, 1.0, "f32")
    with pytest.raises(api.StokesError):
        ctx.set_option(api.STOKES_OPT_PAIRED, 5)
    ctx.close()


def test_pair_kernel_wait_timeout_is_reported(api):
    nx, ny = 128, 96
    prob = rand_problem(nx, ny, 45)
    r = Run(api, prob, "f32")
    r.ctx.set_option(api.STOKES_OPT_WAIT_LIMIT_CYCLES, -1)
    r.smooth(variant="ras", sweeps=4, tile=(56, 32), k=4, overlap=3, seed=1)
    with pytest.raises(api.StokesError) as e:
        r.ctx.synchronize()
    assert e.value.status == api.STOKES_ERR_TIMEOUT
    r.ctx.set_option(api.STOKES_OPT_WAIT_LIMIT_CYCLES, 2_000_000_000)
    r.smooth(variant="ras", sweeps=4, tile=(56, 32), k=4, overlap=3, seed=1)
    r.ctx.synchronize()


# ---------------------------------------------------------------------------
# padding canaries: no smoother reads or writes the layout's padding
# ---------------------------------------------------------------------------
def _with_canaries(api, ctx, t, name):
    """Copy of a packed field with NaN in every padding entry of the layout."""
    import torch
    r, c = ctx.shape[name]
    out = t.clone()
    out[r:, :] = float("nan")
    out[:, c:] = float("nan")
    return out


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("kw", [
    dict(variant="jacobi", sweeps=3), dict(variant="fused", sweeps=3), dict(variant="rbgs", sweeps=2),
    dict(variant="blocked", sweeps=2, tile=(24, 16)),
    dict(variant="ras", sweeps=6, tile=(56, 32), k=4, overlap=3, seed=3),
    dict(variant="ras", sweeps=6, tile=(62, 32), k=2, overlap=0, seed=4),
    dict(variant="ras", sweeps=6, tile=(16, 8), k=3, overlap=1, seed=5),
    dict(variant="ras", sweeps=4, tile=(72, 40), k=2, overlap=1, seed=6),
])
def test_smoothers_ignore_layout_padding(api, dtype, kw):
    """NaN in every padding entry of vx and vy (rows and columns beyond each
    field's extent) changes no unknown and is not overwritten."""
    import torch
    nx, ny = 150, 97
    prob = rand_problem(nx, ny, 46)
    v0 = inputs.random_velocity(nx, ny, 47, 0.1)
    a = Run(api, prob, dtype, v0)
    a.smooth(**kw)
    want = a.v()
    b = Run(api, prob, dtype, v0)
    b.vx = _with_canaries(api, b.ctx, b.vx, "vx")
    b.vy = _with_canaries(api, b.ctx, b.vy, "vy")
    b.smooth(**kw)
    got = b.v()
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    torch.cuda.synchronize()
    for t, name in ((b.vx, "vx"), (b.vy, "vy")):
        r, c = b.ctx.shape[name]
        h = t.double().cpu().numpy()
        assert np.isnan(h[r:, :]).all() and np.isnan(h[:, c:]).all(), name
