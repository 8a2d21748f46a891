"""Pins of the 3D FP64 oracle (the 3D extension the paper names as future
work, Sec. 9) against facts that do not come from itself: the continuum
operator on manufactured polynomials, symmetry and definiteness, the
operator's diagonal read off by unit-vector applies, the reduction of a
z-invariant field to the (separately pinned) 2D oracle, and the RAS
identities of Algorithm 2.  No GPU is needed."""
import numpy as np
import pytest

from paper_2509_19061_gb300 import inputs


@pytest.fixture(scope="module")
def o3(ora):
    from oracle import oracle3d
    oracle3d.lib()
    return oracle3d


def rand_grid3(o3, nx, ny, nz, seed, lx=1.0, ly=1.0, lz=1.0, rng=(-2.0, 2.0)):
    ec, exy, exz, eyz = inputs.random_viscosity3d(nx, ny, nz, seed, rng)
    return o3.Grid3(nx, ny, nz, lx / nx, ly / ny, lz / nz, ec, exy, exz, eyz)


def masks3(nx, ny, nz):
    mx = np.zeros((nz, ny, nx + 1), bool)
    mx[:, :, 1:nx] = True
    my = np.zeros((nz, ny + 1, nx), bool)
    my[:, 1:ny, :] = True
    mz = np.zeros((nz + 1, ny, nx), bool)
    mz[1:nz] = True
    return mx, my, mz


def dot3(a, b, m):
    return sum(float(np.sum(x[mm] * y[mm])) for x, y, mm in zip(a, b, m))


# --------------------------------------------------------------------------
# operator
# --------------------------------------------------------------------------
def test_operator_manufactured_polynomial_3d(o3):
    """Affine viscosity and quadratic velocity: the staggered central
    differences are exact, so M v equals div(eta (grad v + grad v^T)) at every
    unknown whose stencil touches no wall edge (Eq. (1)-(3) in 3D, unequal
    spacings)."""
    nx, ny, nz, lx, ly, lz = 9, 8, 7, 1.3, 0.7, 1.1
    hx, hy, hz = lx / nx, ly / ny, lz / nz
    e0, ex, ey, ez = 2.0, 0.7, -0.4, 0.3
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, size=(3, 10))  # v_c = A[c] . [1, x, y, z, x^2, y^2, z^2, xy, xz, yz]

    def q(c, x, y, z):
        a = A[c]
        return (a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * x + a[5] * y * y + a[6] * z * z + a[7] * x * y
                + a[8] * x * z + a[9] * y * z)

    def grad(c, x, y, z):
        a = A[c]
        return (a[1] + 2 * a[4] * x + a[7] * y + a[8] * z, a[2] + 2 * a[5] * y + a[7] * x + a[9] * z,
                a[3] + 2 * a[6] * z + a[8] * x + a[9] * y)

    def hess(c):
        a = A[c]
        return np.array([[2 * a[4], a[7], a[8]], [a[7], 2 * a[5], a[9]], [a[8], a[9], 2 * a[6]]])

    eta = lambda x, y, z: e0 + ex * x + ey * y + ez * z
    deta = (ex, ey, ez)
    xc, yc, zc = [(np.arange(n) + 0.5) * h for n, h in ((nx, hx), (ny, hy), (nz, hz))]
    xn, yn, zn = [np.arange(n + 1) * h for n, h in ((nx, hx), (ny, hy), (nz, hz))]
    mesh = lambda xs, ys, zs: np.meshgrid(xs, ys, zs, indexing="ij")
    at = lambda f, xs, ys, zs: np.transpose(f(*mesh(xs, ys, zs)), (2, 1, 0))  # [k][j][i]
    g = o3.Grid3(nx, ny, nz, hx, hy, hz, at(eta, xc, yc, zc), at(eta, xn, yn, zc), at(eta, xn, yc, zn),
                 at(eta, xc, yn, zn))
    vx = at(lambda x, y, z: q(0, x, y, z), xn, yc, zc)
    vy = at(lambda x, y, z: q(1, x, y, z), xc, yn, zc)
    vz = at(lambda x, y, z: q(2, x, y, z), xc, yc, zn)
    got = o3.apply_M(g, vx, vy, vz)

    def cont(c, x, y, z):
        # sum_j d/dx_j [eta (d_j v_c + d_c v_j)] by the product rule
        gr = [grad(m, x, y, z) for m in range(3)]
        out = 0.0
        for j in range(3):
            s = gr[c][j] + gr[j][c]
            ds = hess(c)[j, j] + hess(j)[c, j]
            out = out + deta[j] * s + eta(x, y, z) * ds
        return out

    pts = ((xn, yc, zc), (xc, yn, zc), (xc, yc, zn))
    checked = 0
    for c in range(3):
        want = at(lambda x, y, z: cont(c, x, y, z), *pts[c])
        # interior unknowns away from the walls (no zeroed wall edge in the stencil)
        sl = [slice(2, -2)] * 3
        assert np.allclose(got[c][tuple(sl)], want[tuple(sl)], rtol=1e-9, atol=1e-9 * np.abs(want).max())
        checked += got[c][tuple(sl)].size
    assert checked > 100


@pytest.mark.parametrize("nx,ny,nz,l", [(5, 6, 4, (1.0, 1.3, 0.8)), (7, 3, 5, (0.6, 1.0, 1.0))])
def test_operator_symmetric_negative_definite_3d(o3, nx, ny, nz, l):
    g = rand_grid3(o3, nx, ny, nz, 11, *l)
    m = masks3(nx, ny, nz)
    u = inputs.random_velocity3d(nx, ny, nz, 1)
    w = inputs.random_velocity3d(nx, ny, nz, 2)
    Mu, Mw = o3.apply_M(g, *u), o3.apply_M(g, *w)
    a, b = dot3(Mu, w, m), dot3(u, Mw, m)
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
    assert dot3(Mu, u, m) < 0 and dot3(Mw, w, m) < 0


def test_diag_is_operator_diagonal_3d(o3):
    nx, ny, nz = 5, 4, 4
    g = rand_grid3(o3, nx, ny, nz, 12, 1.0, 0.9, 1.2)
    d = o3.diag_M(g)
    m = masks3(nx, ny, nz)
    rng = np.random.default_rng(0)
    for c in range(3):
        idx = np.argwhere(m[c])
        for q in idx[rng.choice(len(idx), 6, replace=False)]:
            e = list(o3.Grid3.zeros(g))
            e[c] = e[c].copy()
            e[c][tuple(q)] = 1.0
            Me = o3.apply_M(g, *e)
            assert Me[c][tuple(q)] == pytest.approx(d[c][tuple(q)], rel=1e-13)


def extrude(a, nz, plus=0):
    return np.repeat(a[None], nz + plus, axis=0)


def zinvariant(o3, nx, ny, nz, seed, zero_z_edges):
    """A 3D grid whose cell and x-y edge viscosities repeat a 2D field in z."""
    ec2, en2 = inputs.random_viscosity(nx, ny, seed, (-2.0, 2.0))
    lx, ly, lz = 1.2, 0.9, 0.7
    exz = np.zeros((nz + 1, ny, nx + 1)) if zero_z_edges else 10 ** np.random.default_rng(seed).uniform(
        -1, 1, (nz + 1, ny, nx + 1))
    eyz = np.zeros((nz + 1, ny + 1, nx)) if zero_z_edges else 10 ** np.random.default_rng(seed + 1).uniform(
        -1, 1, (nz + 1, ny + 1, nx))
    g3 = o3.Grid3(nx, ny, nz, lx / nx, ly / ny, lz / nz, extrude(ec2, nz), extrude(en2, nz), exz, eyz)
    return g3, (ec2, en2, lx / nx, ly / ny)


def test_z_invariant_field_reduces_to_the_2d_operator(o3, ora):
    """vx, vy independent of z, vz = 0, eta_c and eta_xy independent of z (the
    z-edge viscosities arbitrary): the x and y rows of the 3D operator are the
    2D operator of the pinned 2D oracle and the z row vanishes."""
    nx, ny, nz = 9, 7, 5
    g3, (ec2, en2, hx, hy) = zinvariant(o3, nx, ny, nz, 21, zero_z_edges=False)
    g2 = ora.Grid(nx, ny, hx, hy, ec2, en2)
    vx2, vy2 = inputs.random_velocity(nx, ny, 22)
    mx2, my2 = ora.apply_M(g2, vx2, vy2)
    mx, my, mz = o3.apply_M(g3, extrude(vx2, nz), extrude(vy2, nz), np.zeros((nz + 1, ny, nx)))
    for k in range(nz):
        assert np.allclose(mx[k], mx2, rtol=1e-13, atol=1e-13 * np.abs(mx2).max())
        assert np.allclose(my[k], my2, rtol=1e-13, atol=1e-13 * np.abs(my2).max())
    assert np.abs(mz).max() <= 1e-12 * np.abs(mx2).max()


@pytest.mark.parametrize("smoother", ["jacobi", "ras"])
def test_z_invariant_smoothing_reduces_to_the_2d_oracle(o3, ora, smoother):
    """With the z-edge viscosities zero (no shear across z layers) the 3D
    diagonal of vx and vy is the 2D one, so z-invariant Jacobi and RAS with
    tiles spanning the whole z extent (the z shift 0) reproduce the 2D
    oracle's iterates on every layer."""
    nx, ny, nz = 23, 17, 4
    g3, (ec2, en2, hx, hy) = zinvariant(o3, nx, ny, nz, 31, zero_z_edges=True)
    g2 = ora.Grid(nx, ny, hx, hy, ec2, en2)
    prob = inputs.sinker_problem(nx, ny, eta_in=10.0, lx=hx * nx, ly=hy * ny)
    v2 = inputs.random_velocity(nx, ny, 32, 0.1)
    b2 = ora.rhs(g2, prob.fx, prob.fy, None)
    b3 = (extrude(b2[0], nz), extrude(b2[1], nz), np.zeros((nz + 1, ny, nx)))
    v3 = (extrude(v2[0], nz), extrude(v2[1], nz), np.zeros((nz + 1, ny, nx)))
    if smoother == "jacobi":
        want = ora.jacobi(g2, *b2, 0.3, 6, *v2)
        got = o3.jacobi(g3, b3, 0.3, 6, v3)
    else:
        shifts2 = inputs.random_shifts(3, 8, 6, 33)
        shifts3 = np.concatenate([shifts2, np.zeros((3, 1), np.int32)], axis=1)
        want = ora.ras(g2, *b2, 0.3, 7, 8, 6, 3, 1, shift_mode=2, shifts=shifts2, vx=v2[0], vy=v2[1])
        got = o3.ras(g3, b3, 0.3, 7, (8, 6, nz), 3, 1, shift_mode=2, shifts=shifts3, v=v3)
    for k in range(nz):
        assert np.allclose(got[0][k], want[0], rtol=1e-14, atol=1e-14 * np.abs(want[0]).max())
        assert np.allclose(got[1][k], want[1], rtol=1e-14, atol=1e-14 * np.abs(want[1]).max())
    assert np.all(got[2] == 0.0)


# --------------------------------------------------------------------------
# Jacobi and RAS (Algorithm 2 on 3D tiles)
# --------------------------------------------------------------------------
def ras3_case(o3, nx=11, ny=9, nz=8, seed=40):
    g = rand_grid3(o3, nx, ny, nz, seed, 1.0, 0.8, 1.1)
    prob = inputs.sinker3d_problem(nx, ny, nz, eta_in=100.0, lx=1.0, ly=0.8, lz=1.1)
    b = o3.rhs(g, prob.fx, prob.fy, prob.fz)
    v0 = inputs.random_velocity3d(nx, ny, nz, seed + 1, 0.1)
    return g, b, v0


@pytest.mark.parametrize("k", [1, 2, 3])
def test_ras3_whole_domain_tile_is_k_jacobi_sweeps(o3, k):
    g, b, v0 = ras3_case(o3)
    got = o3.ras(g, b, 0.3, k, (g.nx, g.ny, g.nz), k, 0, shift_mode=0, v=v0)
    want = o3.jacobi(g, b, 0.3, k, v0)
    for a, w in zip(got, want):
        assert np.array_equal(a, w)


@pytest.mark.parametrize("k,sweeps", [(2, 5), (3, 6), (4, 4)])
def test_ras3_overlap_threshold_is_k_minus_1(o3, k, sweeps):
    """Overlap k - 1 reproduces global Jacobi (the stencil couples cells at
    Chebyshev distance one, in 3D too); overlap k - 2 does not."""
    g, b, v0 = ras3_case(o3)
    want = o3.jacobi(g, b, 0.3, sweeps, v0)
    got = o3.ras(g, b, 0.3, sweeps, (4, 3, 3), k, k - 1, shift_mode=1, seed=7, v=v0)
    for a, w in zip(got, want):
        assert np.allclose(a, w, rtol=1e-14, atol=1e-15 * np.abs(w).max())
    if k >= 2:
        bad = o3.ras(g, b, 0.3, sweeps, (4, 3, 3), k, k - 2, shift_mode=1, seed=7, v=v0)
        assert max(np.abs(a - w).max() for a, w in zip(bad, want)) > 1e-8 * max(np.abs(w).max() for w in want)


def test_ras3_tile_order_invariant_and_single_writer(o3):
    g, b, v0 = ras3_case(o3)
    a = o3.ras(g, b, 0.3, 5, (5, 4, 3), 2, 0, shift_mode=1, seed=3, v=v0, return_counts=True)
    c = o3.ras(g, b, 0.3, 5, (5, 4, 3), 2, 0, shift_mode=1, seed=3, order_seed=99, v=v0)
    for x, y in zip(a[:3], c):
        assert np.array_equal(x, y)
    for cnt, m in zip(a[3:], masks3(g.nx, g.ny, g.nz)):
        assert np.all(cnt[m] == 1) and np.all(cnt[~m] == 0)


def test_ras3_drawn_shifts_match_explicit_shifts(o3):
    g, b, v0 = ras3_case(o3)
    sh = [o3.ras_shift(1, 17, t, 5, 4, 3) for t in range(3)]
    assert all(0 <= s[0] < 5 and 0 <= s[1] < 4 and 0 <= s[2] < 3 for s in sh)
    a = o3.ras(g, b, 0.3, 6, (5, 4, 3), 2, 1, shift_mode=1, seed=17, v=v0)
    c = o3.ras(g, b, 0.3, 6, (5, 4, 3), 2, 1, shift_mode=2, shifts=sh, v=v0)
    for x, y in zip(a, c):
        assert np.array_equal(x, y)


def test_jacobi3_contracts_on_the_sinker(o3):
    nx = 10
    prob = inputs.sinker3d_problem(nx, eta_in=100.0)
    g = o3.Grid3(nx, nx, nx, prob.hx, prob.hy, prob.hz, prob.eta_c, prob.eta_xy, prob.eta_xz, prob.eta_yz)
    f = (prob.fx, prob.fy, prob.fz)
    b = o3.rhs(g, *f)
    e0 = o3.energy(g, f, None, g.zeros())
    v = o3.jacobi(g, b, 0.3, 30, g.zeros())
    e1 = o3.energy(g, f, None, v)
    assert e0[0] == pytest.approx(e0[2], rel=1e-14)
    assert e1[0] < 0.8 * e0[0]


# --------------------------------------------------------------------------
# energy norm (Sec. 6.4 over three components)
# --------------------------------------------------------------------------
def test_energy3_velocity_weight_and_pressure_part(o3):
    """f a unit vector at one unknown of each component, v = 0: the velocity
    sum is 1 / (-M_uu) with M_uu read off by a unit-vector apply; a uniform
    expansion vx = c x gives D v = c and the pressure part
    c^2 sum(eta_c) / (2/hx^2 + 2/hy^2 + 2/hz^2)."""
    nx, ny, nz = 6, 5, 4
    g = rand_grid3(o3, nx, ny, nz, 50, 1.0, 0.7, 1.3)
    pos = ((2, 3, 2), (1, 2, 4), (2, 1, 3))  # [k][j][i] of a vx, vy, vz unknown
    for c, q in enumerate(pos):
        f = list(g.zeros())
        f[c][q] = 1.0
        rv, rp, ff = o3.energy(g, f, None, g.zeros())
        e = list(g.zeros())
        e[c][q] = 1.0
        Me = o3.apply_M(g, *e)
        assert rp == 0.0
        assert rv == pytest.approx(-1.0 / Me[c][q], rel=1e-13) and ff == pytest.approx(rv, rel=1e-15)
    cc = 0.4
    vx = np.broadcast_to(cc * np.arange(nx + 1) * g.hx, (nz, ny, nx + 1)).copy()
    _, rp, _ = o3.energy(g, g.zeros(), None, (vx, g.zeros()[1], g.zeros()[2]))
    lap = 2 / g.hx ** 2 + 2 / g.hy ** 2 + 2 / g.hz ** 2
    assert rp == pytest.approx(cc * cc * g.eta_c.sum() / lap, rel=1e-13)
