"""The slab decomposition's host side on CPU: the row plan of
stokes_slab_plan (a host computation of the library), and the exchange
protocol of one slab per rank run as world-size 2 and 3 process groups under
gloo, each rank smoothing its slab with the oracle's RAS tiles (Algorithm 2)
and trading halo rows with its neighbours after every outer iteration.  The
gathered result must equal the oracle's RAS on the whole grid."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _api():
    from paper_2509_19061_gb300 import api, build
    build.build()
    return api


@pytest.mark.parametrize("ny,n,tj,o", [(60, 2, 8, 1), (61, 3, 8, 3), (257, 4, 32, 7), (1024, 7, 64, 7)])
def test_slab_plan_partitions_the_rows(ny, n, tj, o):
    api = _api()
    H = tj + o + 1
    plans = [api.stokes_slab_plan(ny, n, tj, o, s) for s in range(n)]
    assert plans[0][0] == 0 and plans[-1][1] == ny
    for s, (r0, r1, R0, R1) in enumerate(plans):
        assert r1 - r0 >= H + 1
        assert R0 == max(0, r0 - H) and R1 == min(ny, r1 + H)
        if s > 0:
            assert plans[s - 1][1] == r0
            # the halo below comes from the neighbour's own rows
            assert plans[s - 1][0] <= R0
        if s + 1 < n:
            assert R1 <= plans[s + 1][1] - 1


def test_slab_plan_rejects_thin_slabs():
    api = _api()
    with pytest.raises(api.StokesError) as e:
        api.stokes_slab_plan(40, 4, 8, 3, 0)  # 10 rows per slab < 8 + 3 + 2
    assert e.value.status == api.STOKES_ERR_ARG
    with pytest.raises(api.StokesError):
        api.stokes_slab_plan(40, 2, 8, 3, 2)  # no slab 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASE = dict(nx=37, ny=66, ti=9, tj=8, seed=11, omega=0.3)


def _problem():
    sys.path.insert(0, ROOT)
    import oracle as ora
    from paper_2509_19061_gb300 import inputs
    nx, ny = CASE["nx"], CASE["ny"]
    prob = inputs.sinker_problem(nx, ny, eta_in=1e3, lx=1.1, ly=1.7)
    prob.eta_c, prob.eta_n = inputs.random_viscosity(nx, ny, 5, (-2.0, 2.0))
    g = ora.Grid(nx, ny, prob.hx, prob.hy, prob.eta_c, prob.eta_n)
    bx, by = ora.rhs(g, prob.fx, prob.fy, None)
    v0 = inputs.random_velocity(nx, ny, 6, 0.1)
    return ora, g, bx, by, v0


def _rank_main(rank, world, port, out_dir, k, o, sweeps):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2509_19061_gb300 import api
    ora, g, bx, by, v0 = _problem()
    nx, ny, ti, tj = CASE["nx"], CASE["ny"], CASE["ti"], CASE["tj"]
    plans = [api.stokes_slab_plan(ny, world, tj, o, s) for s in range(world)]
    r0, r1, R0, R1 = plans[rank]
    # rows this rank does not store hold NaN: reading them would poison the result
    vx = np.full((ny, nx + 1), np.nan)
    vy = np.full((ny + 1, nx), np.nan)
    vx[R0:R1] = v0[0][R0:R1]
    vy[R0:R1 + 1] = v0[1][R0:R1 + 1]

    def exchange(vx, vy):
        reqs, bufs = [], []
        for peer in (rank - 1, rank + 1):
            if not 0 <= peer < world:
                continue
            pr0, pr1, pR0, pR1 = plans[peer]
            # what the peer stores but does not own and this rank owns
            a, b = max(pR0, r0), min(pR1, r1)
            bv = min(pR1 + 1, r1)
            for arr, hi in ((vx, b), (vy, bv)):
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(arr[a:hi])), peer))
            # what this rank stores but does not own and the peer owns
            a, b = max(R0, pr0), min(R1, pr1)
            bv = min(R1 + 1, pr1)
            for arr, hi in ((vx, b), (vy, bv)):
                t = torch.empty((hi - a, arr.shape[1]), dtype=torch.float64)
                reqs.append(dist.irecv(t, peer))
                bufs.append((arr, a, hi, t))
        for r in reqs:
            r.wait()
        for arr, a, hi, t in bufs:
            arr[a:hi] = t.numpy()

    n_outer = (sweeps + k - 1) // k
    cuts_y = lambda sj: [0] + [c for c in range(sj, ny, tj) if c > 0] + [ny]
    for t in range(n_outer):
        ks = sweeps - (n_outer - 1) * k if t == n_outer - 1 else k
        si, sj = ora.ras_shift(1, CASE["seed"], t, ti, tj)
        ntx = ora.tile_count(nx, ti, si)
        cy = cuts_y(sj)
        rows = [b for b in range(len(cy) - 1) if cy[b] < r1 and cy[b + 1] > r0]
        tiles = [(a, b) for b in rows for a in range(ntx)]
        vx, vy = ora.ras_tiles(g, bx, by, CASE["omega"], ti, tj, ks, o, si, sj, tiles, vx, vy, vx, vy)
        exchange(vx, vy)
    own = np.concatenate([vx[r0:r1].ravel(), vy[r0:r1].ravel()])
    assert np.all(np.isfinite(own))
    np.save(os.path.join(out_dir, "vx%d.npy" % rank), vx[r0:r1])
    np.save(os.path.join(out_dir, "vy%d.npy" % rank), vy[r0:r1])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,k,o,sweeps", [(2, 3, 1, 8), (3, 4, 0, 9), (3, 2, 1, 5), (2, 4, 3, 12)])
def test_slab_exchange_protocol_gloo(tmp_path, world, k, o, sweeps):
    import torch.multiprocessing as mp
    _api()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path), k, o, sweeps)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    ora, g, bx, by, v0 = _problem()
    ny = CASE["ny"]
    gx = np.concatenate([np.load(os.path.join(tmp_path, "vx%d.npy" % r)) for r in range(world)])
    gy = np.concatenate([np.load(os.path.join(tmp_path, "vy%d.npy" % r)) for r in range(world)])
    ref = ora.ras(g, bx, by, CASE["omega"], sweeps, CASE["ti"], CASE["tj"], k, o, shift_mode=1, seed=CASE["seed"],
                  vx=v0[0], vy=v0[1])
    assert np.array_equal(gx, ref[0])
    assert np.array_equal(gy, ref[1][:ny])
