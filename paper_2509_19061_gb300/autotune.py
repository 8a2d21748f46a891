"""Autotuner for the RAS smoother inside the multigrid solve.

The RAS tile shape (T_I, T_J), the local sweeps k and the overlap trade
per-sweep throughput against convergence per sweep (Sec. 6.3): a larger k
reads HBM less often but the tile-local Jacobi sweeps damp the global error
less, and a zero overlap is cheapest per sweep but converges slowest.  The
objective is therefore the wall time of the whole solve to E_v <= tol, not
the speed of one sweep.

Results are kept in a JSON cache keyed by (size bucket, dtype, contrast
bucket): size bucket = round(log2(sqrt(nx * ny))), dtype = the precision
the sweeps run in (the V-cycle's inner precision), contrast bucket =
round(log10(max eta / min eta)).  A batch of instances shares one schedule,
tuned on the batch itself (objective: the time until every instance has
converged) and kept under its own name.  Tuning runs on the GPU through the
library; lookups are plain Python.
"""
import json
import math
import os
import time
from dataclasses import asdict, dataclass

DEFAULT_CANDIDATES = [(ti, tj, k, o) for (ti, tj) in ((16, 16), (32, 32), (56, 32))
                      for k in (1, 2, 4, 8) for o in sorted({0, k - 1})]
# 64-column windows, which the FP32 packed-pair kernel sweeps: exact Jacobi at k = 8 and ring-only tiles
DEFAULT_CANDIDATES += [(48, 32, 8, 7), (62, 32, 4, 0), (62, 32, 8, 0), (48, 64, 8, 7), (62, 56, 8, 0)]
# FP64 exact Jacobi at k = 8 on a window that fits the register layout (40 x 40)
DEFAULT_CANDIDATES += [(24, 24, 8, 7)]


def fast_layout(api, nx, ny, ti, tj, overlap, dtype):
    """Whether a launch shape runs a register-resident tile kernel.  Windows
    that fit none (an FP32 window wider than 64 columns at overlap 7, an FP64
    window of more than 512 cells per strip column set) fall to the general
    all-shared-memory kernel, 3 to 5 times slower per sweep, so the tuner
    does not consider them."""
    try:
        return api.stokes_tile_kernel_plan(nx, ny, (ti, tj), overlap, dtype)[0] != "shared"
    except api.StokesError:
        return False


@dataclass
class Choice:
    tile_i: int
    tile_j: int
    k: int
    overlap: int
    seconds: float = float("nan")
    cycles: int = -1

    def smoother(self):
        return dict(variant="ras", tile=(self.tile_i, self.tile_j), k=self.k, overlap=self.overlap)


DEFAULT = Choice(32, 32, 4, 3)

# cache shipped with the package, written on a GB300 by
#   python -m paper_2509_19061_gb300.autotune --out paper_2509_19061_gb300/ras_tuning.json
SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ras_tuning.json")


def contrast_of(eta_c, eta_n):
    lo = min(float(eta_c.min()), float(eta_n.min()))
    hi = max(float(eta_c.max()), float(eta_n.max()))
    return hi / lo


def bucket(nx, ny, contrast, dtype):
    size_b = int(round(math.log2(math.sqrt(nx * ny))))
    con_b = int(round(math.log10(max(contrast, 1.0))))
    return "n%d_%s_c%d" % (size_b, dtype, con_b)


class Cache:
    """JSON file of the best Choice per bucket (and per named batch)."""

    def __init__(self, path):
        self.path = path
        self.entries = {}
        self.batches = {}
        if path and os.path.exists(path):
            with open(path) as f:
                raw = json.load(f)
            self.entries = {k: Choice(**v) for k, v in raw.get("entries", {}).items()}
            self.batches = {k: Choice(**v) for k, v in raw.get("batches", {}).items()}

    def batch(self, name):
        """The Choice tuned for the named batch, else the default."""
        return self.batches.get(name, DEFAULT)

    def lookup(self, nx, ny, contrast, dtype):
        """The cached Choice of the bucket, else the nearest cached size bucket
        of the same dtype and contrast bucket, else the default."""
        key = bucket(nx, ny, contrast, dtype)
        if key in self.entries:
            return self.entries[key]
        size_b = int(key.split("_")[0][1:])
        tail = key.split("_", 1)[1]
        near = [(abs(int(k.split("_")[0][1:]) - size_b), k) for k in self.entries if k.split("_", 1)[1] == tail]
        if near:
            return self.entries[min(near)[1]]
        return DEFAULT

    def record(self, nx, ny, contrast, dtype, choice):
        self.entries[bucket(nx, ny, contrast, dtype)] = choice

    def save(self):
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"objective": "wall seconds of the flexible-CG solve to E_v <= tol",
                       "entries": {k: asdict(v) for k, v in sorted(self.entries.items())},
                       "batches": {k: asdict(v) for k, v in sorted(self.batches.items())}}, f, indent=1)
        os.replace(tmp, self.path)


def tuned_smoother(nx, ny, eta_c, eta_n, dtype="f32", path=SHIPPED):
    """Smoother keyword arguments (variant, tile, k, overlap) of the cached
    choice for this grid, viscosity contrast and sweep precision."""
    return Cache(path).lookup(nx, ny, contrast_of(eta_c, eta_n), dtype).smoother()


def feasible(ti, tj, k, overlap, nx, ny):
    """Tiles no larger than the grid; the overlap below the tile size."""
    return ti <= nx and tj <= ny and 0 <= overlap < min(ti, tj) and k >= 1


def tune(api, prob, dtype="f64", inner="f32", candidates=None, tol=1e-8, max_cycles=300, nu_max=40, seed=1,
         reps=1):
    """Time the solve of `prob` (an inputs.Problem) to E_v <= tol for every
    candidate (tile_i, tile_j, k, overlap); returns (best Choice, list of all
    Choices).  Each candidate is solved once untimed (hierarchy and graph
    capture), then `reps` times from a zero guess; the minimum counts.
    Candidates that do not converge get an infinite time."""
    import torch
    cands = [c for c in (candidates or DEFAULT_CANDIDATES) if feasible(*c, prob.nx, prob.ny)
             and fast_layout(api, prob.nx, prob.ny, c[0], c[1], c[3], inner)]
    ctx = api.StokesContext(prob.nx, prob.ny, prob.lx, prob.ly, dtype)
    ctx.set_problem(prob)
    vx, vy = ctx.field(), ctx.field()
    out = []
    for ti, tj, k, o in cands:
        kw = dict(variant="ras", tile=(ti, tj), k=k, overlap=o, seed=seed, nu_max=nu_max, inner=inner,
                  krylov=True, tol=tol, max_cycles=max_cycles)
        best, cyc = float("inf"), -1
        try:
            vx.zero_()
            vy.zero_()
            ctx.vcycle(vx, vy, None, **kw)
            for _ in range(reps):
                vx.zero_()
                vy.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, e, c = ctx.vcycle(vx, vy, None, **kw)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                if st == api.STOKES_OK:
                    best, cyc = min(best, dt), c
        except api.StokesError:
            best = float("inf")
        out.append(Choice(ti, tj, k, o, best, cyc))
    ctx.close()
    win = min(out, key=lambda c: c.seconds) if out else DEFAULT
    return win, out


def tune_buckets(api, sizes=(256, 1024, 4096), contrasts=(1e2, 1e4, 1e6), dtype="f64", inner="f32", path=None,
                 log=print, candidates=None, cache=None):
    """Tune one representative problem per (size, contrast) bucket: the
    centred sinker of Sec. 6.1 with eta_in = contrast on an n x n grid, FP64
    outer iteration, sweeps in `inner`.  Returns the cache (saved to `path`
    when given)."""
    from . import inputs
    if cache is None:
        cache = Cache(path) if path else Cache(None)
    for n in sizes:
        for c in contrasts:
            prob = inputs.sinker_problem(n, eta_in=c)
            win, table = tune(api, prob, dtype=dtype, inner=inner, candidates=candidates)
            cache.record(n, n, contrast_of(prob.eta_c, prob.eta_n), inner, win)
            log("n=%d contrast=%.0e: best %s in %.4f s (%d cycles); default %s" % (
                n, c, (win.tile_i, win.tile_j, win.k, win.overlap), win.seconds, win.cycles,
                next(("%.4f s" % t.seconds for t in table
                      if (t.tile_i, t.tile_j, t.k, t.overlap) == (32, 32, 4, 3)), "n/a")))
    if path:
        cache.save()
    return cache


def tune_batch(api, probs, name, candidates=None, cache=None, tol=1e-8, max_cycles=300, nu_max=40, seed=1,
               log=print):
    """Tune one schedule for a batch (inputs.Problem list, solved together by
    the batched path: FP64 outer flexible CG, FP32 sweeps) by the wall time
    until every instance reaches E_v <= tol; schedules that leave an
    instance unconverged get an infinite time.  Records the winner under
    `name` in `cache` (when given) and returns (winner, table)."""
    import torch
    cands = candidates or [(32, 32, 4, 3), (56, 32, 4, 3), (32, 32, 8, 7), (32, 32, 4, 0), (56, 32, 4, 0),
                           (32, 32, 8, 0), (56, 32, 8, 0), (32, 32, 2, 1), (16, 16, 4, 3),
                           (48, 32, 8, 7), (48, 64, 8, 7), (62, 56, 8, 0)]
    n_max = max(max(q.nx, q.ny) for q in probs)
    cands = [c for c in cands if fast_layout(api, n_max, n_max, c[0], c[1], c[3], "f32")]
    b = api.BatchContext([q.nx for q in probs], [q.ny for q in probs], [q.lx for q in probs],
                         [q.ly for q in probs], "f64")
    b.set_problems(probs)
    vx, vy = b.slab(), b.slab()
    out = []
    for ti, tj, k, o in cands:
        kw = dict(variant="ras", tile=(ti, tj), k=k, overlap=o, seed=seed, nu_max=nu_max, inner="f32", krylov=True,
                  tol=tol, max_cycles=max_cycles)
        vx.zero_()
        vy.zero_()
        b.solve(vx, vy, None, **kw)  # plans and graph
        vx.zero_()
        vy.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, e, cyc, sts = b.solve(vx, vy, None, **kw)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ok = st == api.STOKES_OK
        out.append(Choice(ti, tj, k, o, dt if ok else float("inf"), int(max(cyc))))
        log("batch %s: %s %.3f s, max %d cycles, %s" % (name, (ti, tj, k, o), dt, max(cyc),
                                                       "converged" if ok else "not converged"))
    b.close()
    win = min(out, key=lambda c: c.seconds)
    if cache is not None:
        cache.batches[name] = win
    return win, out


BATCH_NAME = "batch256_seed5"


if __name__ == "__main__":
    import argparse

    from . import api as _api
    from . import build as _build
    ap = argparse.ArgumentParser(description="tune the RAS smoother per size/contrast bucket")
    ap.add_argument("--out", required=True, help="JSON cache to write")
    ap.add_argument("--sizes", type=int, nargs="*", default=[256, 1024, 4096])
    ap.add_argument("--contrasts", type=float, nargs="+", default=[1e2, 1e4, 1e6])
    ap.add_argument("--dtype", default="f64")
    ap.add_argument("--inner", default="f32")
    ap.add_argument("--f64-sizes", type=int, nargs="*", default=[256, 1024],
                    help="sizes also tuned with FP64 sweeps (tiles up to 32 x 32)")
    ap.add_argument("--batch", type=int, default=256, help="instances of the tuned batch (0: none)")
    a = ap.parse_args()
    _build.build()
    cache = Cache(None)
    cache.path = a.out
    if a.sizes:
        tune_buckets(_api, a.sizes, a.contrasts, a.dtype, "f32", cache=cache)
    if a.f64_sizes:
        f64c = [c for c in DEFAULT_CANDIDATES if c[0] <= 32]
        tune_buckets(_api, a.f64_sizes, a.contrasts, a.dtype, "f64", candidates=f64c, cache=cache)
    if a.batch > 0:
        from . import inputs as _inputs
        probs = [_inputs.batch_problem(sp) for sp in _inputs.batch_specs(seed=5, count=a.batch)]
        tune_batch(_api, probs, BATCH_NAME, cache=cache)
    cache.save()
