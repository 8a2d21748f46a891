"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/stokes.h declares; argument errors are reported without
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_19061_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    with open(os.path.join(ROOT, "include", "stokes.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stokes_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("stokes_create", "stokes_get_layout", "stokes_set_viscosity", "stokes_set_rhs",
                 "stokes_apply_operator", "stokes_smooth", "stokes_residual_energy_norm", "stokes_vcycle",
                 "stokes_destroy", "stokes_strerror"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2509_19061_gb300 import api
    assert set(declared_symbols()) <= set(api.exported_symbols())


def test_argument_errors_without_device(lib):
    from paper_2509_19061_gb300 import api
    out = ctypes.c_void_p(123)
    f = api._lib()
    assert f.stokes_create(1, 8, 1.0, 1.0, 1, None, ctypes.byref(out)) == api.STOKES_ERR_ARG
    assert out.value is None
    assert f.stokes_create(8, 8, 0.0, 1.0, 1, None, ctypes.byref(out)) == api.STOKES_ERR_ARG
    assert f.stokes_create(8, 8, 1.0, 1.0, 7, None, ctypes.byref(out)) == api.STOKES_ERR_ARG
    assert f.stokes_create((1 << 18) + 1, 8, 1.0, 1.0, 1, None, ctypes.byref(out)) == api.STOKES_ERR_ARG
    assert f.stokes_create(8, (1 << 18) + 1, 1.0, 1.0, 1, None, ctypes.byref(out)) == api.STOKES_ERR_ARG
    assert f.stokes_get_layout(None, 0, None, None, None, None) == api.STOKES_ERR_ARG
    assert f.stokes_smooth(None, None, None, None, None) == api.STOKES_ERR_ARG
    assert f.stokes_destroy(None) == api.STOKES_OK
    assert f.stokes_strerror(api.STOKES_ERR_DIVERGED).decode().startswith("diverged")
    assert f.stokes_set_option(None, api.STOKES_OPT_PAIRED, 1) == api.STOKES_ERR_ARG
    for bad in [(0, 8, 8, 8, 1, 0, 1, 1), (8, 8, 8, 8, -1, 0, 1, 1), (8, 8, 8, 8, 1, 2, 1, 1),
                (8, 8, 8, 8, 1, 0, 1, 3), (8, 8, 0, 8, 1, 0, 1, 1)]:
        assert f.stokes_tile_kernel_plan(*bad, None, None, None) == api.STOKES_ERR_ARG, bad


def test_product_path_has_no_oracle_dependency():
    """The package never imports the oracle or falls back to CPU code."""
    pkg = os.path.join(ROOT, "paper_2509_19061_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".h", ".cuh")):
                with open(os.path.join(dirpath, fn)) as f:
                    src = f.read()
                assert "import oracle" not in src and "from oracle" not in src, fn
                assert "stokes_oracle" not in src, fn


def test_batch_argument_errors_without_device(lib):
    from paper_2509_19061_gb300 import api
    f = api._lib()
    out = ctypes.c_void_p(123)
    n2 = (ctypes.c_int * 2)(32, 1)
    l2 = (ctypes.c_double * 2)(1.0, 1.0)
    assert f.stokes_batch_create(2, n2, n2, l2, l2, 1, None, ctypes.byref(out)) == api.STOKES_ERR_ARG
    assert out.value is None
    assert f.stokes_batch_create(0, n2, n2, l2, l2, 1, None, ctypes.byref(out)) == api.STOKES_ERR_ARG
    assert f.stokes_batch_get_layout(None, 0, None, None, None) == api.STOKES_ERR_ARG
    assert f.stokes_batch_smooth(None, None, None, None, None) == api.STOKES_ERR_ARG
    assert f.stokes_batch_solve(None, None, None, None, None, None, None, None) == api.STOKES_ERR_ARG
    assert f.stokes_batch_destroy(None) == api.STOKES_OK


def test_batched_workload_recipe():
    """Sides are multiples of 64 between 64 and 1024 (so that halving reaches
    a coarsest level of at most 16 x 16 cells), contrasts in [1e2, 1e6],
    sinkers inside the box; the table is a pure function of the seed."""
    from paper_2509_19061_gb300 import inputs
    a = inputs.batch_specs(seed=5, count=256)
    assert a == inputs.batch_specs(seed=5, count=256)
    ns = [s.n for s in a]
    assert all(n % 64 == 0 and 64 <= n <= 1024 for n in ns)
    assert len(set(ns)) >= 12
    for n in ns:
        m = n
        while m % 2 == 0 and m > 16:
            m //= 2
        assert 2 * m * (m - 1) <= 1024
    assert all(1e2 <= s.contrast <= 1e6 for s in a)
    assert all(s.radius + 0.3 > 0 and 0.05 <= s.radius <= 0.2 and 0.3 <= s.cx <= 0.7 for s in a)
    cells = np.array([n * n for n in ns], dtype=np.float64)
    assert 1.0e5 < cells.mean() < 3.0e5
