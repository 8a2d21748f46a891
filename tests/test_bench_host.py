"""Host-side arithmetic of bench.py (CPU): the energy-norm weights the
benchmark uses to state the FP32 error equal -diag(M) of the oracle."""
import numpy as np

import bench
import oracle as ora
from paper_2509_19061_gb300 import inputs


def test_energy_weights_are_minus_diag_m():
    for nx, ny, lx, ly in ((37, 23, 1.3, 0.9), (16, 16, 1.0, 1.0), (5, 9, 0.5, 2.0)):
        prob = inputs.sinker_problem(nx, ny, eta_in=1e3, lx=lx, ly=ly)
        prob.eta_c, prob.eta_n = inputs.random_viscosity(nx, ny, nx + ny, (-2.0, 2.0))
        wx, wy = bench.energy_weights(prob)
        dx, dy = ora.diag_M(ora.Grid(nx, ny, prob.hx, prob.hy, prob.eta_c, prob.eta_n))
        assert wx.shape == dx.shape and wy.shape == dy.shape
        assert np.allclose(wx, -dx, rtol=1e-14, atol=0.0)
        assert np.allclose(wy, -dy, rtol=1e-14, atol=0.0)
