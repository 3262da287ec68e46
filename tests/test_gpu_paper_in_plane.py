"""Section 3.2 (Figs. 7-8) on the GPU at the paper's 3 x 301 grid: in-plane
heat flow along a film with diffuse walls, driven by the periodic
temperature gradient (Eqs. 58-60), Kn_N = 0.01 and Kn_R from the diffusive
to the hydrodynamic regime, against the cross-section profile of Eq. 68
and the effective conductivity of Eq. 69."""
import numpy as np
import pytest

import paper_2010_01847_gb300 as plbm
from tests.test_oracle_pins import eq68, eq69

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


# (Kn_R, steps, core tolerance, mean tolerance); the oracle on this grid gives
# core errors 1e-11, 3e-7, 6e-4, 6.7e-3, 5.4e-3 and mean errors 0.12 %,
# 0.36 %, <1 %, 0.77 %, <2 % for Kn_R = 0.01, 0.1, 1, 10, 100
CASES = [(0.01, 60000, 1e-4, 5e-3), (0.1, 60000, 1e-4, 8e-3), (1.0, 30000, 2e-3, 0.01),
         (10.0, 150000, 1e-2, 0.015), (100.0, 150000, 1.2e-2, 0.02)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("kn_R,steps,core_tol,mean_tol", CASES)
def test_in_plane_film_follows_eqs_68_69(kn_R, steps, core_tol, mean_tol, precision):
    nx, ny = 3, 301
    d = ny - 1
    tau_N, tau_R = plbm.tau_from_kn(0.01, d), plbm.tau_from_kn(kn_R, d)
    lat = plbm.Lattice(nx, ny, tau_N, tau_R, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3,
                       precision=precision)
    lat.init(np.ones((ny, nx)))
    lat.step(steps)
    e, qx, qy = lat.moments()
    slope = np.polyfit(np.arange(nx), e.mean(0), 1)[0]
    tau_r = tau_R
    Q = qx.mean(1) / (-(5 / 9) * tau_r * slope)     # q_x over the Fourier flux
    Y = np.arange(ny) / d
    core = (Y >= 0.2) & (Y <= 0.8)
    assert np.abs(Q - eq68(Y, 0.01, kn_R))[core].max() < core_tol
    assert Q.mean() == pytest.approx(eq69(0.01, kn_R), rel=mean_tol)
    assert np.abs(qy).max() < 1e-3 * np.abs(qx).max()
