"""Out-of-bounds writes into neighbouring memory, checked without a
sanitizer: the two population buffers are handed to lbm_create_ex as views
into one larger allocation whose guard bands (before, between and after
them) hold a known byte pattern; after init, steps, fused and stand-alone
residuals and read-outs on lattices that exercise every kernel, ragged
sizes and every boundary kind, the guard bands must be untouched."""
import numpy as np
import pytest

import paper_2010_01847_gb300 as plbm
from paper_2010_01847_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

GUARD = 1 << 16          # bytes, a multiple of 256 (buffer alignment)
PATTERN = 0xA5

S = plbm.SIDES
CASES = [
    # (nx, ny, bc_x, bc_y, delta_e, kernel, precision, sides)
    (37, 29, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3, "scalar", "fp32", None),
    (200, 72, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 2e-3, "vector", "fp32", None),
    (96, 33, plbm.PERIODIC, plbm.PERIODIC, 0.0, "vector", "fp16", None),
    (2048, 24, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3, "staged", "fp32", None),
    (4096, 9, plbm.PERIODIC_GRADIENT, plbm.PERIODIC, -1e-3, "vector", "bf16", None),
    # 16-bit storage on the scalar kernel: tiles of 8 nodes (nx % 8 == 0) and of one node
    (96, 33, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3, "scalar", "bf16", None),
    (37, 29, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3, "scalar", "fp16", None),
    (200, 40, S, S, 0.0, "vector", "fp16",
     [(plbm.ISOTHERMAL, 1.0), (plbm.ISOTHERMAL, 1.0), (plbm.ISOTHERMAL, 1.0),
      (plbm.HEAT_FLUX, 1e-4)]),
    (1024, 2, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3, "staged", "fp64", None),
    (1, 1, plbm.PERIODIC, plbm.PERIODIC, 0.0, "scalar", "fp32", None),
    (41, 41, S, S, 0.0, "scalar", "fp32",
     [(plbm.ISOTHERMAL, 1.0), (plbm.ISOTHERMAL, 1.0), (plbm.ISOTHERMAL, 1.0),
      (plbm.HEAT_FLUX, 1e-4)]),
    (401, 3, S, plbm.PERIODIC, 0.0, "scalar", "fp16", [(plbm.HEAT_FLUX, 1e-4), (plbm.DIFFUSE, 0)]),
    # cluster-resident: column slabs (16 CTAs, ragged last slab), row slabs, one CTA
    (201, 201, S, S, 0.0, "resident", "fp32",
     [(plbm.ISOTHERMAL, 1.0), (plbm.ISOTHERMAL, 1.0), (plbm.ISOTHERMAL, 1.0),
      (plbm.HEAT_FLUX, 1e-4)]),
    (17, 1000, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3, "resident", "fp32", None),
    (37, 29, plbm.PERIODIC, plbm.PERIODIC, 0.0, "resident", "fp32", None),
    (8, 2, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3, "resident", "fp32", None),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_{c[5]}_{c[6]}")
def test_guard_bands_untouched(case):
    nx, ny, bcx, bcy, de, kernel, precision, sides = case
    nbytes = plbm.load_library().lbm_population_bytes(plbm.Grid(nx, ny),
                                                       plbm.PRECISIONS[precision])
    nb = (nbytes + 255) // 256 * 256
    total = 3 * GUARD + 2 * nb
    raw = torch.full((total,), PATTERN, dtype=torch.uint8, device="cuda")
    a = raw[GUARD:GUARD + nb]
    b = raw[2 * GUARD + nb:2 * GUARD + 2 * nb]
    lat = plbm.Lattice(nx, ny, 0.9, 15.0, bcx, bcy, de, precision=precision, kernel=kernel,
                       buffers=(a, b), graph_chunk=8,
                       sides=None if sides is None else dict(enumerate(sides)))
    lat.init(*inputs.random_state_fields(nx, ny, seed=nx + 7 * ny))
    lat.residual()
    lat.step(21)
    lat.step_residual(5)
    lat.residual()
    lat.moments()
    lat.populations()
    lat.sync()
    lat.close()
    host = raw.cpu().numpy()
    guards = [host[:GUARD], host[GUARD + nbytes:2 * GUARD + nb],
              host[2 * GUARD + nb + nbytes:]]
    for k, gband in enumerate(guards):
        bad = np.flatnonzero(gband != PATTERN)
        assert bad.size == 0, (k, bad[:8])
