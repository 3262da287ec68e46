"""The failure path of the staged kernel's bounded waits, exercised without a
GPU fault: the same wait runs against a barrier that nothing completes, gives
up at its clock limit, reports it through the status word, and the CUDA
context stays usable afterwards."""
import numpy as np
import pytest

import paper_2010_01847_gb300 as plbm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def test_bounded_wait_gives_up_and_context_survives():
    gave_up, seconds = plbm.check_bounded_wait()
    assert gave_up
    assert 0.5 < seconds < 30.0          # the clock limit is ~2 s at full SM clock
    # the context still runs the solver
    lat = plbm.Lattice(64, 8, 0.9, 10.0)
    lat.init(np.ones((8, 64)))
    lat.step(5)
    lat.sync()
    e, _, _ = lat.moments()
    np.testing.assert_allclose(e, 1.0, atol=1e-6)
