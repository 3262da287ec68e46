"""The failure paths of the bounded waits, exercised without a GPU fault:
the waits of the staged kernel and of the cluster-resident kernel run
against a barrier that nothing completes, give up at their clock limit,
report it through the status word, and the CUDA context stays usable."""
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


def test_resident_wait_gives_up_reports_and_context_steps_again():
    """The cluster-resident kernel's own ghost wait (not the staged one)."""
    nx, ny = 128, 32
    lat = plbm.Lattice(nx, ny, 0.9, 10.0, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3)
    assert lat.kernel == "resident"
    lat.init(np.ones((ny, nx)))
    lat.step(10)
    lat.sync()
    lat.probe_resident_wait()
    with pytest.raises(plbm.LBMError) as ex:
        lat.sync()
    assert ex.value.status == plbm.ETIMEOUT
    assert "cluster-resident" in str(ex.value)
    # a fresh init clears the status word; the kernel steps as before
    lat.init(np.ones((ny, nx)))
    lat.step(200)
    lat.sync()
    ref = plbm.Lattice(nx, ny, 0.9, 10.0, plbm.PERIODIC_GRADIENT, plbm.DIFFUSE_WALLS, 1e-3,
                       kernel="scalar")
    ref.init(np.ones((ny, nx)))
    ref.step(200)
    assert np.array_equal(lat.populations(), ref.populations())
