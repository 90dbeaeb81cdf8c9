"""Failure detection without a GPU fault: the bounded mbarrier wait of the
table-staged step gives up on a barrier that nothing completes, reports it,
and leaves the device usable (a lattice steps and matches afterwards)."""
import numpy as np
import pytest

from paper_1906_11925_gb300 import geometry as G
from paper_1906_11925_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)


def test_bounded_wait_gives_up_and_device_stays_usable():
    g = G.tube(radius=3, length=8, nx=7, ny=7)
    nbr, link = lbm.links_build(15, g.xyz, g.io_xyz, g.io_id, g.periodic)
    A = lbm.Lattice(15, g.xyz, nbr, link, 0.8, rho_mean=g.rho_mean)
    A.step(10)
    for limit in (1, 64, 4096):
        assert lbm.check_wait_timeout(limit) is True
    A.step(10)
    B = lbm.Lattice(15, g.xyz, nbr, link, 0.8, rho_mean=g.rho_mean)
    B.step(20)
    assert np.array_equal(A.get_state(), B.get_state())
    assert abs(A.mass() - B.mass()) == 0.0
    assert float(torch.ones(4, device="cuda").sum()) == 4.0
    with pytest.raises(lbm.LbmError):
        lbm.check_wait_timeout(0)
