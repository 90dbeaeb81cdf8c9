"""Velocity (Ladd) iolets with a per-site velocity profile on the GPU against
the FP64 oracle (pulsatile parabolic inlet into a tube, density outlet)."""
import numpy as np
import pytest

import oracle
from paper_1906_11925_gb300 import geometry as G
from paper_1906_11925_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

FP32, FP16 = lbm.STORE_FP32, lbm.STORE_FP16
TOL = {FP32: 1e-5, FP16: 2e-3}


def setup(q):
    g = G.tube(radius=6, length=24, nx=13, ny=13, rho_in=1.0, rho_out=1.0)
    # iolet 0 (z = -1): velocity inlet along +z, U(t) = 0.004 + 0.002 sin(2 pi t / 50)
    g.rho_mean = np.array([0.004, 1.0])
    g.amp = np.array([0.002, 0.0])
    g.period = np.array([50.0, 0.0])
    g.phase = np.array([0.3, 0.0])
    x, y, z = g.xyz.T
    r2 = (x - 6.0) ** 2 + (y - 6.0) ** 2
    weight = np.clip(2.0 * (1.0 - r2 / 36.0), 0.0, None)  # parabolic profile, mean ~1
    kind = np.array([lbm.IOLET_VELOCITY, lbm.IOLET_DENSITY], np.int32)
    normal = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 0.0]])
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    return g, nbr, link, weight, kind, normal


@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("storage", [FP32, FP16])
@pytest.mark.parametrize("streaming", [lbm.STREAM_PULL, lbm.STREAM_AA])
def test_velocity_inlet_matches_oracle(q, storage, streaming):
    tau, steps = 0.7, 301
    g, nbr, link, weight, kind, normal = setup(q)
    L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=storage, rho_mean=g.rho_mean, amp=g.amp,
                    period=g.period, phase=g.phase, iolet_kind=kind, iolet_normal=normal,
                    velocity_weight=weight, streaming=streaming)
    L.step(steps)
    rho, u, _ = [t.cpu().numpy() for t in L.macros()]
    f = oracle.default().run_bc(q, nbr, link, tau, oracle.rest_state(q, g.n), steps, io_kind=kind,
                                io_normal=normal, weight=weight, geom=g)
    orho, ou, _ = oracle.macros(q, link, tau, f)
    eu = np.linalg.norm(u - ou) / np.linalg.norm(ou)
    er = np.linalg.norm(rho - orho) / np.linalg.norm(orho)
    print("velocity iolet", q, storage, streaming, eu, er)
    assert eu <= TOL[storage] and er <= TOL[storage]
    assert ou[:, 2].mean() > 1e-3  # the inlet really drives a flow


def test_velocity_iolet_gradient_runs_and_matches_its_own_finite_difference():
    """lbm_objective_grad differentiates velocity iolets (the oracle check is
    in test_gpu_adjoint.py): dJ/d(mean speed) against central differences of
    the GPU forward run."""
    q = 15
    g, nbr, link, weight, kind, normal = setup(q)
    io = dict(rho_mean=np.array(g.rho_mean, np.float64), amp=g.amp, period=g.period, phase=g.phase)
    bc = dict(iolet_kind=kind, iolet_normal=normal, velocity_weight=weight)

    def J(mean):
        io2 = dict(io, rho_mean=mean)
        L = lbm.Lattice(q, g.xyz, nbr, link, 0.7, **io2, **bc)
        r = L.objective_grad(lbm.OBJ_DENSITY, np.ones(g.n), 12, 0, 13, scale=1.0 / 13)
        return r

    r = J(io["rho_mean"])
    k = int(np.flatnonzero(np.asarray(kind) == 1)[0])
    h = 1e-3
    mp, mm = io["rho_mean"].copy(), io["rho_mean"].copy()
    mp[k] += h
    mm[k] -= h
    fd = (J(mp)["J"] - J(mm)["J"]) / (2 * h)
    assert abs(r["dmean"][k] - fd) <= 1e-2 * abs(fd), (r["dmean"][k], fd)
