"""The checkpointed discrete adjoint on the GPU (lbm_objective_grad) against
the FP64 oracle's store-all adjoint (itself pinned to central differences).

Tolerances (relative to the largest entry of each gradient): fp32 forward
with float32 adjoint 1e-3; fp16-deviation forward 2e-2.
"""
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
TOL = {FP32: 1e-3, FP16: 2e-2}


def pulsatile_tube():
    g = G.tube(radius=4, length=16, nx=9, ny=9, rho_in=1.002, rho_out=0.999)
    g.amp = np.array([0.001, 0.0005])
    g.period = np.array([9.0, 13.0])
    g.phase = np.array([0.4, 1.3])
    return g


def setup(q, storage, tau=0.7, seed=3):
    g = pulsatile_tube()
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=storage, rho_mean=g.rho_mean, amp=g.amp,
                    period=g.period, phase=g.phase)
    rng = np.random.default_rng(seed)
    f0 = oracle.rest_state(q, g.n) * (1.0 + 0.002 * (2.0 * rng.random((q, g.n)) - 1.0))
    # let the flow develop so that the wall shear stress is well away from 0
    f0 = oracle.run(q, nbr, link, tau, f0, 60, geom=g)
    L.set_populations(f0)
    L.set_time(60)
    x, y, z = g.xyz.T
    has_wall = (link == 1).any(axis=0)
    weight = ((z >= 4) & (z < 12) & has_wall).astype(np.float64)
    return g, nbr, link, L, f0, weight


def rel(a, b):
    a, b = np.atleast_1d(np.asarray(a, np.float64)), np.atleast_1d(np.asarray(b, np.float64))
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("storage", [FP32, FP16])
@pytest.mark.parametrize("kind", [lbm.OBJ_WSS, lbm.OBJ_DENSITY])
def test_adjoint_matches_oracle(q, storage, kind):
    tau, nsteps = 0.7, 14
    g, nbr, link, L, f0, weight = setup(q, storage, tau)
    t0, tb, te, scale = 60, 63, 75, 1.0 / 12
    got = L.objective_grad(kind, weight, nsteps, tb, te, scale=scale, n_snap=4, want_df0=True)
    ref = oracle.default().gradient(q, nbr, link, tau, f0, nsteps, kind, weight, tb, te, scale=scale,
                                    t0=t0, geom=g, want_lam0=True)
    errs = dict(J=rel(got["J"], ref["J"]), dtau=rel(got["dtau"], ref["dtau"]),
                dmean=rel(got["dmean"], ref["dmean"]), damp=rel(got["damp"], ref["damp"]),
                dphase=rel(got["dphase"], ref["dphase"]), df0=rel(got["df0"], ref["lam0"]))
    print("adjoint", q, storage, kind, errs)
    for k, v in errs.items():
        assert v <= TOL[storage], (k, v)
    assert L.time == t0 + nsteps


def test_adjoint_does_not_depend_on_snapshot_count():
    q = 19
    outs = []
    for n_snap in (1, 2, 3, 5, 15):
        g, nbr, link, L, f0, weight = setup(q, FP32)
        outs.append(L.objective_grad(lbm.OBJ_WSS, weight, 14, 61, 75, n_snap=n_snap, want_df0=True))
        fw, ad = L.adjoint_counts()
        assert fw == lbm.revolve_steps(14, n_snap) and ad == 14
    for o in outs[1:]:
        for k in ("J", "dtau", "dmean", "damp", "dphase", "df0"):
            assert np.array_equal(np.asarray(o[k]), np.asarray(outs[0][k])), k


@pytest.mark.parametrize("storage", [FP32, FP16])
def test_adjoint_leaves_the_final_state(storage):
    q = 15
    g, nbr, link, A, f0, weight = setup(q, storage)
    g, nbr, link, B, f0, weight = setup(q, storage)
    A.objective_grad(lbm.OBJ_DENSITY, weight, 23, 60, 90, n_snap=3)
    B.step(23)
    assert A.time == B.time == 83
    assert np.array_equal(A.get_state(), B.get_state())


def test_zero_steps_is_the_explicit_term():
    q = 19
    g, nbr, link, L, f0, weight = setup(q, FP32)
    got = L.objective_grad(lbm.OBJ_DENSITY, weight, 0, 60, 61, scale=2.0, want_df0=True)
    rho, _, _ = oracle.macros(q, link, 0.7, f0)
    assert rel(got["J"], 2.0 * np.sum(weight * rho)) <= 1e-6
    assert np.allclose(got["df0"], 2.0 * weight[None, :].repeat(q, 0))
    assert got["dtau"] == 0.0 and np.all(got["dmean"] == 0.0)


def test_autograd_function_matches_objective_grad():
    q = 15
    g, nbr, link, L, f0, weight = setup(q, FP32)
    obj = lbm.HemeObjective(L, lbm.OBJ_WSS, weight, 10, 62, 71, scale=0.1, n_snap=3)
    tau = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
    mean = torch.tensor(g.rho_mean, requires_grad=True)
    amp = torch.tensor(g.amp, requires_grad=True)
    phase = torch.tensor(g.phase, requires_grad=True)
    J = obj(tau, mean, amp, phase)
    (3.0 * J).backward()
    ref = obj.evaluate(0.7, g.rho_mean, g.amp, g.phase)
    assert float(J.detach()) == ref["J"]
    assert float(tau.grad) == 3.0 * ref["dtau"]
    assert np.array_equal(mean.grad.numpy(), 3.0 * ref["dmean"])
    assert np.array_equal(amp.grad.numpy(), 3.0 * ref["damp"])
    assert np.array_equal(phase.grad.numpy(), 3.0 * ref["dphase"])


def velocity_inlet_tube(q, storage, streaming, tau=0.7, seed=4):
    """The pulsatile tube with its inlet (iolet 0) a velocity iolet: a
    parabolic weight profile across the inlet sites, speed schedule
    0.002 + 0.0005 sin(2 pi t / 9 + 0.4) along the inward normal +z."""
    g = pulsatile_tube()
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    x, y, z = g.xyz.T.astype(np.float64)
    prof = np.clip(1.0 - ((x - 4.0) ** 2 + (y - 4.0) ** 2) / 20.25, 0.05, None)
    bc = dict(iolet_kind=[1, 0], iolet_normal=[[0.0, 0.0, 1.0], [0.0, 0.0, 0.0]], velocity_weight=prof)
    io = dict(rho_mean=np.array([0.002, 0.999]), amp=np.array([0.0005, 0.0003]),
              period=np.array([9.0, 13.0]), phase=np.array([0.4, 1.3]))
    L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=storage, streaming=streaming, **io, **bc)
    rng = np.random.default_rng(seed)
    f0 = oracle.rest_state(q, g.n) * (1.0 + 0.002 * (2.0 * rng.random((q, g.n)) - 1.0))
    obc = dict(io_kind=np.array([1, 0]), io_normal=np.array(bc["iolet_normal"]), weight=prof)
    f0 = oracle.default().run_bc(q, nbr, link, tau, f0, 60, **obc, **io)
    L.set_populations(f0)
    L.set_time(60)
    has_wall = (link == 1).any(axis=0)
    weight = ((z >= 4) & (z < 12) & has_wall).astype(np.float64)
    return g, nbr, link, L, f0, weight, obc, io


@pytest.mark.parametrize("streaming", [lbm.STREAM_PULL, lbm.STREAM_AA])
@pytest.mark.parametrize("q,kind", [(15, lbm.OBJ_WSS), (19, lbm.OBJ_DENSITY)])
@pytest.mark.parametrize("storage", [FP32, FP16])
def test_adjoint_with_a_velocity_iolet_matches_oracle(q, kind, storage, streaming):
    """Gradients through a velocity (Ladd) inlet: dJ/dtau and the derivatives
    with respect to the inlet's speed schedule (mean, amp, phase) and the
    outlet's density schedule, and dJ/df0, against the FP64 oracle."""
    tau, nsteps = 0.7, 14
    g, nbr, link, L, f0, weight, obc, io = velocity_inlet_tube(q, storage, streaming, tau)
    t0, tb, te, scale = 60, 63, 75, 1.0 / 12
    got = L.objective_grad(kind, weight, nsteps, tb, te, scale=scale, n_snap=4, want_df0=True)
    ref = oracle.default().gradient(q, nbr, link, tau, f0, nsteps, kind, weight, tb, te, scale=scale,
                                    t0=t0, want_lam0=True, **obc, **io)
    errs = dict(J=rel(got["J"], ref["J"]), dtau=rel(got["dtau"], ref["dtau"]),
                dmean=rel(got["dmean"], ref["dmean"]), damp=rel(got["damp"], ref["damp"]),
                dphase=rel(got["dphase"], ref["dphase"]), df0=rel(got["df0"], ref["lam0"]))
    print("velocity-iolet adjoint", q, storage, kind, streaming, errs, "dU/dmean", ref["dmean"][0])
    assert abs(ref["dmean"][0]) > 0.0
    for k, v in errs.items():
        assert v <= TOL[storage], (k, v)


@pytest.mark.parametrize("storage", [FP32, FP16])
def test_velocity_iolet_adjoint_aa_equals_pull(storage):
    """The AA-form sweep gives the pull-form sweep's gradients bit for bit
    with a velocity inlet too."""
    q = 19
    outs = []
    for streaming in (lbm.STREAM_PULL, lbm.STREAM_AA):
        g, nbr, link, L, f0, weight, obc, io = velocity_inlet_tube(q, storage, streaming)
        outs.append(L.objective_grad(lbm.OBJ_WSS, weight, 15, 62, 76, n_snap=3, want_df0=True))
    for k in ("J", "dtau", "dmean", "damp", "dphase", "df0"):
        assert np.array_equal(np.asarray(outs[0][k]), np.asarray(outs[1][k])), k
