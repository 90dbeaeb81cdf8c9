"""The adjoint sweep of an AA-form context (AA-form forward recomputation,
AA-form adjoint steps in place on one buffer): J, every gradient, dJ/df(t0)
and the final state bit for bit those of the pull-form sweep on the same
state, for both start phases of the AA buffer, odd and even step counts,
several snapshot counts, both storage forms and both objectives (the pull
form's sweep is checked against the FP64 oracle in test_gpu_adjoint.py)."""
import numpy as np
import pytest

import oracle
from paper_1906_11925_gb300 import geometry as G
from paper_1906_11925_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

KEYS = ("J", "dtau", "dmean", "damp", "dphase", "df0")


def contexts(q, storage, pre, seed=5):
    g = G.tube(radius=4, length=16, nx=9, ny=9, rho_in=1.002, rho_out=0.999)
    amp, period, phase = [0.001, 0.0005], [9.0, 13.0], [0.4, 1.3]
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    rng = np.random.default_rng(seed)
    f0 = oracle.rest_state(q, g.n) * (1.0 + 0.002 * (2.0 * rng.random((q, g.n)) - 1.0))
    f0 = oracle.run(q, nbr, link, 0.7, f0, 60, geom=g)
    out = []
    for streaming in (lbm.STREAM_AA, lbm.STREAM_PULL):
        L = lbm.Lattice(q, g.xyz, nbr, link, 0.7, storage=storage, streaming=streaming, rho_mean=g.rho_mean,
                        amp=amp, period=period, phase=phase)
        L.set_populations(f0)
        L.set_time(60)
        L.step(pre)  # pre odd: the AA buffer starts the sweep in its swapped phase
        out.append(L)
    has_wall = (link == 1).any(axis=0)
    z = g.xyz[:, 2]
    weight = ((z >= 4) & (z < 12) & has_wall).astype(np.float64)
    return out[0], out[1], weight


@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("storage", [lbm.STORE_FP32, lbm.STORE_FP16, lbm.STORE_I16])
@pytest.mark.parametrize("kind", [lbm.OBJ_WSS, lbm.OBJ_DENSITY])
@pytest.mark.parametrize("pre", [0, 1])
def test_aa_sweep_equals_pull_sweep(q, storage, kind, pre):
    A, P, weight = contexts(q, storage, pre)
    for nsteps, n_snap in ((13, 3), (14, 1), (9, 15), (14, 4)):
        t0 = A.time
        tb, te = t0 + 2, t0 + nsteps + 1
        a = A.objective_grad(kind, weight, nsteps, tb, te, scale=0.1, n_snap=n_snap, want_df0=True)
        p = P.objective_grad(kind, weight, nsteps, tb, te, scale=0.1, n_snap=n_snap, want_df0=True)
        for k in KEYS:
            assert np.array_equal(np.asarray(a[k]), np.asarray(p[k])), (nsteps, n_snap, k)
        assert A.adjoint_counts() == P.adjoint_counts()
        assert A.time == P.time == t0 + nsteps
        assert np.array_equal(A.get_populations(), P.get_populations())
    A.step(5)  # the AA phase after the sweeps
    P.step(5)
    assert np.array_equal(A.get_populations(), P.get_populations())


@pytest.mark.parametrize("pre", [0, 1])
def test_aa_zero_steps_and_one_step(pre):
    A, P, weight = contexts(19, lbm.STORE_FP32, pre)
    for nsteps in (0, 1, 2):
        t0 = A.time
        a = A.objective_grad(lbm.OBJ_DENSITY, weight, nsteps, t0, t0 + nsteps + 1, scale=2.0, want_df0=True)
        p = P.objective_grad(lbm.OBJ_DENSITY, weight, nsteps, t0, t0 + nsteps + 1, scale=2.0, want_df0=True)
        for k in KEYS:
            assert np.array_equal(np.asarray(a[k]), np.asarray(p[k])), (nsteps, k)
        assert np.array_equal(A.get_populations(), P.get_populations())
