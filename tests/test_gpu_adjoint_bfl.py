"""The checkpointed discrete adjoint with interpolated (BFL) walls, on the
GPU through the C ABI, against the FP64 oracle's store-all adjoint
(orc_gradient_bc, pinned to central differences of every parameter).

Interpolated walls couple two sites within one step: a q < 1/2 link of site
x takes (1 - 2q) of the population that its fluid upstream site x + c_p sends
to x.  The GPU sweep keeps that step local: site x stores lam_opp(p) with the
(1 - 2q) lam_p term already added, which the upstream site reads as its lam*
(lbm_adjoint.cu), and dJ/df(t0) has the term taken out again.  Tolerances as
for the half-way walls (relative to the largest entry of each gradient):
fp32 forward 1e-3, fp16-deviation forward 2e-2."""
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
PULL, AA = lbm.STREAM_PULL, lbm.STREAM_AA
TOL = {FP32: 1e-3, FP16: 2e-2}


def rel(a, b):
    a, b = np.atleast_1d(np.asarray(a, np.float64)), np.atleast_1d(np.asarray(b, np.float64))
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def bfl_tube(q, storage, streaming, velocity_inlet=False, tau=0.7, seed=5):
    """A pulsatile tube (radius 4.3, so that most wall links cut the wall away
    from the half-way point) with interpolated walls at the analytic
    cylinder; optionally its inlet a velocity (Ladd) iolet with a parabolic
    weight profile.  The flow is developed for 60 steps by the oracle."""
    g = G.tube(radius=4.3, length=16, nx=11, ny=11, rho_in=1.002, rho_out=0.999)
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    wq = G.wall_fractions(g, lbm.lattice_vectors(q), link)
    io = dict(rho_mean=np.array([1.002, 0.999]), amp=np.array([0.001, 0.0005]),
              period=np.array([9.0, 13.0]), phase=np.array([0.4, 1.3]))
    bc, obc = dict(wall_q=wq), dict(wall_q=wq)
    if velocity_inlet:
        x, y, _ = g.xyz.T.astype(np.float64)
        prof = np.clip(1.0 - ((x - 5.0) ** 2 + (y - 5.0) ** 2) / 18.5, 0.05, None)
        io["rho_mean"] = np.array([0.002, 0.999])
        io["amp"] = np.array([0.0005, 0.0003])
        bc.update(iolet_kind=[1, 0], iolet_normal=[[0.0, 0.0, 1.0], [0.0, 0.0, 0.0]], velocity_weight=prof)
        obc.update(io_kind=np.array([1, 0]), io_normal=np.array(bc["iolet_normal"]), weight=prof)
    L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=storage, streaming=streaming, **io, **bc)
    rng = np.random.default_rng(seed)
    f0 = oracle.rest_state(q, g.n) * (1.0 + 0.002 * (2.0 * rng.random((q, g.n)) - 1.0))
    f0 = oracle.default().run_bc(q, nbr, link, tau, f0, 60, **obc, **io)
    L.set_populations(f0)
    L.set_time(60)
    has_wall = (link == 1).any(axis=0)
    z = g.xyz[:, 2]
    weight = ((z >= 4) & (z < 12) & has_wall).astype(np.float64)
    return g, nbr, link, wq, L, f0, weight, obc, io


@pytest.mark.parametrize("streaming", [PULL, AA])
@pytest.mark.parametrize("q,kind", [(15, lbm.OBJ_WSS), (19, lbm.OBJ_DENSITY), (19, lbm.OBJ_WSS)])
@pytest.mark.parametrize("storage", [FP32, FP16])
def test_bfl_adjoint_matches_oracle(q, kind, storage, streaming):
    """dJ/dtau, the iolet schedule derivatives and dJ/df0 through
    interpolated walls, against the oracle."""
    tau, nsteps = 0.7, 14
    g, nbr, link, wq, L, f0, weight, obc, io = bfl_tube(q, storage, streaming, tau=tau)
    frac = wq[link == 1]
    assert (np.abs(frac - 0.5) > 1e-3).mean() > 0.8 and (frac < 0.5).any() and (frac > 0.5).any()
    tb, te, scale = 63, 75, 1.0 / 12
    got = L.objective_grad(kind, weight, nsteps, tb, te, scale=scale, n_snap=4, want_df0=True)
    ref = oracle.default().gradient(q, nbr, link, tau, f0, nsteps, kind, weight, tb, te, scale=scale,
                                    t0=60, want_lam0=True, **obc, **io)
    errs = {k: rel(got[k], ref[r]) for k, r in (("J", "J"), ("dtau", "dtau"), ("dmean", "dmean"),
                                                 ("damp", "damp"), ("dphase", "dphase"), ("df0", "lam0"))}
    print("bfl adjoint q%d kind %d storage %d streaming %d" % (q, kind, storage, streaming), errs)
    for k, v in errs.items():
        assert v <= TOL[storage], (k, v)


@pytest.mark.parametrize("streaming", [PULL, AA])
def test_bfl_adjoint_with_a_velocity_inlet(streaming):
    """Interpolated walls and a velocity (Ladd) inlet together (D3Q19, WSS)."""
    q, tau, nsteps = 19, 0.7, 12
    g, nbr, link, wq, L, f0, weight, obc, io = bfl_tube(q, FP32, streaming, velocity_inlet=True, tau=tau)
    got = L.objective_grad(lbm.OBJ_WSS, weight, nsteps, 62, 72, n_snap=3, want_df0=True)
    ref = oracle.default().gradient(q, nbr, link, tau, f0, nsteps, lbm.OBJ_WSS, weight, 62, 72, t0=60,
                                    want_lam0=True, **obc, **io)
    assert abs(ref["dmean"][0]) > 0.0
    for k, r in (("J", "J"), ("dtau", "dtau"), ("dmean", "dmean"), ("damp", "damp"), ("dphase", "dphase"),
                 ("df0", "lam0")):
        assert rel(got[k], ref[r]) <= TOL[FP32], (k, rel(got[k], ref[r]))


@pytest.mark.parametrize("storage", [FP32, FP16])
def test_bfl_adjoint_aa_equals_pull(storage):
    """The AA-form sweep gives the pull-form sweep's gradients bit for bit
    with interpolated walls too."""
    outs = []
    for streaming in (PULL, AA):
        g, nbr, link, wq, L, f0, weight, obc, io = bfl_tube(19, storage, streaming)
        outs.append(L.objective_grad(lbm.OBJ_WSS, weight, 15, 62, 76, n_snap=3, want_df0=True))
    for k in ("J", "dtau", "dmean", "damp", "dphase", "df0"):
        assert np.array_equal(np.asarray(outs[0][k]), np.asarray(outs[1][k])), k


def test_bfl_adjoint_matches_central_differences_of_the_gpu_forward():
    """dJ/dtau and dJ/d(inlet mean) of the sweep against central differences
    of J from the GPU's own forward runs (fp32, D3Q19, density objective)."""
    q, tau, nsteps = 19, 0.7, 12
    g, nbr, link, wq, L, f0, weight, obc, io = bfl_tube(q, FP32, PULL, tau=tau)
    got = L.objective_grad(lbm.OBJ_DENSITY, weight, nsteps, 62, 72, scale=0.1, n_snap=3)

    def J(tau_=tau, dmean=0.0):
        io2 = dict(io, rho_mean=io["rho_mean"] + np.array([dmean, 0.0]))
        M = lbm.Lattice(q, g.xyz, nbr, link, tau_, wall_q=wq, **io2)
        M.set_populations(f0)
        M.set_time(60)
        return M.objective_grad(lbm.OBJ_DENSITY, weight, nsteps, 62, 72, scale=0.1, n_snap=3)["J"]

    h = 1e-3
    fd_tau = (J(tau_=tau + h) - J(tau_=tau - h)) / (2 * h)
    fd_mean = (J(dmean=h) - J(dmean=-h)) / (2 * h)
    print("bfl adjoint vs GPU central differences: dtau %.6e / %.6e, dmean %.6e / %.6e"
          % (got["dtau"], fd_tau, got["dmean"][0], fd_mean))
    # (float32 forward runs: the differences carry the forward's rounding,
    # so the bar is 1e-2; the oracle comparison above is the tight one)
    assert abs(got["dtau"] - fd_tau) <= 1e-2 * abs(fd_tau), (got["dtau"], fd_tau)
    assert abs(got["dmean"][0] - fd_mean) <= 1e-2 * abs(fd_mean), (got["dmean"][0], fd_mean)
