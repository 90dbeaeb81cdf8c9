"""AA-pattern in-place streaming (one population buffer) against the pull
form and the oracle.  Both forms call the same collision code, so every
population must be bitwise identical after any number of steps, odd or even.
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
PULL, AA = lbm.STREAM_PULL, lbm.STREAM_AA


def make(g, q, tau, storage, streaming, **kw):
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=storage, rho_mean=g.rho_mean, amp=g.amp,
                    period=g.period, phase=g.phase, streaming=streaming, **kw)
    return L, nbr, link


def near_rest(q, n, seed):
    rng = np.random.default_rng(seed)
    return oracle.rest_state(q, n) * (1.0 + 0.01 * (2.0 * rng.random((q, n)) - 1.0))


@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("storage", [FP32, FP16, lbm.STORE_I16])
def test_aa_is_bitwise_equal_to_pull(q, storage):
    g = G.random_mask((10, 9, 8), p=0.6, seed=51, n_iolets=3)
    A, _, _ = make(g, q, 0.66, storage, AA)
    P, _, _ = make(g, q, 0.66, storage, PULL)
    f0 = near_rest(q, g.n, 7)
    A.set_populations(f0)
    P.set_populations(f0)
    for nsteps in (1, 1, 5, 24):  # after 1 (odd), 2 (even), 7 (odd), 31 (odd) steps
        A.step(nsteps)
        P.step(nsteps)
        assert np.array_equal(A.get_populations(), P.get_populations())
        ra, ua, wa = [t.cpu().numpy() for t in A.macros()]
        rp, up, wp = [t.cpu().numpy() for t in P.macros()]
        assert np.array_equal(ra, rp) and np.array_equal(ua, up) and np.array_equal(wa, wp)
        # the mass sums raw slots per site (in float, then float64 over the
        # sites), and the slots of a site are grouped differently in each layout
        assert abs(A.mass() - P.mass()) <= 1e-9 * P.mass()
        assert np.array_equal(A.get_populations_noalloc(), P.get_populations())
    A.step(1)  # even count again
    P.step(1)
    assert np.array_equal(A.get_populations(), P.get_populations())


@pytest.mark.parametrize("storage", [FP32, FP16, lbm.STORE_I16])
def test_aa_tube_poiseuille_1000_steps(storage):
    q, tau = 15, 0.8
    g = G.tube()
    # (int16: the finest scale that holds this flow's deviations, < 8e-4)
    L, nbr, link = make(g, q, tau, storage, AA, **({"fp16_scale_log2": 24} if storage == lbm.STORE_I16 else {}))
    L.step(999)  # ends in the swapped layout
    L.step(1)
    rho, u, _ = [t.cpu().numpy() for t in L.macros()]
    f = oracle.run(q, nbr, link, tau, oracle.rest_state(q, g.n), 1000, geom=g)
    orho, ou, _ = oracle.macros(q, link, tau, f)
    tol = {FP32: 1e-5, FP16: 2e-3, lbm.STORE_I16: 2e-3}[storage]
    assert np.linalg.norm(u - ou) / np.linalg.norm(ou) <= tol
    assert np.linalg.norm(rho - orho) / np.linalg.norm(orho) <= tol


def test_aa_resume_at_odd_phase_is_bit_exact():
    g = G.random_mask((9, 8, 7), p=0.6, seed=52, n_iolets=2)
    q = 19
    A, _, _ = make(g, q, 0.75, FP16, AA)
    B, _, _ = make(g, q, 0.75, FP16, AA)
    f0 = near_rest(q, g.n, 8)
    A.set_populations(f0)
    B.set_populations(f0)
    A.step(30)
    B.step(13)  # odd: swapped layout
    blob, t = B.get_state(), B.time
    C, _, _ = make(g, q, 0.75, FP16, AA)
    C.set_state(blob)
    C.set_time(t)
    C.step(17)
    assert np.array_equal(A.get_state(), C.get_state())
    # a swapped-phase blob is rejected by a pull context
    P, _, _ = make(g, q, 0.75, FP16, PULL)
    with pytest.raises(lbm.LbmError):
        P.set_state(blob)


def test_aa_set_populations_in_swapped_phase():
    g = G.random_mask((8, 8, 8), p=0.55, seed=53, n_iolets=2)
    q = 15
    A, _, _ = make(g, q, 0.7, FP32, AA)
    P, _, _ = make(g, q, 0.7, FP32, PULL)
    A.step(3)  # swapped layout
    A.set_time(0)  # same clock as P: the pulsatile iolets depend on t
    f0 = near_rest(q, g.n, 9)
    A.set_populations(f0)
    P.set_populations(f0)
    assert np.array_equal(A.get_populations(), P.get_populations())
    A.step(4)
    P.step(4)
    assert np.array_equal(A.get_populations(), P.get_populations())


@pytest.mark.parametrize("start_odd", [False, True])
def test_aa_adjoint_equals_pull_adjoint(start_odd):
    g = G.tube(radius=4, length=14, nx=9, ny=9, rho_in=1.002, rho_out=0.999)
    g.amp = np.array([0.001, 0.0])
    g.period = np.array([11.0, 0.0])
    q = 19
    A, nbr, link = make(g, q, 0.7, FP32, AA)
    P, _, _ = make(g, q, 0.7, FP32, PULL)
    pre = 31 if start_odd else 30
    A.step(pre)
    P.step(pre)
    w = (link == 1).any(axis=0).astype(np.float64)
    ra = A.objective_grad(lbm.OBJ_WSS, w, 12, pre + 2, pre + 13, n_snap=3, want_df0=True)
    rp = P.objective_grad(lbm.OBJ_WSS, w, 12, pre + 2, pre + 13, n_snap=3, want_df0=True)
    for k in ("J", "dtau", "dmean", "damp", "dphase", "df0"):
        assert np.array_equal(np.asarray(ra[k]), np.asarray(rp[k])), k
    assert A.time == P.time == pre + 12
    assert np.array_equal(A.get_populations(), P.get_populations())
    A.step(3)
    P.step(3)
    assert np.array_equal(A.get_populations(), P.get_populations())


def test_aa_uses_one_population_buffer():
    g = G.tube()
    A, _, _ = make(g, 19, 0.7, FP32, AA)
    P, _, _ = make(g, 19, 0.7, FP32, PULL)
    ia, ip = A.info(), P.info()
    # one buffer of 19 planes plus its 128 guard slots
    assert ip["device_bytes"] - ia["device_bytes"] == (19 * ip["npad"] + 128) * 4
