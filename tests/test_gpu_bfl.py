"""Interpolated (BFL) walls on the GPU against the FP64 oracle, through the
C ABI, in both streaming forms (pull and the in-place AA pattern, which must
agree bit for bit).  Tolerances as for the half-way walls: relative L2 <=
1e-5 with fp32 storage, <= 2e-3 with fp16-deviation storage."""
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
TOL = {FP32: 1e-5, FP16: 2e-3}


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def tube_case(q):
    g = G.tube(radius=5.3, length=24, nx=13, ny=13, rho_in=1.002, rho_out=0.999)
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    wq = G.wall_fractions(g, lbm.lattice_vectors(q), link)
    return g, nbr, link, wq


@pytest.mark.parametrize("streaming", [PULL, AA])
@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("storage", [FP32, FP16])
def test_bfl_tube_matches_oracle(q, storage, streaming):
    g, nbr, link, wq = tube_case(q)
    assert ((wq[link == 1] != 0.5).mean()) > 0.9
    tau, steps = 0.7, 300
    L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=storage, rho_mean=g.rho_mean, wall_q=wq,
                    streaming=streaming)
    L.step(steps)
    f = L.get_populations()
    rho, u, wss = [t.cpu().numpy() for t in L.macros()]
    mass = L.mass()
    o = oracle.default()
    fo = o.run_bc(q, nbr, link, tau, o.rest_state(q, g.n), steps, wall_q=wq, geom=g)
    orho, ou, owss = o.macros(q, link, tau, fo)
    rest = oracle.rest_state(q, g.n)
    print("tube q%d storage %d streaming %d: f dev %.3e u %.3e rho %.3e wss %.3e" % (
        q, storage, streaming, rel(f - rest, fo - rest), rel(u, ou), rel(rho, orho), rel(wss, owss)))
    assert rel(f - rest, fo - rest) < TOL[storage]
    assert rel(u, ou) < TOL[storage], rel(u, ou)
    assert rel(rho, orho) < TOL[storage]
    assert rel(wss, owss) < TOL[storage], rel(wss, owss)
    assert abs(mass / o.mass(fo) - 1.0) < 1e-6


@pytest.mark.parametrize("streaming", [PULL, AA])
@pytest.mark.parametrize("q", [15, 19])
def test_bfl_random_mask_with_both_iolet_kinds(q, streaming):
    """Random walls with random fractions (thin gaps, q < 1/2 links without
    an upstream fluid site), a density iolet and a velocity iolet."""
    g = G.random_mask((9, 8, 7), p=0.6, seed=71, n_iolets=2)
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    rng = np.random.default_rng(9)
    wq = np.round(rng.uniform(0.0, 1.0, (q, g.n)) * 2 ** 24).clip(1) / 2 ** 24
    kind = [0, 1]
    nrm = [[0, 0, 0], [0.6, 0.0, 0.8]]
    w = 0.5 + rng.random(g.n)
    mean, amp, period, phase = [1.001, 0.002], [0.0005, 0.001], [17.0, 23.0], [0.1, 0.4]
    f0 = oracle.rest_state(q, g.n) * (1.0 + 0.01 * (2 * rng.random((q, g.n)) - 1))
    L = lbm.Lattice(q, g.xyz, nbr, link, 0.65, rho_mean=mean, amp=amp, period=period, phase=phase,
                    iolet_kind=kind, iolet_normal=nrm, velocity_weight=w, wall_q=wq, streaming=streaming)
    L.set_populations(f0)
    assert rel(L.get_populations(), f0) < 1e-7
    L.step(20)
    fo = oracle.default().run_bc(q, nbr, link, 0.65, f0, 20, io_kind=kind, io_normal=nrm, weight=w,
                                 wall_q=wq, rho_mean=mean, amp=amp, period=period, phase=phase)
    f = L.get_populations()
    d, do = f - oracle.rest_state(q, g.n), fo - oracle.rest_state(q, g.n)
    assert rel(d, do) < 1e-5, rel(d, do)
    assert abs(L.mass() / oracle.mass(fo) - 1.0) < 1e-7


def test_bfl_at_half_is_halfway_bitwise():
    g = G.random_mask((8, 7, 6), p=0.6, seed=72, n_iolets=2)
    q = 19
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    A = lbm.Lattice(q, g.xyz, nbr, link, 0.7, rho_mean=g.rho_mean, wall_q=np.full((q, g.n), 0.5))
    B = lbm.Lattice(q, g.xyz, nbr, link, 0.7, rho_mean=g.rho_mean)
    A.step(25)
    B.step(25)
    assert np.array_equal(A.get_state(), B.get_state())


def test_bfl_links_state_and_adjoint():
    g, nbr, link, wq = tube_case(15)
    L = lbm.Lattice(15, g.xyz, nbr, link, 0.7, rho_mean=g.rho_mean, wall_q=wq)
    n2, l2 = L.get_links()
    assert np.array_equal(n2, nbr) and np.array_equal(l2, link)
    L.step(10)
    blob, t = L.get_state(), L.time
    L.step(7)
    M = lbm.Lattice(15, g.xyz, nbr, link, 0.7, rho_mean=g.rho_mean, wall_q=wq)
    M.set_state(blob)
    M.set_time(t)
    M.step(7)
    assert np.array_equal(L.get_state(), M.get_state())
    # (the adjoint of interpolated walls: tests/test_gpu_adjoint_bfl.py)
    r = L.objective_grad(lbm.OBJ_DENSITY, np.ones(g.n), 5, L.time, L.time + 5)
    assert np.isfinite(r["J"]) and np.isfinite(r["dtau"])


def test_bfl_vessel_tree_full_size():
    """The benchmark's interpolated-wall workload: the vessel tree with the
    wall fractions of its analytic shape, five steps from a perturbed state,
    every population against the oracle."""
    import bench

    g = bench.make_geometry("vessel_tree")
    q, tau = 19, 0.6
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    wq = bench.wall_fractions_cached(g, q, link)
    rng = np.random.default_rng(11)
    f0 = oracle.rest_state(q, g.n) * (1.0 + 1e-3 * (2 * rng.random((q, g.n)) - 1))
    L = lbm.Lattice(q, g.xyz, nbr, link, tau, rho_mean=g.rho_mean, wall_q=wq)
    L.set_populations(f0)
    L.step(5)
    f = L.get_populations()
    L.close()
    A = lbm.Lattice(q, g.xyz, nbr, link, tau, rho_mean=g.rho_mean, wall_q=wq, streaming=AA)
    A.set_populations(f0)
    A.step(5)
    assert np.array_equal(A.get_populations(), f)  # the AA form, bit for bit
    A.close()
    fo = oracle.default().run_bc(q, nbr, link, tau, f0, 5, wall_q=wq, geom=g)
    rest = oracle.rest_state(q, 1)
    e = rel(f - rest, fo - rest)
    print("vessel tree BFL, 5 steps: deviation rel-L2 %.3e" % e)
    assert e < 1e-5


@pytest.mark.parametrize("streaming", [PULL, AA])
@pytest.mark.parametrize("qv", [1.0, 2.0 ** -24, 0.5 - 2.0 ** -24, 0.5 + 2.0 ** -24])
def test_bfl_extreme_fractions(qv, streaming):
    """Every wall at the same fraction: at the far end of the link (q = 1),
    at the site itself (q = 2^-24), and just either side of 1/2."""
    q = 19
    g = G.random_mask((8, 7, 6), p=0.65, seed=73, n_iolets=2)
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    wq = np.full((q, g.n), qv)
    rng = np.random.default_rng(5)
    f0 = oracle.rest_state(q, g.n) * (1.0 + 0.01 * (2 * rng.random((q, g.n)) - 1))
    L = lbm.Lattice(q, g.xyz, nbr, link, 0.7, rho_mean=g.rho_mean, amp=g.amp, period=g.period,
                    phase=g.phase, wall_q=wq, streaming=streaming)
    L.set_populations(f0)
    L.step(15)
    fo = oracle.default().run_bc(q, nbr, link, 0.7, f0, 15, wall_q=wq, geom=g)
    rest = oracle.rest_state(q, g.n)
    assert rel(L.get_populations() - rest, fo - rest) < 1e-5


@pytest.mark.parametrize("storage", [FP32, FP16])
@pytest.mark.parametrize("q", [15, 19])
def test_bfl_aa_equals_pull_bitwise(q, storage):
    """Interpolated walls with both iolet kinds: the AA form gives the pull
    form's populations bit for bit after odd and even step counts, and its
    mass and fields agree; a state blob of the AA form resumes exactly."""
    g = G.random_mask((9, 8, 7), p=0.6, seed=74, n_iolets=2)
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    rng = np.random.default_rng(12)
    wq = np.round(rng.uniform(0.0, 1.0, (q, g.n)) * 2 ** 24).clip(1) / 2 ** 24
    kw = dict(rho_mean=[1.001, 0.002], amp=[0.0005, 0.001], period=[17.0, 23.0], phase=[0.1, 0.4],
              iolet_kind=[0, 1], iolet_normal=[[0, 0, 0], [0.6, 0.0, 0.8]],
              velocity_weight=0.5 + rng.random(g.n), wall_q=wq, storage=storage)
    f0 = oracle.rest_state(q, g.n) * (1.0 + 0.01 * (2 * rng.random((q, g.n)) - 1))
    P = lbm.Lattice(q, g.xyz, nbr, link, 0.66, streaming=PULL, **kw)
    A = lbm.Lattice(q, g.xyz, nbr, link, 0.66, streaming=AA, **kw)
    P.set_populations(f0)
    A.set_populations(f0)
    for n in (1, 6, 33, 40):  # t = 1, 7 (swapped layouts), 40, 80 (natural)
        P.step(n)
        A.step(n)
        assert np.array_equal(A.get_populations(), P.get_populations()), n
    # (the mass sums each site's raw slots in float, in the order the layout
    # holds them: the two agree to that summation's rounding, at most q
    # roundings of 2^-24 of the summed deviations)
    dev = P.get_populations() - oracle.rest_state(q, g.n)
    assert abs(A.mass() - P.mass()) <= q * 2.0 ** -24 * np.abs(dev).sum()
    ra, ua, wa = [t.cpu().numpy() for t in A.macros()]
    rp, up, wp = [t.cpu().numpy() for t in P.macros()]
    assert np.array_equal(ra, rp) and np.array_equal(ua, up) and np.array_equal(wa, wp)
    A.step(3)
    blob, t = A.get_state(), A.time
    A.step(4)
    B = lbm.Lattice(q, g.xyz, nbr, link, 0.66, streaming=AA, **kw)
    B.set_state(blob)
    B.set_time(t)
    B.step(4)
    assert np.array_equal(A.get_state(), B.get_state())
