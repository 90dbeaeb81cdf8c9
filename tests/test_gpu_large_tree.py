"""The vessel tree at the scale of tens of millions of fluid sites: every
length of the seeded tree x1.86 (root radius 89.28) in a 2048^3 box,
69,461,776 sites, D3Q19.  Its neighbour table holds 19 x 69.5M int32
entries (below the 2^31 limit of the int32 slot offsets).  Checked through
the C ABI:
  - the fused fp32 step (pull streaming) against the FP64 oracle over every
    population, from a perturbed state, relative L2 <= 1e-5;
  - AA-pattern streaming bitwise equal to the pull form in both storage
    forms, after an odd and an even step count."""
import numpy as np
import pytest

from paper_1906_11925_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

Q, TAU = 19, 0.6


@pytest.fixture(scope="module")
def big():
    import bench

    g = bench.make_geometry("vessel_tree_large")
    nbr, link = lbm.links_build(Q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    return g, nbr, link


def lattice(big, storage, streaming):
    g, nbr, link = big
    return lbm.Lattice(Q, g.xyz, nbr, link, TAU, storage=storage, rho_mean=g.rho_mean, amp=g.amp,
                       period=g.period, phase=g.phase, streaming=streaming)


def test_large_tree_shape(big):
    g, nbr, link = big
    assert g.n == 69_461_776
    assert g.n_iolets == 33
    assert Q * ((g.n + 127) // 128 * 128) < 2 ** 31


def test_large_tree_fp32_matches_oracle(big):
    import oracle

    g, nbr, link = big
    rng = np.random.default_rng(12)
    f0 = oracle.rest_state(Q, g.n)
    f0 *= 1.0 + 1e-3 * (2 * rng.random((Q, g.n)) - 1)
    L = lattice(big, lbm.STORE_FP32, lbm.STREAM_PULL)
    L.set_populations(f0)
    L.step(3)
    f = L.get_populations()
    L.close()
    fo = oracle.default().run_bc(Q, nbr, link, TAU, f0, 3, geom=g)
    del f0
    rest = oracle.rest_state(Q, 1)
    f -= rest
    fo -= rest
    e = np.linalg.norm(f - fo) / np.linalg.norm(fo)
    print("tree x1.86 (%d sites), 3 fp32 steps: deviation rel-L2 %.3e" % (g.n, e))
    assert e < 1e-5


@pytest.mark.parametrize("storage", [lbm.STORE_FP32, lbm.STORE_FP16])
def test_large_tree_aa_equals_pull(big, storage):
    A = lattice(big, storage, lbm.STREAM_AA)
    P = lattice(big, storage, lbm.STREAM_PULL)
    for n in (5, 1):  # 5 steps (odd: swapped slots), then 6 (natural layout)
        A.step(n)
        P.step(n)
        assert np.array_equal(A.get_populations(), P.get_populations())
    assert abs(A.mass() - P.mass()) <= 1e-9 * P.mass()
    A.close()
    P.close()


def test_large_tree_pressure_drop_gradient(big):
    """The gradient of the pressure-drop objective at this scale (fp16
    forward, float32 adjoint, float64 accumulation, binomial checkpointing):
    dJ/d(inlet mean density) and dJ/d(mean of one outlet) against central
    differences of the GPU forward (h = 1e-4)."""
    g, nbr, link = big
    L = lattice(big, lbm.STORE_FP16, lbm.STREAM_PULL)
    L.step(200)
    inlet = (link == 2).any(axis=0)
    outlet = (link >= 3).any(axis=0)
    weight = np.where(inlet, 1.0 / (3.0 * inlet.sum()), 0.0) - np.where(outlet, 1.0 / (3.0 * outlet.sum()), 0.0)
    n, t0 = 60, L.time
    state0 = L.get_state()
    sc = 1.0 / (n + 1)
    r = L.objective_grad(lbm.OBJ_DENSITY, weight, n, t0, t0 + n + 1, scale=sc, n_snap=8)

    def J(mean):
        L.set_state(state0)
        L.set_time(t0)
        L.set_iolets(mean, g.amp, g.period, g.phase)
        return L.objective_grad(lbm.OBJ_DENSITY, weight, n, t0, t0 + n + 1, scale=sc, n_snap=8)["J"]

    assert J(g.rho_mean) == r["J"]  # bitwise reproducible
    h = 1e-4
    for k in (0, 7):
        mp, mm = g.rho_mean.copy(), g.rho_mean.copy()
        mp[k] += h
        mm[k] -= h
        d = (J(mp) - J(mm)) / (2 * h)
        print("tree x1.86 gradient: dJ/dmean[%d] %.6e vs FD %.6e" % (k, r["dmean"][k], d))
        assert abs(r["dmean"][k] / d - 1) < 1e-2
    L.close()
