"""The benchmark's other legs at the full vessel-tree size (10,787,566 sites,
D3Q19) in the configurations the benchmark times:
  - AA-pattern streaming: bitwise equal to the pull form (itself checked
    against the oracle at this size), after an odd and an even step count;
  - the gradient of the pressure-drop objective (fp16-deviation or fp32
    forward, float32 adjoint, binomial checkpointing): dJ/d(inlet mean
    density) against central differences of the GPU forward solver, dJ/dtau
    against central differences of the FP64 oracle, and the AA-form sweep
    bit for bit equal to the pull-form sweep."""
import numpy as np
import pytest

from paper_1906_11925_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

Q, TAU = 19, 0.6


@pytest.fixture(scope="module")
def tree():
    import bench

    g = bench.make_geometry("vessel_tree")
    nbr, link = lbm.links_build(Q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    return g, nbr, link


def lattice(tree, storage, streaming=lbm.STREAM_PULL):
    g, nbr, link = tree
    return lbm.Lattice(Q, g.xyz, nbr, link, TAU, storage=storage, rho_mean=g.rho_mean, amp=g.amp,
                       period=g.period, phase=g.phase, streaming=streaming)


@pytest.mark.parametrize("storage", [lbm.STORE_FP32, lbm.STORE_FP16, lbm.STORE_I16])
def test_aa_equals_pull_on_the_tree(tree, storage):
    A = lattice(tree, storage, lbm.STREAM_AA)
    P = lattice(tree, storage)
    for n in (7, 6):  # 7 (odd, swapped layout), then 13 (odd) ... and an even total below
        A.step(n)
        P.step(n)
        assert np.array_equal(A.get_populations(), P.get_populations())
    A.step(1)
    P.step(1)  # 14 steps: natural layout
    assert np.array_equal(A.get_populations(), P.get_populations())
    assert abs(A.mass() - P.mass()) <= 1e-9 * P.mass()


@pytest.mark.parametrize("storage,tol", [(lbm.STORE_FP32, 5e-4), (lbm.STORE_FP16, 1e-2)])
def test_pressure_drop_gradient_on_the_tree(tree, storage, tol):
    """dJ/d(inlet mean) against central differences of the GPU forward
    (h = 1e-4); dJ/dtau against central differences of the FP64 oracle from
    the same state (h = 1e-6: the float32 forward resolves J's change with
    tau only to ~10 ulps at usable h)."""
    import oracle

    g, nbr, link = tree
    L = lattice(tree, storage)
    L.step(200)  # some flow
    inlet = (link == 2).any(axis=0)
    outlet = (link >= 3).any(axis=0)
    weight = np.where(inlet, 1.0 / (3.0 * inlet.sum()), 0.0) - np.where(outlet, 1.0 / (3.0 * outlet.sum()), 0.0)
    n, t0 = 100, L.time
    state0, f0 = L.get_state(), L.get_populations()
    sc = 1.0 / (n + 1)
    r = L.objective_grad(lbm.OBJ_DENSITY, weight, n, t0, t0 + n + 1, scale=sc, n_snap=16)
    # the AA-form sweep (the benchmark's) gives the same bits at this size
    A = lattice(tree, storage, lbm.STREAM_AA)
    A.step(200)
    ra = A.objective_grad(lbm.OBJ_DENSITY, weight, n, t0, t0 + n + 1, scale=sc, n_snap=16)
    for k in ("J", "dtau", "dmean", "damp", "dphase"):
        assert np.array_equal(np.asarray(ra[k]), np.asarray(r[k])), k
    A.close()

    def J(mean):
        L.set_state(state0)
        L.set_time(t0)
        L.set_iolets(mean, g.amp, g.period, g.phase)
        return L.objective_grad(lbm.OBJ_DENSITY, weight, n, t0, t0 + n + 1, scale=sc, n_snap=16)["J"]

    assert J(g.rho_mean) == r["J"]  # bitwise reproducible
    hm = 1e-4
    mp, mm = g.rho_mean.copy(), g.rho_mean.copy()
    mp[0] += hm
    mm[0] -= hm
    d_mean = (J(mp) - J(mm)) / (2 * hm)
    o = oracle.default()

    def Jo(tau):
        return o.objective_run(Q, nbr, link, tau, f0, n, lbm.OBJ_DENSITY, weight, t0, t0 + n + 1,
                               scale=sc, t0=t0, geom=g)

    ht = 1e-6
    d_tau = (Jo(TAU + ht) - Jo(TAU - ht)) / (2 * ht)
    e_tau, e_mean = abs(r["dtau"] / d_tau - 1), abs(r["dmean"][0] / d_mean - 1)
    print("tree gradient storage %d: dtau %.6e vs %.6e (%.2e), dmean0 %.6e vs %.6e (%.2e)" % (
        storage, r["dtau"], d_tau, e_tau, r["dmean"][0], d_mean, e_mean))
    assert e_tau < tol and e_mean < tol
