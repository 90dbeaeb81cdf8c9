"""Fused AA step pairs over slab chunks (LBM_ORDER_SLABS): each even step and
the odd step after it run as one pass over chunks of whole z planes, the odd
step of a chunk launched two chunks behind the even steps.  The per-site
arithmetic is that of the plain AA kernels and the order only permutes
independent sites, so the populations must equal the other forms' bit for
bit, whatever the step count (fused pairs inside the CUDA-graph chunks, plain
steps around them)."""
import numpy as np
import pytest

from paper_1906_11925_gb300 import geometry as G
from paper_1906_11925_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

STORAGES = [lbm.STORE_FP32, lbm.STORE_FP16, lbm.STORE_I16]


def lattices(g, q, tau, storage, **kw):
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    common = dict(storage=storage, rho_mean=g.rho_mean, amp=g.amp, period=g.period, phase=g.phase, **kw)
    if storage == lbm.STORE_I16:
        common["fp16_scale_log2"] = 24
    S = lbm.Lattice(q, g.xyz, nbr, link, tau, streaming=lbm.STREAM_AA, site_order=lbm.ORDER_SLABS, **common)
    A = lbm.Lattice(q, g.xyz, nbr, link, tau, streaming=lbm.STREAM_AA, **common)
    P = lbm.Lattice(q, g.xyz, nbr, link, tau, streaming=lbm.STREAM_PULL, **common)
    return S, A, P, nbr, link


@pytest.mark.parametrize("storage", STORAGES)
def test_slab_pairs_equal_the_plain_forms_on_the_aneurysm(storage):
    """Pulsatile inlet, D3Q15: a few slab chunks."""
    g = G.aneurysm()
    S, A, P, _, _ = lattices(g, 15, 0.55, storage)
    assert S.slab_chunks() >= 2
    assert A.slab_chunks() == 0 and P.slab_chunks() == 0
    for n in (101, 64, 1):  # t = 101 (swapped), 165 (swapped), 166 (natural)
        for L in (S, A, P):
            L.step(n)
        fs = S.get_populations()
        assert np.array_equal(fs, A.get_populations()), n
        assert np.array_equal(fs, P.get_populations()), n
    assert abs(S.mass() - P.mass()) <= 1e-12 * P.mass()


@pytest.fixture(scope="module")
def tree():
    import bench

    g = bench.make_geometry("vessel_tree")
    return g


@pytest.mark.parametrize("storage", [lbm.STORE_FP32, lbm.STORE_FP16])
def test_slab_pairs_on_the_tree(tree, storage):
    """The benchmark tree (D3Q19, 33 iolets): many chunks, bitwise the plain
    AA form after an odd and an even step count."""
    S, A, P, _, _ = lattices(tree, 19, 0.6, storage)
    del P
    assert S.slab_chunks() >= 10
    for n in (67, 33):
        S.step(n)
        A.step(n)
        assert np.array_equal(S.get_populations(), A.get_populations()), n


@pytest.mark.parametrize("storage", [lbm.STORE_FP32, lbm.STORE_FP16])
def test_row_order_equals_the_default_order_on_the_tree(tree, storage):
    """The benchmark's launch configuration (AA streaming, sites in row order,
    CUDA-graph chunks) gives the default order's populations bit for bit."""
    q = 19
    nbr, link = lbm.links_build(q, tree.xyz, tree.io_xyz, tree.io_id, tree.periodic)
    kw = dict(storage=storage, rho_mean=tree.rho_mean, amp=tree.amp, period=tree.period, phase=tree.phase,
              streaming=lbm.STREAM_AA)
    R = lbm.Lattice(q, tree.xyz, nbr, link, 0.6, site_order=lbm.ORDER_ROWS, **kw)
    A = lbm.Lattice(q, tree.xyz, nbr, link, 0.6, **kw)
    for n in (67, 33):  # two graph chunks and three single steps, then one chunk and one step
        R.step(n)
        A.step(n)
        assert np.array_equal(R.get_populations(), A.get_populations()), n
    # (the mass sums the same values in another order)
    assert abs(R.mass() - A.mass()) <= 1e-12 * A.mass()


def test_slab_pairs_with_interpolated_walls(tree):
    """Interpolated walls (their sites run in the unfused tail launches) on
    the tree: bitwise the pull form."""
    import bench

    q = 19
    nbr, link = lbm.links_build(q, tree.xyz, tree.io_xyz, tree.io_id, tree.periodic)
    wq = bench.wall_fractions_cached(tree, q, link)
    kw = dict(rho_mean=tree.rho_mean, wall_q=wq)
    S = lbm.Lattice(q, tree.xyz, nbr, link, 0.6, streaming=lbm.STREAM_AA, site_order=lbm.ORDER_SLABS, **kw)
    P = lbm.Lattice(q, tree.xyz, nbr, link, 0.6, streaming=lbm.STREAM_PULL, **kw)
    assert S.slab_chunks() >= 10
    S.step(70)
    P.step(70)
    assert np.array_equal(S.get_populations(), P.get_populations())


def test_periodic_z_runs_unfused():
    """A periodic z axis puts neighbours many chunks apart: no fused pairs,
    and the steps still match."""
    g = G.periodic_box(64, 64, 200)  # four or more chunks: the wrap is three apart
    q = 19
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    rng = np.random.default_rng(1)
    import oracle

    f0 = oracle.rest_state(q, g.n) * (1.0 + 0.01 * (2 * rng.random((q, g.n)) - 1))
    S = lbm.Lattice(q, g.xyz, nbr, link, 0.7, streaming=lbm.STREAM_AA, site_order=lbm.ORDER_SLABS)
    A = lbm.Lattice(q, g.xyz, nbr, link, 0.7, streaming=lbm.STREAM_AA)
    assert S.slab_chunks() == 0
    S.set_populations(f0)
    A.set_populations(f0)
    S.step(40)
    A.step(40)
    assert np.array_equal(S.get_populations(), A.get_populations())
