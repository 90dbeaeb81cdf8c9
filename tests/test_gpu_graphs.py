"""lbm_step's CUDA-graph chunks (32 steps per replay) against one launch per
step: bitwise the same state in every streaming and storage form, with
time-varying density iolets, velocity iolets and interpolated walls, across
a change of tau (which drops the captured graphs), and when the caller
captures the stream itself; and the driven form with velocity iolets."""
import numpy as np
import pytest

from paper_1906_11925_gb300 import geometry as G
from paper_1906_11925_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

FORMS = [(lbm.STORE_FP32, lbm.STREAM_PULL), (lbm.STORE_FP16, lbm.STREAM_PULL),
         (lbm.STORE_FP32, lbm.STREAM_AA), (lbm.STORE_FP16, lbm.STREAM_AA)]


def case(q, seed=81, velocity=True, bfl=False):
    g = G.random_mask((11, 10, 9), p=0.6, seed=seed, n_iolets=2)
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    rng = np.random.default_rng(seed)
    kw = dict(rho_mean=[1.002, 0.999], amp=[0.001, 0.0005], period=[17.0, 29.0], phase=[0.3, 1.1])
    if velocity:
        # iolet 1 a velocity iolet: its schedule is a speed
        kw.update(rho_mean=[1.002, 0.02], iolet_kind=[0, 1], iolet_normal=[[0, 0, 0], [0.6, 0.0, 0.8]],
                  velocity_weight=0.5 + rng.random(g.n))
    if bfl:
        kw["wall_q"] = np.round(rng.uniform(0.0, 1.0, (q, g.n)) * 2 ** 24).clip(1) / 2 ** 24
    return g, nbr, link, kw


def pair(q, storage, streaming, **ck):
    g, nbr, link, kw = case(q, **ck)
    mk = lambda: lbm.Lattice(q, g.xyz, nbr, link, 0.7, storage=storage, streaming=streaming, **kw)
    return mk(), mk()


@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("storage,streaming", FORMS)
def test_graph_chunks_equal_launch_per_step(q, storage, streaming):
    A, B = pair(q, storage, streaming, bfl=(streaming == lbm.STREAM_PULL and q == 19))
    A.step(3)      # odd: the chunks start from the other buffer / layout
    A.step(100)    # 3 chunks + 4 steps
    A.step(64)
    for _ in range(167):
        B.step(1)
    assert A.time == B.time == 167
    assert np.array_equal(A.get_state(), B.get_state())
    A.set_tau(0.8)
    B.set_tau(0.8)
    A.step(70)
    for _ in range(70):
        B.step(1)
    assert np.array_equal(A.get_state(), B.get_state())
    assert np.isfinite(A.mass())


def test_graph_inside_a_caller_capture():
    """Steps recorded into the caller's own CUDA graph run launch by launch
    (steady iolets: the replayed values repeat)."""
    q = 19
    g = G.random_mask((10, 9, 8), p=0.6, seed=82, n_iolets=2)
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    kw = dict(rho_mean=[1.002, 0.999])
    cs = torch.cuda.Stream()
    A = lbm.Lattice(q, g.xyz, nbr, link, 0.7, stream=cs, **kw)
    B = lbm.Lattice(q, g.xyz, nbr, link, 0.7, **kw)
    A.step(2)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cs):
        A.step(40)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    B.step(2 + 120)
    assert np.array_equal(A.get_populations(), B.get_populations())


@pytest.mark.parametrize("streaming", [lbm.STREAM_PULL, lbm.STREAM_AA])
def test_driven_velocity_iolets_match_schedule(streaming):
    """lbm_step_driven takes the values of a velocity iolet as its speed."""
    q = 15
    g, nbr, link, kw = case(q, seed=83)
    kw.update(amp=[0.0, 0.0])
    A = lbm.Lattice(q, g.xyz, nbr, link, 0.7, streaming=streaming, **kw)
    B = lbm.Lattice(q, g.xyz, nbr, link, 0.7, streaming=streaming, **kw)
    A.step(40)
    B.step_driven(np.tile(kw["rho_mean"], (40, 1)), mass=False)
    assert np.isfinite(A.mass())
    assert np.array_equal(A.get_state(), B.get_state())


def test_set_stream_orders_the_new_stream_after_the_old():
    """Steps queued on a second stream after lbm_set_stream start after the
    steps still queued on the first (no host synchronisation in between)."""
    q = 19
    g, nbr, link, kw = case(q, seed=84)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    A = lbm.Lattice(q, g.xyz, nbr, link, 0.7, stream=s1, **kw)
    B = lbm.Lattice(q, g.xyz, nbr, link, 0.7, **kw)
    A.step(300)
    A.set_stream(s2)
    A.step(45)
    A.set_stream(s1)
    A.step(33)
    B.step(378)
    assert np.array_equal(A.get_state(), B.get_state())
