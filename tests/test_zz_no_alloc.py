"""lbm_get_populations_noalloc: the population read-back for callers whose
device memory must not be touched by cudaMalloc/cudaFree (a pool-owning
framework, a fixed memory budget, or a latency-bound loop that cannot afford
the device-wide synchronisation of cudaFree).  It stages the float64 values
in the library's static device array instead of a fresh allocation, so its
output must equal lbm_get_populations' output, call after call.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1906_11925_gb300 import geometry as G
from paper_1906_11925_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

MAX_VALUES = 1 << 20  # capacity of the static array, in float64 values


def _lattice(g, q, storage, seed):
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    L = lbm.Lattice(q, g.xyz, nbr, link, 0.7, storage=storage, rho_mean=g.rho_mean, amp=g.amp,
                    period=g.period, phase=g.phase)
    rng = np.random.default_rng(seed)
    f0 = oracle.rest_state(q, g.n) * (1.0 + 0.01 * (2.0 * rng.random((q, g.n)) - 1.0))
    L.set_populations(f0)
    return L


def _noalloc_via_abi(L):
    """Call the entry point directly through the C ABI."""
    lib = lbm.load_library()
    out = np.full((L.q, L.n), np.nan)
    st = lib.lbm_get_populations_noalloc(L._ctx, out.ctypes.data_as(C.c_void_p))
    assert st == 0, lib.lbm_last_error(L._ctx).decode()
    return out


@pytest.mark.parametrize("storage", [lbm.STORE_FP32, lbm.STORE_FP16])
def test_noalloc_matches_get_populations(storage):
    A = _lattice(G.tube(), 15, storage, seed=1)          # 15 x 12,608 values
    A.step(9)
    ref = A.get_populations()
    first = _noalloc_via_abi(A)
    second = _noalloc_via_abi(A)
    assert np.array_equal(first, ref)
    assert np.array_equal(second, ref)

    # a second context of another lattice and size reuses the same array
    B = _lattice(G.random_mask((9, 8, 7), p=0.6, seed=4, n_iolets=2), 19, storage, seed=2)
    B.step(5)
    refb = B.get_populations()
    assert np.array_equal(_noalloc_via_abi(B), refb)
    assert np.array_equal(_noalloc_via_abi(B), refb)

    # and the first context again, after it has moved on
    A.step(3)
    ref2 = A.get_populations()
    assert not np.array_equal(ref2, ref)
    assert np.array_equal(_noalloc_via_abi(A), ref2)
    assert np.array_equal(A.get_populations_noalloc(), ref2)


def test_noalloc_rejects_sizes_beyond_the_static_array():
    g = G.periodic_box(40, 40, 40)                      # 19 x 64,000 > 2^20 values
    assert 19 * g.n > MAX_VALUES
    L = _lattice(g, 19, lbm.STORE_FP32, seed=3)
    with pytest.raises(lbm.LbmError) as ei:
        L.get_populations_noalloc()
    assert ei.value.name == "LBM_ERR_ARG"
    assert "exceeds the static scratch" in str(ei.value)
    # the context stays usable
    assert L.get_populations().shape == (19, g.n)


def test_noalloc_refuses_a_capturing_stream():
    """The call copies to host memory and waits for the context's stream,
    which cannot be recorded into a CUDA graph: while that stream is being
    captured it returns LBM_ERR_STATE, does nothing, and leaves the capture
    usable."""
    q = 15
    g = G.tube(radius=4, length=12, nx=9, ny=9)
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    cs = torch.cuda.Stream()
    A = lbm.Lattice(q, g.xyz, nbr, link, 0.7, rho_mean=g.rho_mean, stream=cs)
    B = lbm.Lattice(q, g.xyz, nbr, link, 0.7, rho_mean=g.rho_mean)
    A.step(2)
    torch.cuda.synchronize()
    lib = lbm.load_library()
    out = np.full((q, g.n), np.nan)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cs):
        A.step(4)
        st = lib.lbm_get_populations_noalloc(A._ctx, out.ctypes.data_as(C.c_void_p))
    assert st == 6, st  # LBM_ERR_STATE
    assert "captured" in lib.lbm_last_error(A._ctx).decode()
    assert np.isnan(out).all()
    graph.replay()
    torch.cuda.synchronize()
    B.step(6)
    ref = B.get_populations()
    assert np.array_equal(A.get_populations(), ref)
    assert np.array_equal(_noalloc_via_abi(A), ref)
