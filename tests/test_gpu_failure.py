"""Failure detection without a GPU fault: the bounded mbarrier wait of the
table-staged step gives up on a barrier that nothing completes, reports it,
and leaves the device usable (a lattice steps and matches afterwards); the
instability check of lbm_step (a fast site, a NaN in the stored state) and
the input check of lbm_set_populations; the guard words after the planes of
the population buffers (an out-of-range write check)."""
import numpy as np
import pytest

from paper_1906_11925_gb300 import geometry as G
from paper_1906_11925_gb300 import lbm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)


def test_bounded_wait_gives_up_and_device_stays_usable():
    g = G.tube(radius=3, length=8, nx=7, ny=7)
    nbr, link = lbm.links_build(15, g.xyz, g.io_xyz, g.io_id, g.periodic)
    A = lbm.Lattice(15, g.xyz, nbr, link, 0.8, rho_mean=g.rho_mean)
    A.step(10)
    for limit in (1, 64, 4096):
        assert lbm.check_wait_timeout(limit) is True
    A.step(10)
    B = lbm.Lattice(15, g.xyz, nbr, link, 0.8, rho_mean=g.rho_mean)
    B.step(20)
    assert np.array_equal(A.get_state(), B.get_state())
    assert abs(A.mass() - B.mass()) == 0.0
    assert float(torch.ones(4, device="cuda").sum()) == 4.0
    with pytest.raises(lbm.LbmError):
        lbm.check_wait_timeout(0)


FORMS = [(lbm.STORE_FP32, lbm.STREAM_PULL), (lbm.STORE_FP16, lbm.STREAM_PULL),
         (lbm.STORE_FP32, lbm.STREAM_AA), (lbm.STORE_FP16, lbm.STREAM_AA),
         (lbm.STORE_I16, lbm.STREAM_PULL), (lbm.STORE_I16, lbm.STREAM_AA)]


def small(storage=lbm.STORE_FP32, streaming=lbm.STREAM_PULL, q=19, seed=91):
    g = G.random_mask((9, 8, 7), p=0.6, seed=seed, n_iolets=2)
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    # (int16: a coarse scale whose range, 8, holds the fast sites of these tests)
    kw = {"fp16_scale_log2": 12} if storage == lbm.STORE_I16 else {}
    L = lbm.Lattice(q, g.xyz, nbr, link, 0.7, storage=storage, streaming=streaming, rho_mean=g.rho_mean, **kw)
    return g, nbr, link, L


def fast_site_state(q, n, x, ux):
    """Rest populations with site x carrying the equilibrium of speed ux
    along +x (its pre-collision state: the first step keeps rho and j)."""
    f = oracle_rest(q, n)
    c, w = lbm.lattice_vectors(q), f[:, 0].copy()
    cu = c[:, 0] * ux
    f[:, x] = w * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * ux * ux)
    return f


def with_nan(L, storage, i, x):
    """The raw state blob of L with slot (i, x) set to a NaN."""
    blob = L.get_state().copy()
    esz = 4 if storage == lbm.STORE_FP32 else 2
    # fp16: a NaN; int16: the saturation code, which reads as NaN
    nan = {lbm.STORE_FP16: np.array([0x7E00], np.uint16), lbm.STORE_I16: np.array([32767], np.int16),
           lbm.STORE_FP32: np.array([np.nan], np.float32)}[storage]
    npad = (blob.nbytes - 8) // (19 * esz)
    off = (i * npad + x) * esz
    blob[off:off + esz] = nan.view(np.uint8)
    return blob


def oracle_rest(q, n):
    import oracle

    return oracle.rest_state(q, n)


@pytest.mark.parametrize("storage,streaming", FORMS)
def test_stability_check_reports_the_first_failing_range(storage, streaming):
    g, nbr, link, L = small(storage, streaming)
    x = int(np.flatnonzero((link < 2).all(axis=0))[0])  # a site without iolet links
    L.set_populations(fast_site_state(19, g.n, x, 0.45))
    L.set_stability_check(1, u_max=0.3)
    with pytest.raises(lbm.LbmError) as ei:
        L.step(12)
    assert ei.value.name == "LBM_ERR_UNSTABLE"
    assert "times 0 .. 0" in str(ei.value)
    assert L.time == 12  # the steps ran; the check reports after them
    # a looser bound passes
    L.set_stability_check(4, u_max=0.9)
    L.step(8)
    # a NaN spreads and stays: the first check (after 5 steps) fails
    L.set_state(with_nan(L, storage, 3, x))
    L.set_time(0)
    L.set_stability_check(5)
    with pytest.raises(lbm.LbmError) as ei:
        L.step(12)
    assert "times 0 .. 4" in str(ei.value)


@pytest.mark.parametrize("storage,streaming", FORMS)
def test_checked_steps_match_unchecked_bitwise(storage, streaming):
    _, _, _, A = small(storage, streaming)
    _, _, _, B = small(storage, streaming)
    A.set_stability_check(7)
    A.step(75)  # graph chunks between the checks
    B.step(75)
    assert np.array_equal(A.get_state(), B.get_state())
    A.set_stability_check(0)
    A.step(40)
    B.step(40)
    assert np.array_equal(A.get_state(), B.get_state())


@pytest.mark.parametrize("storage", [lbm.STORE_FP32, lbm.STORE_FP16, lbm.STORE_I16])
def test_non_finite_state_is_reported(storage):
    g, nbr, link, L = small(storage)
    f = oracle_rest(19, g.n)
    before = L.get_state()
    out_of_range = {lbm.STORE_FP32: 1e39, lbm.STORE_FP16: 5.0, lbm.STORE_I16: 20.0}[storage]
    for bad in (np.nan, np.inf, out_of_range):
        f2 = f.copy()
        f2[3, 11] = bad
        with pytest.raises(lbm.LbmError) as ei:
            L.set_populations(f2)
        assert ei.value.name == "LBM_ERR_UNSTABLE"
        assert np.array_equal(L.get_state(), before)  # unchanged
    # a NaN that reaches the stored state (a raw blob) is caught by the check
    L.set_state(with_nan(L, storage, 3, 11))
    L.set_stability_check(2)
    with pytest.raises(lbm.LbmError) as ei:
        L.step(2)
    assert ei.value.name == "LBM_ERR_UNSTABLE"


@pytest.mark.parametrize("storage,streaming", FORMS)
def test_guard_words_survive_every_call(storage, streaming):
    g, nbr, link, L = small(storage, streaming, seed=92)
    assert g.n % 128 != 0  # plane padding present
    assert L.check_guards()
    rng = np.random.default_rng(3)
    f0 = oracle_rest(19, g.n) * (1.0 + 0.01 * (2 * rng.random((19, g.n)) - 1))
    L.set_populations(f0)
    L.step(3)
    L.step(70)
    L.macros()
    L.mass()
    L.get_populations()
    w = np.where((link >= 2).any(axis=0), 1.0, 0.0)
    L.objective_grad(lbm.OBJ_DENSITY, w, 9, L.time, L.time + 10, n_snap=3)
    V = lbm.Volume.for_lattice(L)
    V.from_lattice(L, lbm.QTY_SPEED)
    V.close()
    assert L.check_guards()
    # positive control: a state blob whose plane padding differs
    good = L.get_state()
    blob = good.copy()
    esz = 4 if storage == lbm.STORE_FP32 else 2
    blob[g.n * esz:g.n * esz + esz] = 0  # first padding slot of plane 0
    L.set_state(blob)
    assert not L.check_guards()
    L.set_state(good)
    assert L.check_guards()
