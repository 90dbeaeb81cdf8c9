"""Ray-marched volume rendering (Section 3.3.2) on the GPU against the FP64
oracle's renderer, through the C ABI.

Tolerances (float32 kernel against the float64 oracle):
  - FILTER_EXACT (float32 trilinear weights): the sample positions carry a
    relative error of a few 2^-24 of the ray length (< 200 voxels here), i.e.
    < 1e-4 voxels; with volume gradients < 0.2 per voxel, transfer scales <= 2
    and LUT slopes < 2 per unit s, a sample's colour moves by < 1e-4 and a
    pixel (a convex combination of them, plus opacity terms of the same size)
    by < 2e-4.  Tests: max |diff| <= 2e-4, relative L2 <= 5e-5.
  - FILTER_TEXTURE: the texture unit quantises each trilinear weight to 1/256,
    so a sample moves by up to 3 x 2^-9 x (largest voxel step, < 0.2) ~ 1.2e-3
    in value, x scale x LUT slope (< 4) ~ 5e-3 in colour.  Tests: max |diff|
    <= 1e-2, relative L2 <= 3e-3.
  - Early termination (a_stop < 1) is a threshold on A: where A crosses it
    within rounding the two sides stop one sample apart, which changes the
    pixel by at most 1 - a_stop; such pixels must be rare.
The empty-brick skipping must leave the image bitwise unchanged.
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


def blobs(shape, k, seed, sparse=False):
    """Sum of k Gaussian blobs (sigma 1.5..4 voxels) in a [nz, ny, nx] box;
    sparse: values below 0.05 are set to exactly 0."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v = np.zeros(shape)
    for _ in range(k):
        c = rng.random(3) * [nx, ny, nz]
        s = 1.5 + 2.5 * rng.random()
        v += rng.random() * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * s * s))
    v = v / v.max()
    if sparse:
        v[v < 0.05] = 0.0
    return v.astype(np.float32)


def upload(vol_np):
    nz, ny, nx = vol_np.shape
    V = lbm.Volume(nx, ny, nz)
    V.upload(torch.from_numpy(vol_np).cuda())
    return V


def view_kwargs(view):
    return dict(eye=view.eye, center=view.center, up=view.up, fov_y=view.fov_y, dt=view.dt,
                tf_scale=view.tf_scale, tf_offset=view.tf_offset, lut=view.lut, a_stop=view.a_stop)


def oracle_image(vol_np, view):
    return oracle.default().render(vol_np, view.width, view.height, **view_kwargs(view))


def gpu_image(V, view):
    img = V.render(view)
    torch.cuda.synchronize()
    return img.cpu().numpy()


def check(got, want, max_abs, rel_l2):
    err = np.abs(got.astype(np.float64) - want)
    rel = np.linalg.norm(err) / max(np.linalg.norm(want), 1e-30)
    assert err.max() <= max_abs and rel <= rel_l2, (err.max(), rel)
    return err.max(), rel


SHAPE = (17, 21, 29)  # nz, ny, nx: none a multiple of the 8-voxel brick
CTR = [14.0, 10.0, 8.0]


def views(w=37, h=23, **kw):
    """Outside and oblique, inside the volume, grazing, looking away, on an axis."""
    lut = lbm.default_lut(0.6)
    base = dict(lut=lut, a_stop=1.0, dt=0.37, tf_scale=1.7, tf_offset=0.05)
    base.update(kw)
    return {
        "oblique": lbm.View(w, h, [50.0, -30.0, 40.0], CTR, up=[0, 0, 1], fov_y=0.5, **base),
        "inside": lbm.View(w, h, [12.0, 9.0, 7.0], [30.0, 20.0, 9.0], up=[0, 0, 1], fov_y=1.2, **base),
        "wide": lbm.View(w, h, [14.0, 10.0, -25.0], CTR, up=[0, 1, 0], fov_y=1.4, **base),
        "away": lbm.View(w, h, [60.0, 10.0, 8.0], [90.0, 10.0, 8.0], up=[0, 0, 1], fov_y=0.4, **base),
        "axis": lbm.View(w, h, [14.0, 10.0, 60.0], CTR, up=[0, 1, 0], fov_y=0.3, **base),
    }


@pytest.mark.parametrize("name", ["oblique", "inside", "wide", "away", "axis"])
def test_exact_filter_matches_oracle(name):
    vol = blobs(SHAPE, 12, seed=1)
    V = upload(vol)
    view = views(filter=lbm.FILTER_EXACT)[name]
    got, want = gpu_image(V, view), oracle_image(vol, view)
    if name == "away":
        assert np.abs(got).max() == 0.0 and np.abs(want).max() == 0.0
        return
    assert (want[..., 3] > 0.01).mean() > 0.05
    print(name, check(got, want, 2e-4, 5e-5))


@pytest.mark.parametrize("w,h", [(1, 1), (16, 8), (33, 9), (128, 72)])
def test_exact_filter_image_sizes(w, h):
    vol = blobs(SHAPE, 10, seed=2)
    V = upload(vol)
    view = views(w, h, filter=lbm.FILTER_EXACT)["oblique"]
    check(gpu_image(V, view), oracle_image(vol, view), 2e-4, 5e-5)


def test_texture_filter_matches_oracle():
    vol = blobs(SHAPE, 12, seed=3)
    V = upload(vol)
    for name in ("oblique", "inside", "wide"):
        view = views(64, 48, filter=lbm.FILTER_TEXTURE)[name]
        print(name, check(gpu_image(V, view), oracle_image(vol, view), 1e-2, 3e-3))


def test_early_termination_bounded():
    vol = blobs(SHAPE, 12, seed=4)
    V = upload(vol)
    lut = lbm.default_lut(8.0)  # nearly opaque: most rays stop early
    view = views(64, 48, filter=lbm.FILTER_EXACT, lut=lut, a_stop=0.95)["oblique"]
    got, want = gpu_image(V, view), oracle_image(vol, view)
    err = np.abs(got.astype(np.float64) - want).max(axis=-1)
    assert (want[..., 3] >= 0.95).mean() > 0.2
    assert err.max() <= (1 - 0.95) + 2e-4
    assert (err > 2e-4).mean() < 0.01


@pytest.mark.parametrize("filt", [lbm.FILTER_TEXTURE, lbm.FILTER_EXACT])
def test_empty_skipping_is_bitwise_invisible(filt):
    vol = blobs((40, 36, 45), 6, seed=5, sparse=True)
    assert (vol == 0).mean() > 0.5
    V = upload(vol)
    for name, view in views(96, 64, filter=filt).items():
        view.skip_empty = True
        a = V.render(view).clone()
        view.skip_empty = False
        b = V.render(view)
        assert torch.equal(a, b), name
    # the counting kernel draws the same image; skipping takes fewer samples
    view = views(96, 64, filter=filt)["oblique"]
    ref = V.render(view).clone()
    n_skip, n_full = torch.zeros(2, dtype=torch.int64, device="cuda"), torch.zeros(2, dtype=torch.int64, device="cuda")
    view.counters = n_skip
    assert torch.equal(V.render(view), ref)
    view.skip_empty, view.counters = False, n_full
    assert torch.equal(V.render(view), ref)
    (ts, js), (tf, jf) = n_skip.tolist(), n_full.tolist()
    assert jf == 0 and js > 0 and 0 < ts < tf, (ts, js, tf, jf)
    # a LUT that gives value 0 some opacity turns skipping off by itself
    lut = lbm.default_lut(0.6)
    lut[:2, 3] = 0.05
    view = views(96, 64, filter=filt, lut=lut)["oblique"]
    a = V.render(view).clone()
    view.skip_empty = False
    assert torch.equal(a, V.render(view))
    if filt == lbm.FILTER_EXACT:
        check(a.cpu().numpy(), oracle_image(vol, view), 2e-4, 5e-5)


def test_render_rejects_bad_views():
    V = upload(blobs((8, 8, 8), 2, seed=6))
    good = views(8, 8)["oblique"]
    for field, bad in [("dt", 0.0), ("dt", 1e-5), ("fov_y", 0.0), ("a_stop", 0.0), ("a_stop", 1.5),
                       ("filter", 7)]:
        v = views(8, 8)["oblique"]
        setattr(v, field, bad)
        with pytest.raises(lbm.LbmError):
            V.render(v)
    # an empty image is refused by the library itself
    import ctypes as C
    st = views(8, 8)["oblique"]._struct()
    st.width = 0
    buf = torch.empty(8, 8, 4, device="cuda")
    lib = lbm.load_library()
    assert lib.lbm_render(V._v, C.byref(st), C.c_void_p(buf.data_ptr()), None) == 1
    v = views(8, 8)["oblique"]
    v.up = v.center - v.eye  # parallel to the view direction
    with pytest.raises(lbm.LbmError):
        V.render(v)
    v = views(8, 8)["oblique"]
    v.lut[3, 1] = np.nan
    with pytest.raises(lbm.LbmError):
        V.render(v)
    V.render(good)


# ------------------------------------------------------------ lattice volumes

def _lattice(g, q=19, tau=0.7, steps=150, storage=lbm.STORE_FP32):
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    L = lbm.Lattice(q, g.xyz, nbr, link, tau, storage=storage, rho_mean=g.rho_mean, amp=g.amp,
                    period=g.period, phase=g.phase)
    L.step(steps)
    return L, nbr, link


def _dense(g, values, origin, shape):
    v = np.zeros(shape, np.float32)
    p = g.xyz - np.asarray(origin)
    ok = np.all((p >= 0) & (p < np.array(shape[::-1])), axis=1)
    v[p[ok, 2], p[ok, 1], p[ok, 0]] = values[ok]
    return v


@pytest.mark.parametrize("storage", [lbm.STORE_FP32, lbm.STORE_FP16])
def test_volume_from_lattice_holds_the_macros(storage):
    g = G.tube(radius=6, length=30, nx=15, ny=15, rho_in=1.002, rho_out=0.999)
    L, _, _ = _lattice(g, storage=storage)
    lo, dims = L.box()
    assert tuple(lo) == tuple(g.xyz.min(0)) and tuple(dims) == tuple(g.xyz.max(0) - g.xyz.min(0) + 1)
    rho, u, wss = [t.cpu().numpy() for t in L.macros()]
    speed = np.linalg.norm(u.astype(np.float64), axis=1)
    V = lbm.Volume.for_lattice(L)
    shape = V.shape
    for qty, ref in ((lbm.QTY_DENSITY, rho), (lbm.QTY_SPEED, speed), (lbm.QTY_WSS, wss)):
        V.from_lattice(L, qty)
        got = V.download().cpu().numpy()
        want = _dense(g, ref.astype(np.float32), lo, shape)
        fluid = _dense(g, np.ones(g.n, np.float32), lo, shape) > 0
        assert np.all(got[~fluid] == 0.0)
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= 1e-6 * scale, qty
    # a cropped window with an offset origin: sites outside it are left out
    org = (lo[0] + 3, lo[1] - 2, lo[2] + 5)
    W = lbm.Volume(9, 11, 13)
    W.from_lattice(L, lbm.QTY_SPEED, origin=org)
    got = W.download().cpu().numpy()
    want = _dense(g, speed.astype(np.float32), org, W.shape)
    assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()


def test_volume_refill_and_upload_cycle():
    g = G.random_mask((14, 12, 10), p=0.55, seed=61, n_iolets=2)
    L, _, _ = _lattice(g, q=15, steps=20)
    V = lbm.Volume.for_lattice(L)
    V.from_lattice(L, lbm.QTY_SPEED)
    L.step(7)
    V.from_lattice(L, lbm.QTY_SPEED)  # same lattice and origin: only the sites are rewritten
    fresh = lbm.Volume.for_lattice(L)
    fresh.from_lattice(L, lbm.QTY_SPEED)
    assert torch.equal(V.download(), fresh.download())
    noise = torch.rand(V.shape, device="cuda") + 0.5
    V.upload(noise)
    assert torch.equal(V.download(), noise)
    V.from_lattice(L, lbm.QTY_SPEED)  # clears the uploaded values again
    assert torch.equal(V.download(), fresh.download())
    view = lbm.View(40, 30, [30.0, -20.0, 25.0], [7.0, 6.0, 5.0], up=[0, 0, 1], fov_y=0.6, dt=0.3,
                    tf_scale=1.0 / max(float(fresh.download().max()), 1e-12))
    a = V.render(view).clone()
    view.skip_empty = False
    assert torch.equal(a, V.render(view))


def test_lattice_render_matches_oracle_simulation():
    """The whole path: GPU steps -> speed volume -> image, against oracle
    steps -> oracle speed -> oracle image."""
    q, tau, steps = 19, 0.7, 200
    g = G.tube(radius=5, length=24, nx=13, ny=13, rho_in=1.003, rho_out=0.998)
    L, nbr, link = _lattice(g, q=q, tau=tau, steps=steps)
    V = lbm.Volume.for_lattice(L)
    V.from_lattice(L, lbm.QTY_SPEED)
    o = oracle.default()
    f = o.run(q, nbr, link, tau, o.rest_state(q, g.n), steps, geom=g)
    _, ou, _ = o.macros(q, link, tau, f)
    speed = np.linalg.norm(ou, axis=1)
    vol = _dense(g, speed.astype(np.float32), V.origin, V.shape)
    ctr = (np.array(V.shape[::-1]) - 1) / 2.0
    view = lbm.View.orbit(ctr, 60.0, 0.7, 0.4, 48, 64, fov_y=0.6, dt=0.4,
                          tf_scale=1.0 / float(speed.max()), a_stop=1.0, filter=lbm.FILTER_EXACT)
    got, want = gpu_image(V, view), oracle_image(vol, view)
    assert (want[..., 3] > 0.01).mean() > 0.1
    print(check(got, want, 1e-3, 1e-4))


def test_vessel_tree_full_size_sampled():
    """The benchmark's render workload: the vessel tree's speed volume
    (770 x 907 x 953 voxels) after the benchmark's spin-up, 1920 x 1080, in
    the benchmark's launch configuration; 400 sampled pixels of each filter
    against the oracle on the same volume (a_stop = 0.99 here, so a pixel may
    differ by one sample past the threshold, <= 0.01)."""
    import bench

    g = bench.make_geometry("vessel_tree")
    L, _, _ = _lattice(g, q=19, tau=0.6, steps=bench.RENDER_SPINUP)
    _, u, _ = L.macros(want=("u",))
    umax = float(torch.linalg.vector_norm(u, dim=1).max())
    V = lbm.Volume.for_lattice(L)
    V.from_lattice(L, lbm.QTY_SPEED)
    vol = V.download().cpu().numpy()
    L.close()
    view = bench.render_view(V, 1.0 / umax)
    rng = np.random.default_rng(7)
    img = V.render(view).cpu().numpy()
    alpha = img[..., 3]
    hit = np.argwhere(alpha > 0.01)
    miss = np.argwhere(alpha <= 0.01)
    assert len(hit) > 1000, len(hit)
    pick = np.concatenate([hit[rng.choice(len(hit), 300, replace=False)],
                           miss[rng.choice(len(miss), 100, replace=False)]])
    pix = pick[:, ::-1].copy()  # (px, py)
    want = oracle.default().render_pixels(vol, view.width, view.height, pix, **view_kwargs(view))
    got = img[pick[:, 0], pick[:, 1]]
    err_tex = np.abs(got - want).max(axis=1)
    view.filter = lbm.FILTER_EXACT
    ex = V.render(view).cpu().numpy()[pick[:, 0], pick[:, 1]]
    err_ex = np.abs(ex - want).max(axis=1)
    print("texture filter: max %.3g p99 %.3g; exact: max %.3g, share > 2e-4: %.4f" % (
        err_tex.max(), np.quantile(err_tex, 0.99), err_ex.max(), (err_ex > 2e-4).mean()))
    assert err_ex.max() <= 0.01 + 2e-4
    assert (err_ex > 2e-4).mean() < 0.02
    assert err_tex.max() <= 3e-2 and np.quantile(err_tex, 0.9) <= 1e-2


def test_degenerate_volumes():
    """A 1 x 1 x 1 volume, a one-voxel-thick slab, and the volume of a lattice
    without sites (all zero) against the oracle."""
    for shape in [(1, 1, 1), (1, 9, 13), (7, 1, 5)]:
        vol = (0.3 + 0.5 * np.random.default_rng(sum(shape)).random(shape)).astype(np.float32)
        V = upload(vol)
        ctr = (np.array(shape[::-1], np.float64) - 1) / 2.0
        for filt in (lbm.FILTER_EXACT, lbm.FILTER_TEXTURE):
            view = lbm.View.orbit(ctr, 12.0, 0.4, 0.3, 24, 17, fov_y=0.9, dt=0.21, a_stop=1.0,
                                  lut=lbm.default_lut(0.8), filter=filt)
            got, want = gpu_image(V, view), oracle_image(vol, view)
            assert (want[..., 3] > 0).any()
            tol = (2e-4, 5e-5) if filt == lbm.FILTER_EXACT else (1e-2, 3e-3)
            check(got, want, *tol)
    g = G.random_mask((3, 3, 3), p=0.0, seed=1, n_iolets=0)
    assert g.n == 0
    nbr, link = lbm.links_build(19, g.xyz, g.io_xyz, g.io_id, g.periodic)
    L = lbm.Lattice(19, g.xyz, nbr, link, 0.7)
    V = lbm.Volume.for_lattice(L)
    V.from_lattice(L, lbm.QTY_SPEED)
    assert V.shape == (1, 1, 1) and float(V.download().abs().max()) == 0.0
    img = V.render(lbm.View(8, 8, [5.0, 5.0, 5.0], [0.0, 0.0, 0.0], up=[0, 0, 1]))
    assert float(img.abs().max()) == 0.0


@pytest.mark.parametrize("w,h", [(48, 20), (1, 1), (33, 9)])
def test_sample_counters_count_every_ray_once(w, h):
    """Nearly parallel rays (fov 1e-3 from 100 voxels away) cross the whole
    box along z: every ray takes ceil(8 / 0.3) = 27 samples."""
    vol = np.full((8, 9, 9), 0.5, np.float32)
    V = upload(vol)
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    view = lbm.View(w, h, [4.0, 4.0, -100.0], [4.0, 4.0, 4.0], up=[0, 1, 0], fov_y=1e-3, dt=0.3,
                    a_stop=1.0, lut=lbm.default_lut(0.01), skip_empty=False, counters=cnt)
    V.render(view)
    assert cnt.tolist() == [27 * w * h, 0]
