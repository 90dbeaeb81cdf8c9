"""The C-ABI library loads, exports every declared entry point, and its
host-only parts (link building, argument and table validation) behave as
specified -- no GPU needed."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1906_11925_gb300 import geometry as G
from paper_1906_11925_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:lbm_status|void|const char \*)\s*(lbm_\w+)\s*\(",
                                 txt, re.M)))


def test_library_exports_every_declared_symbol():
    lib = lbm.load_library()
    syms = declared_symbols()
    assert len(syms) >= 18
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(lbm.EXPORTED) == syms


@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("geom", ["tube", "mask_open", "mask_periodic", "slab", "aneurysm"])
def test_links_bit_exact_vs_oracle(q, geom):
    g = {"tube": lambda: G.tube(),
         "mask_open": lambda: G.random_mask((7, 6, 5), p=0.5, seed=11, n_iolets=4),
         "mask_periodic": lambda: G.random_mask((6, 5, 4), p=0.6, seed=12, periodic=True),
         "slab": lambda: G.slab(16, 3, 5),
         "aneurysm": lambda: G.aneurysm()}[geom]()
    a = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    b = oracle.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])


def test_links_empty():
    nbr, link = lbm.links_build(19, np.zeros((0, 3)))
    assert nbr.shape == (19, 0)


@pytest.mark.parametrize("case", ["dup", "q", "io_id", "coord"])
def test_links_errors(case):
    xyz = np.array([[0, 0, 0], [1, 0, 0]])
    kw = {}
    q = 15
    if case == "dup":
        xyz = np.array([[0, 0, 0], [0, 0, 0]])
    elif case == "q":
        q = 27
    elif case == "io_id":
        kw = dict(io_xyz=np.array([[2, 0, 0]]), io_id=np.array([64]))
    else:
        xyz = np.array([[1 << 19, 0, 0]])
    with pytest.raises(lbm.LbmError) as ei:
        lbm.links_build(q, xyz, **kw)
    assert ei.value.name == "LBM_ERR_ARG"


def _create(q, g, nbr=None, link=None, **kw):
    if nbr is None:
        nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    args = dict(tau=0.8, rho_mean=g.rho_mean, amp=g.amp, period=g.period, phase=g.phase,
                stream=0)
    args.update(kw)
    return lbm.Lattice(q, g.xyz, nbr, link, **args)


@pytest.mark.parametrize("kw", [dict(tau=0.5), dict(tau=float("nan")), dict(storage=3),
                                dict(rho0=0.0), dict(storage=1, fp16_scale_log2=30),
                                dict(storage=2, fp16_scale_log2=31), dict(storage=2, fp16_scale_log2=-1)])
def test_create_rejects_bad_params_before_any_gpu_call(kw):
    g = G.tube(radius=2, length=4, nx=5, ny=5)
    with pytest.raises(lbm.LbmError) as ei:
        _create(15, g, **kw)
    assert ei.value.name == "LBM_ERR_ARG"


@pytest.mark.parametrize("corrupt", ["asym", "range", "flag", "rest", "iolet_id"])
def test_create_rejects_bad_table(corrupt):
    g = G.tube(radius=2, length=4, nx=5, ny=5)
    nbr, link = lbm.links_build(15, g.xyz, g.io_xyz, g.io_id, g.periodic)
    nbr = nbr.copy()
    link = link.copy()
    x = int(np.nonzero(link[1] == 0)[0][0])
    if corrupt == "asym":
        nbr[1, x] = (nbr[1, x] + 1) % g.n
    elif corrupt == "range":
        nbr[1, x] = g.n
    elif corrupt == "flag":
        link[1, x] = 1
    elif corrupt == "rest":
        nbr[0, 0] = 1
    else:
        xs = np.nonzero(link[6] >= 2)[0]
        link[6, xs[0]] = 2 + 7
    with pytest.raises(lbm.LbmError) as ei:
        _create(15, g, nbr=nbr, link=link)
    assert ei.value.name == "LBM_ERR_TABLE"


def _dp_steps(l, f, memo={}):
    """Brute-force minimum number of forward steps to reverse l steps with f
    free snapshot slots (the start state stored), by dynamic programming."""
    if l <= 1:
        return 0
    if f == 0:
        return l * (l - 1) // 2
    key = (l, f)
    if key not in memo:
        memo[key] = min(m + _dp_steps(l - m, f - 1) + _dp_steps(m, f) for m in range(1, l))
    return memo[key]


def test_revolve_schedule_is_optimal():
    """lbm_revolve_steps (the schedule lbm_objective_grad executes) equals the
    brute-force optimum plus the one extra step that forms the final state,
    and Griewank's closed form r l - C(s + r, s + 1) (s = n_snap)."""
    from math import comb
    for l in range(1, 70):
        for s in range(1, 8):
            got = lbm.revolve_steps(l, s)
            want = 0 if l == 0 else _dp_steps(l, s - 1) + 1
            assert got == want, (l, s, got, want)
            if l > 1:
                r = 0
                while comb(s + r, s) < l:
                    r += 1
                assert got == r * l - comb(s + r, s + 1) + 1, (l, s)
    # the stated adjoint workloads: 4000 steps / 64 snapshots, 3000 steps / 40
    assert lbm.revolve_steps(4000, 64) == 9789 + 1
    assert lbm.revolve_steps(3000, 40) == 3 * 3000 - comb(43, 41) + 1
    assert lbm.revolve_steps(5, 6) == 5


@pytest.mark.parametrize("case", ["kind", "no_normal", "not_unit"])
def test_create_rejects_bad_velocity_iolet(case):
    g = G.tube(radius=2, length=4, nx=5, ny=5)
    kind = np.array([lbm.IOLET_VELOCITY, 0], np.int32)
    normal = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 0.0]])
    if case == "kind":
        kind[1] = 7
    if case == "not_unit":
        normal[0] = [0.0, 0.0, 2.0]
    with pytest.raises(lbm.LbmError) as ei:
        _create(15, g, iolet_kind=kind, iolet_normal=None if case == "no_normal" else normal)
    assert ei.value.name == "LBM_ERR_ARG"


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of lbm_params, lbm_objective and lbm_view have the
    sizes and field offsets the C compiler gives the header's structs."""
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "lbm.h"\n'
                   'int main(void) {\n'
                   '  printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(lbm_params),\n'
                   '         offsetof(lbm_params, velocity_weight), sizeof(lbm_objective),\n'
                   '         sizeof(lbm_view), offsetof(lbm_view, fov_y), offsetof(lbm_view, filter),\n'
                   '         offsetof(lbm_view, lut));\n  printf("%zu\\n", offsetof(lbm_view, counters_d));\n'
                   '  printf("%zu\\n", offsetof(lbm_params, site_order));\n'
                   '  return 0;\n}\n')
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    want = [C.sizeof(lbm._Params), lbm._Params.velocity_weight.offset, C.sizeof(lbm._Objective),
            C.sizeof(lbm._View), lbm._View.fov_y.offset, lbm._View.filter.offset, lbm._View.lut.offset,
            lbm._View.counters_d.offset, lbm._Params.site_order.offset]
    assert got == want


def test_binding_constants_match_the_header(tmp_path):
    """Every enum value the binding passes through the ABI (storage forms,
    streaming forms, site orders, iolet kinds, objectives, rendered
    quantities, filters) and every status name it reports equals the
    header's, as the C compiler sees it; and the benchmark's site-order
    choices name the binding's constants."""
    names = ["STORE_FP32", "STORE_FP16", "STORE_I16", "STREAM_PULL", "STREAM_AA", "IOLET_DENSITY",
             "IOLET_VELOCITY", "MAX_IOLETS", "ORDER_MORTON_RUNS", "ORDER_MORTON", "ORDER_ROWS",
             "ORDER_SLABS", "OBJ_WSS", "OBJ_DENSITY", "QTY_DENSITY", "QTY_SPEED", "QTY_WSS",
             "FILTER_TEXTURE", "FILTER_EXACT"]
    status = sorted(lbm._STATUS.items())
    src = tmp_path / "enums.c"
    body = "".join('  printf("%%d\\n", (int)LBM_%s);\n' % n for n in names)
    body += "".join('  printf("%%d\\n", (int)%s);\n' % nm for _, nm in status)
    src.write_text('#include <stdio.h>\n#include "lbm.h"\nint main(void) {\n' + body + "  return 0;\n}\n")
    exe = tmp_path / "enums"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == [getattr(lbm, n) for n in names] + [code for code, _ in status]
    import bench
    orders = {k: getattr(lbm, c) for k, (c, _) in bench.SITE_ORDERS.items()}
    assert orders == {"rows": lbm.ORDER_ROWS, "runs": lbm.ORDER_MORTON_RUNS, "morton": lbm.ORDER_MORTON}


def test_render_calls_reject_bad_arguments_before_any_gpu_call():
    lib = lbm.load_library()
    out = C.c_void_p()
    for dims in [(0, 4, 4), (4, -1, 4), (4, 4, 16385)]:
        assert lib.lbm_volume_create(*dims, C.byref(out)) == 1
        assert out.value is None
    assert "16384" in lib.lbm_last_error(None).decode()
    assert lib.lbm_volume_create(4, 4, 4, None) == 1
    v = lbm.View(8, 8, [10.0, 0, 0], [0, 0, 0])._struct()
    assert lib.lbm_render(None, C.byref(v), None, None) == 1
    assert lib.lbm_volume_upload(None, None, None) == 1
    assert lib.lbm_volume_download(None, None, None) == 1
    assert lib.lbm_lattice_box(None, None, None) == 1
    assert lib.lbm_volume_from_lattice(None, None, 1, None) == 1
    lib.lbm_volume_destroy(None)


def test_default_lut_leaves_zero_clear():
    lut = lbm.default_lut()
    assert lut.shape == (256, 4) and lut[0, 3] == 0.0 and np.all(np.diff(lut[:, 3]) >= 0)
    v = lbm.View.orbit([1.0, 2.0, 3.0], 10.0, 0.3, 0.2, 64, 32).zoom(2.0)
    assert np.isclose(np.linalg.norm(v.eye - v.center), 10.0)
    assert np.isclose(math.tan(v.fov_y / 2), math.tan(0.3) / 2.0)


@pytest.mark.parametrize("q", [15, 19])
def test_lattice_vectors_match_the_link_tables(q):
    """The binding's direction table is the order the link builder uses."""
    g = G.periodic_box(5, 4, 3)
    nbr, _ = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    e = lbm.lattice_vectors(q)
    for i in range(q):
        d = (g.xyz[nbr[i]] - g.xyz) % g.periodic
        assert np.all(d == e[i] % g.periodic), i
    assert np.array_equal(e, np.asarray(oracle.lattice(q)[0]).reshape(q, 3))


@pytest.mark.parametrize("case", ["zero", "above_one", "nan"])
def test_create_rejects_bad_wall_fractions(case):
    g = G.tube(radius=2, length=4, nx=5, ny=5)
    q = 15
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    wq = np.full((q, g.n), 0.3)
    kw = {}
    if case == "zero":
        wq[link == 1] = 0.0
    elif case == "above_one":
        wq[np.nonzero(link == 1)[0][0], np.nonzero(link == 1)[1][0]] = 1.5
    else:
        wq[link == 1] = np.nan
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Lattice(q, g.xyz, nbr, link, 0.7, rho_mean=g.rho_mean, wall_q=wq, stream=0, **kw)
    assert ei.value.name == "LBM_ERR_ARG"


def test_wall_fractions_of_the_tube_are_exact():
    """Against the circle crossing computed independently here: for each wall
    link of the tube, the wall point p + q c lies on the cylinder."""
    g = G.tube(radius=5.3, length=6, nx=13, ny=13)
    q = 19
    nbr, link = lbm.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    e = lbm.lattice_vectors(q)
    wq = G.wall_fractions(g, e, link)
    ii, xx = np.nonzero(link == 1)
    pts = g.xyz[xx] + wq[ii, xx][:, None] * e[ii]
    r = np.hypot(pts[:, 0] - 6.0, pts[:, 1] - 6.0)
    assert np.abs(r - 5.3).max() < 1e-5
    assert np.all((wq[ii, xx] > 0) & (wq[ii, xx] <= 1)) and np.all(wq[link != 1] == 0.5)
    assert np.all(np.round(wq * 2 ** 24) == wq * 2 ** 24)


@pytest.mark.parametrize("q,n", [(19, 113_025_409), (19, 120_000_000), (15, 143_165_569),
                                 (15, (1 << 31) - 1024)])
def test_size_limit_is_checked_before_any_table_read(q, n):
    """The kernels address population slots with 32-bit offsets: lbm_create
    refuses q * npad >= 2^31 (npad = n rounded up to 128; largest D3Q19
    lattice 113,025,408 sites) before it reads the site arrays, so that
    one-element stand-ins for them are never touched."""
    import ctypes as C

    npad = max(128, -(-n // 128) * 128)
    assert q * npad >= 2 ** 31  # (a size below the limit would read the stand-ins)
    lib = lbm.load_library()
    p = lbm._Params(q=q, storage=0, tau=0.8, rho0=1.0, fp16_scale_log2=14, n_iolets=0)
    tiny_i32 = np.zeros(4, np.int32)
    tiny_u8 = np.zeros(4, np.uint8)
    ctx = C.c_void_p()
    st = lib.lbm_create(C.byref(ctx), C.byref(p), n, tiny_i32.ctypes.data_as(C.c_void_p),
                        tiny_i32.ctypes.data_as(C.c_void_p), tiny_u8.ctypes.data_as(C.c_void_p), None)
    msg = lib.lbm_last_error(None).decode()
    assert st == 1 and not ctx.value  # LBM_ERR_ARG
    assert "too many sites" in msg, msg
