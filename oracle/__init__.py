"""FP64 CPU oracle for the sparse LBGK collide-and-stream path (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package.  It wraps ``oracle.c`` (plain C, float64, optional OpenMP over sites)
through ctypes and shares no code with the CUDA library.  Each function
follows the stated reading of the paper's method (Section 2: collision and
propagation over sparse fluid sites; Section 4: simple bounce-back walls;
Section 3.3.2: ray-marched volume rendering);
see ``oracle.c`` for the definitions.

All arrays use caller site order; populations are float64 [q, n].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None  # the default Oracle instance
_lock = threading.Lock()


def _compile(src: str, out: str) -> None:
    base = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", src, "-o", out + ".tmp", "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(out + ".tmp", out)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP when available); returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    _compile(_SRC, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    lib = C.CDLL(path)
    P = C.c_void_p
    i64, i32, f64 = C.c_int64, C.c_int, C.c_double
    lib.orc_lattice.argtypes = [i32, P, P, P]
    lib.orc_equilibrium.argtypes = [i32, f64, P, P]
    lib.orc_links_build.argtypes = [i32, i64, P, i64, P, P, P, P, P]
    lib.orc_step.argtypes = [i32, i64, P, P, f64, i32, P, P, P, P, i64, P, P]
    lib.orc_run.argtypes = [i32, i64, P, P, f64, i32, P, P, P, P, i64, i64, P, P]
    lib.orc_run_bc.argtypes = [i32, i64, P, P, f64, i32, P, P, P, P, P, P, P, P, i64, i64, P, P]
    lib.orc_macros.argtypes = [i32, i64, P, f64, P, P, P, P]
    lib.orc_mass.argtypes = [i32, i64, P]
    lib.orc_mass.restype = f64
    lib.orc_adjoint_step.argtypes = [i32, i64, P, P, f64, i32, P, P, P, P, i64, P, P, P, P, P, P, P]
    lib.orc_objective.argtypes = [i32, i64, P, f64, i32, P, P, f64, P, P]
    lib.orc_objective.restype = f64
    lib.orc_gradient.argtypes = [i32, i64, P, P, f64, i32, P, P, P, P, i64, i64, P, i32, P,
                                 i64, i64, f64, P, P, P, P, P, P]
    lib.orc_objective_run.argtypes = [i32, i64, P, P, f64, i32, P, P, P, P, i64, i64, P, i32, P,
                                      i64, i64, f64]
    lib.orc_objective_run.restype = f64
    lib.orc_adjoint_step_bc.argtypes = [i32, i64, P, P, f64, i32, P, P, P, P, P, P, P, P, i64, P, P, P, P,
                                        P, P, P]
    lib.orc_gradient_bc.argtypes = [i32, i64, P, P, f64, i32, P, P, P, P, P, P, P, P, i64, i64, P, i32, P,
                                    i64, i64, f64, P, P, P, P, P, P]
    lib.orc_objective_run_bc.argtypes = [i32, i64, P, P, f64, i32, P, P, P, P, P, P, P, P, i64, i64, P, i32,
                                         P, i64, i64, f64]
    lib.orc_objective_run_bc.restype = f64
    lib.orc_render.argtypes = [P, i32, i32, i32, i32, i32, P, P, P, f64, f64, f64, f64, f64, P, P]
    lib.orc_render_pixels.argtypes = [P, i32, i32, i32, i32, i32, P, P, P, f64, f64, f64, f64,
                                      f64, P, i64, P, P]
    lib.orc_num_threads.restype = i32
    lib.orc_set_threads.argtypes = [i32]
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class _Iolets:
    def __init__(self, geom=None, rho_mean=None, amp=None, period=None, phase=None):
        if geom is not None:
            rho_mean, amp, period, phase = geom.rho_mean, geom.amp, geom.period, geom.phase
        k = 0 if rho_mean is None else len(rho_mean)
        z = np.zeros(max(k, 1))
        self.k = k
        self.mean = _c(rho_mean if k else z, np.float64)
        self.amp = _c(amp if (k and amp is not None) else z, np.float64)
        self.period = _c(period if (k and period is not None) else z, np.float64)
        self.phase = _c(phase if (k and phase is not None) else z, np.float64)


def _bc(q, n, io_kind=None, io_normal=None, weight=None, wall_q=None):
    """The boundary arrays of orc_step_bc (None where absent)."""
    kind = None if io_kind is None else _c(io_kind, np.int32)
    nrm = None if io_normal is None else _c(io_normal, np.float64).reshape(-1, 3)
    w = None if weight is None else _c(weight, np.float64)
    wq = None if wall_q is None else _c(wall_q, np.float64).reshape(q, n)
    return kind, nrm, w, wq


class Oracle:
    """The oracle functions bound to one compiled copy of the C source."""

    def __init__(self, path: str):
        self.path = path
        self.lib = _bind(path)

    def num_threads(self) -> int:
        return int(self.lib.orc_num_threads())

    def set_threads(self, nt: int) -> None:
        self.lib.orc_set_threads(int(nt))

    def lattice(self, q: int):
        """(c [q,3] int32, w [q] float64, opp [q] int32) of D3Q15 or D3Q19."""
        e = np.zeros((q, 3), np.int32)
        w = np.zeros(q, np.float64)
        opp = np.zeros(q, np.int32)
        if self.lib.orc_lattice(q, _p(e), _p(w), _p(opp)) != 0:
            raise ValueError("q must be 15 or 19")
        return e, w, opp

    def equilibrium(self, q: int, rho: float, u) -> np.ndarray:
        u = _c(u, np.float64)
        out = np.zeros(q, np.float64)
        if self.lib.orc_equilibrium(q, float(rho), _p(u), _p(out)) != 0:
            raise ValueError("q must be 15 or 19")
        return out

    def links_build(self, q: int, xyz, io_xyz=None, io_id=None, periodic=(0, 0, 0)):
        """Neighbour table nbr int32 [q, n] and link flags uint8 [q, n]."""
        xyz = _c(xyz, np.int32).reshape(-1, 3)
        n = xyz.shape[0]
        io_xyz = _c(np.zeros((0, 3)) if io_xyz is None else io_xyz, np.int32).reshape(-1, 3)
        io_id = _c(np.zeros(0) if io_id is None else io_id, np.int32)
        per = _c(periodic, np.int32)
        nbr = np.zeros((q, n), np.int32)
        link = np.zeros((q, n), np.uint8)
        r = self.lib.orc_links_build(q, n, _p(xyz), io_xyz.shape[0], _p(io_xyz), _p(io_id),
                                     _p(per), _p(nbr), _p(link))
        if r != 0:
            raise ValueError("orc_links_build failed with %d" % r)
        return nbr, link

    def step(self, q, nbr, link, tau, f, t=0, geom=None, **io):
        """One push-form step t -> t+1; returns the new [q, n] populations."""
        nbr = _c(nbr, np.int32)
        link = _c(link, np.uint8)
        f = _c(f, np.float64)
        n = f.shape[1]
        I = _Iolets(geom, **io)
        out = np.empty_like(f)
        r = self.lib.orc_step(q, n, _p(nbr), _p(link), float(tau), I.k, _p(I.mean), _p(I.amp),
                              _p(I.period), _p(I.phase), int(t), _p(f), _p(out))
        if r != 0:
            raise ValueError("orc_step failed")
        return out

    def run(self, q, nbr, link, tau, f, nsteps, t0=0, geom=None, **io):
        """nsteps steps from time t0; returns the state at t0 + nsteps."""
        nbr = _c(nbr, np.int32)
        link = _c(link, np.uint8)
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        n = f.shape[1]
        I = _Iolets(geom, **io)
        work = np.empty_like(f)
        r = self.lib.orc_run(q, n, _p(nbr), _p(link), float(tau), I.k, _p(I.mean), _p(I.amp),
                             _p(I.period), _p(I.phase), int(t0), int(nsteps), _p(f), _p(work))
        if r != 0:
            raise ValueError("orc_run failed")
        return f

    def run_inplace(self, q, nbr, link, tau, f, work, nsteps, t0=0, geom=None, **io):
        """nsteps steps from time t0 on the caller's arrays: f (float64
        [q, n], C order) holds the state on entry and on exit, work is
        scratch of the same shape.  No copy is made, so a caller that steps
        one state repeatedly pays only for the steps themselves."""
        for a in (f, work):
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.shape != f.shape:
                raise ValueError("f and work must be C-contiguous float64 arrays of one shape")
        nbr = _c(nbr, np.int32)
        link = _c(link, np.uint8)
        I = _Iolets(geom, **io)
        r = self.lib.orc_run(q, f.shape[1], _p(nbr), _p(link), float(tau), I.k, _p(I.mean),
                             _p(I.amp), _p(I.period), _p(I.phase), int(t0), int(nsteps), _p(f),
                             _p(work))
        if r != 0:
            raise ValueError("orc_run failed")

    def run_bc(self, q, nbr, link, tau, f, nsteps, io_kind=None, io_normal=None, weight=None,
               t0=0, geom=None, wall_q=None, **io):
        """As run(), with velocity (Ladd) iolets: io_kind[k] = 1 marks iolet k as
        a velocity iolet with unit inward normal io_normal[k] and speed given by
        its schedule; weight [n] scales the speed per site (None = 1); and
        interpolated (BFL) walls: wall_q [q, n] is the fluid fraction of each
        wall link (None = every wall half-way)."""
        nbr = _c(nbr, np.int32)
        link = _c(link, np.uint8)
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        n = f.shape[1]
        I = _Iolets(geom, **io)
        kind = None if io_kind is None else _c(io_kind, np.int32)
        nrm = None if io_normal is None else _c(io_normal, np.float64).reshape(-1, 3)
        w = None if weight is None else _c(weight, np.float64)
        wq = None if wall_q is None else _c(wall_q, np.float64).reshape(q, n)
        work = np.empty_like(f)
        r = self.lib.orc_run_bc(q, n, _p(nbr), _p(link), float(tau), I.k, _p(I.mean), _p(I.amp),
                                _p(I.period), _p(I.phase), _p(kind), _p(nrm), _p(w), _p(wq),
                                int(t0), int(nsteps), _p(f), _p(work))
        if r != 0:
            raise ValueError("orc_run_bc failed")
        return f

    def macros(self, q, link, tau, f):
        """(rho [n], u [n,3], wss [n]) of the pre-collision state f."""
        link = _c(link, np.uint8)
        f = _c(f, np.float64)
        n = f.shape[1]
        rho = np.empty(n)
        u = np.empty((n, 3))
        wss = np.empty(n)
        if self.lib.orc_macros(q, n, _p(link), float(tau), _p(f), _p(rho), _p(u), _p(wss)) != 0:
            raise ValueError("orc_macros failed")
        return rho, u, wss

    def mass(self, f) -> float:
        f = _c(f, np.float64)
        return float(self.lib.orc_mass(f.shape[0], f.shape[1], _p(f)))

    OBJ_WSS = 0
    OBJ_DENSITY = 1

    def adjoint_step(self, q, nbr, link, tau, f, lam_next, t=0, geom=None, io_kind=None, io_normal=None,
                     weight=None, wall_q=None, **io):
        """lam(t) = (dF_t/df)^T lam(t+1) at the state f = f(t) (the boundary
        arguments as in run_bc); returns (lam, dJ/dtau, dJ/dmean[K],
        dJ/damp[K], dJ/dphase[K]) of this step."""
        nbr = _c(nbr, np.int32)
        link = _c(link, np.uint8)
        f = _c(f, np.float64)
        ln = _c(lam_next, np.float64)
        n = f.shape[1]
        I = _Iolets(geom, **io)
        kind, nrm, w, wq = _bc(q, n, io_kind, io_normal, weight, wall_q)
        lam = np.empty_like(f)
        dtau = np.zeros(1)
        K = max(I.k, 1)
        dm, da, dp = np.zeros(K), np.zeros(K), np.zeros(K)
        r = self.lib.orc_adjoint_step_bc(q, n, _p(nbr), _p(link), float(tau), I.k, _p(I.mean),
                                         _p(I.amp), _p(I.period), _p(I.phase), _p(kind), _p(nrm), _p(w),
                                         _p(wq), int(t), _p(f), _p(ln), _p(lam), _p(dtau), _p(dm), _p(da),
                                         _p(dp))
        if r != 0:
            raise ValueError("orc_adjoint_step failed")
        return lam, float(dtau[0]), dm[:I.k], da[:I.k], dp[:I.k]

    def objective(self, q, link, tau, kind, m, f, scale=1.0, grad=False):
        """sum_x m_x q(x) of state f (kind 0 = wall shear stress, 1 = density);
        with grad=True also (scale * d/df, scale * explicit d/dtau)."""
        link = _c(link, np.uint8)
        f = _c(f, np.float64)
        m = _c(m, np.float64)
        n = f.shape[1]
        lam = np.zeros_like(f) if grad else None
        dtau = np.zeros(1)
        J = self.lib.orc_objective(q, n, _p(link), float(tau), int(kind), _p(m), _p(f),
                                   float(scale), _p(lam), _p(dtau))
        return (J, lam, float(dtau[0])) if grad else J

    def gradient(self, q, nbr, link, tau, f0, nsteps, kind, m, t_begin, t_end, scale=1.0,
                 t0=0, geom=None, want_lam0=False, io_kind=None, io_normal=None, weight=None,
                 wall_q=None, **io):
        """Objective J = scale * sum_{t_begin <= t < t_end} sum_x m_x q(x, t) over
        the states of an nsteps run from f0 at time t0, and its gradient by the
        discrete adjoint (every state stored).  Returns a dict with J, dtau,
        dmean, damp, dphase (per iolet) and optionally lam0 = dJ/df0."""
        nbr = _c(nbr, np.int32)
        link = _c(link, np.uint8)
        f0 = _c(f0, np.float64)
        m = _c(m, np.float64)
        n = f0.shape[1]
        I = _Iolets(geom, **io)
        bk, bn, bw, bq = _bc(q, n, io_kind, io_normal, weight, wall_q)
        K = max(I.k, 1)
        J, dtau = np.zeros(1), np.zeros(1)
        dm, da, dp = np.zeros(K), np.zeros(K), np.zeros(K)
        lam0 = np.zeros_like(f0) if want_lam0 else None
        r = self.lib.orc_gradient_bc(q, n, _p(nbr), _p(link), float(tau), I.k, _p(I.mean), _p(I.amp),
                                     _p(I.period), _p(I.phase), _p(bk), _p(bn), _p(bw), _p(bq), int(t0),
                                     int(nsteps), _p(f0), int(kind), _p(m), int(t_begin), int(t_end),
                                     float(scale), _p(J), _p(dtau), _p(dm), _p(da), _p(dp), _p(lam0))
        if r != 0:
            raise ValueError("orc_gradient failed")
        out = dict(J=float(J[0]), dtau=float(dtau[0]), dmean=dm[:I.k], damp=da[:I.k],
                   dphase=dp[:I.k])
        if want_lam0:
            out["lam0"] = lam0
        return out

    def objective_run(self, q, nbr, link, tau, f0, nsteps, kind, m, t_begin, t_end, scale=1.0,
                      t0=0, geom=None, io_kind=None, io_normal=None, weight=None, wall_q=None, **io):
        """J alone, by running forward in C (used for finite differences)."""
        nbr = _c(nbr, np.int32)
        link = _c(link, np.uint8)
        f0 = _c(f0, np.float64)
        m = _c(m, np.float64)
        I = _Iolets(geom, **io)
        bk, bn, bw, bq = _bc(q, f0.shape[1], io_kind, io_normal, weight, wall_q)
        return float(self.lib.orc_objective_run_bc(q, f0.shape[1], _p(nbr), _p(link), float(tau), I.k,
                                                   _p(I.mean), _p(I.amp), _p(I.period), _p(I.phase),
                                                   _p(bk), _p(bn), _p(bw), _p(bq), int(t0), int(nsteps),
                                                   _p(f0), int(kind), _p(m), int(t_begin), int(t_end),
                                                   float(scale)))

    def render(self, vol, width, height, eye, center, up, fov_y, dt, tf_scale, tf_offset, lut,
               a_stop=0.99):
        """Ray-marched RGBA image float32 [height, width, 4] of vol [nz, ny, nx]
        (Section 3.3.2; definitions in orc_render)."""
        vol = _c(vol, np.float32)
        nz, ny, nx = vol.shape
        lut = _c(lut, np.float32).reshape(256, 4)
        out = np.zeros((height, width, 4), np.float32)
        v3 = lambda a: _c(a, np.float64)
        e, c, u = v3(eye), v3(center), v3(up)
        r = self.lib.orc_render(_p(vol), nx, ny, nz, int(width), int(height), _p(e), _p(c), _p(u),
                                float(fov_y), float(dt), float(tf_scale), float(tf_offset),
                                float(a_stop), _p(lut),
                                _p(out))
        if r != 0:
            raise ValueError("orc_render failed")
        return out

    def render_pixels(self, vol, width, height, pixels, eye, center, up, fov_y, dt, tf_scale,
                      tf_offset, lut, a_stop=0.99):
        """The pixels [(px, py), ...] of the same image, float32 [len(pixels), 4]."""
        vol = _c(vol, np.float32)
        nz, ny, nx = vol.shape
        lut = _c(lut, np.float32).reshape(256, 4)
        pix = _c(pixels, np.int32).reshape(-1, 2)
        out = np.zeros((pix.shape[0], 4), np.float32)
        v3 = lambda a: _c(a, np.float64)
        e, c, u = v3(eye), v3(center), v3(up)
        r = self.lib.orc_render_pixels(_p(vol), nx, ny, nz, int(width), int(height), _p(e), _p(c),
                                       _p(u), float(fov_y), float(dt), float(tf_scale),
                                       float(tf_offset), float(a_stop), _p(lut), pix.shape[0],
                                       _p(pix), _p(out))
        if r != 0:
            raise ValueError("orc_render_pixels failed")
        return out

    def rest_state(self, q: int, n: int, rho0: float = 1.0) -> np.ndarray:
        """f_i = w_i rho0 at every site (fluid at rest)."""
        _, w, _ = self.lattice(q)
        return np.repeat((w * rho0)[:, None], n, axis=1)


def default() -> Oracle:
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
        return _lib


def variant(src_text: str, workdir: str) -> Oracle:
    """Compile a modified copy of the oracle source (used by the tests that
    plant a mistake in the oracle and check that a pin catches it)."""
    os.makedirs(workdir, exist_ok=True)
    src = os.path.join(workdir, "oracle_variant.c")
    with open(src, "w") as fh:
        fh.write(src_text)
    out = os.path.join(workdir, "liboracle_variant.so")
    _compile(src, out)
    return Oracle(out)


def source() -> str:
    with open(_SRC) as fh:
        return fh.read()


def num_threads() -> int:
    return default().num_threads()


def set_threads(nt: int) -> None:
    default().set_threads(nt)


def lattice(q):
    return default().lattice(q)


def equilibrium(q, rho, u):
    return default().equilibrium(q, rho, u)


def links_build(q, xyz, io_xyz=None, io_id=None, periodic=(0, 0, 0)):
    return default().links_build(q, xyz, io_xyz, io_id, periodic)


def step(q, nbr, link, tau, f, t=0, geom=None, **io):
    return default().step(q, nbr, link, tau, f, t, geom, **io)


def run(q, nbr, link, tau, f, nsteps, t0=0, geom=None, **io):
    return default().run(q, nbr, link, tau, f, nsteps, t0, geom, **io)


def macros(q, link, tau, f):
    return default().macros(q, link, tau, f)


def mass(f):
    return default().mass(f)


def rest_state(q: int, n: int, rho0: float = 1.0) -> np.ndarray:
    """f_i = w_i rho0 at every site (fluid at rest)."""
    return default().rest_state(q, n, rho0)
