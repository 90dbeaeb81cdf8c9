"""Python binding of libhemelb_gb300 (ctypes, argument marshalling only).

Every call goes through the C ABI of ``include/lbm.h``; the names follow it
(``lbm_links_build`` -> ``links_build``, ``lbm_create`` -> ``Lattice`` ...).
PyTorch supplies device memory for outputs and the CUDA stream.  There is no
CPU fallback: if the shared library is missing the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

STORE_FP32 = 0
STORE_FP16 = 1
STORE_I16 = 2
STREAM_PULL = 0
STREAM_AA = 1
IOLET_DENSITY = 0
IOLET_VELOCITY = 1
MAX_IOLETS = 64
ORDER_MORTON_RUNS = 0
ORDER_MORTON = 1
ORDER_ROWS = 2
ORDER_SLABS = 3

_STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_TABLE", 3: "LBM_ERR_NOMEM",
           4: "LBM_ERR_CUDA", 5: "LBM_ERR_UNSTABLE", 6: "LBM_ERR_STATE"}

EXPORTED = (
    "lbm_links_build", "lbm_create", "lbm_destroy", "lbm_last_error", "lbm_set_stream", "lbm_slab_chunks",
    "lbm_step", "lbm_step_driven", "lbm_get_time", "lbm_set_time", "lbm_macros", "lbm_mass",
    "lbm_weighted_sum", "lbm_check_wait_timeout", "lbm_set_stability_check", "lbm_check_guards",
    "lbm_get_populations", "lbm_get_populations_noalloc", "lbm_set_populations",
    "lbm_state_bytes", "lbm_get_state",
    "lbm_set_state", "lbm_get_links", "lbm_info",
    "lbm_objective_grad", "lbm_revolve_steps", "lbm_adjoint_counts", "lbm_release_workspace",
    "lbm_set_tau", "lbm_set_iolets",
    "lbm_volume_create", "lbm_volume_destroy", "lbm_volume_upload", "lbm_volume_download",
    "lbm_lattice_box", "lbm_volume_from_lattice", "lbm_render",
)

QTY_DENSITY = 0
QTY_SPEED = 1
QTY_WSS = 2
FILTER_TEXTURE = 0
FILTER_EXACT = 1

OBJ_WSS = 0
OBJ_DENSITY = 1

# Lattice vectors in the direction order of the C ABI (include/lbm.h): the
# rest vector, then opposite pairs.
_VEC15 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
          (1, 1, 1), (-1, -1, -1), (1, 1, -1), (-1, -1, 1), (1, -1, 1), (-1, 1, -1),
          (-1, 1, 1), (1, -1, -1)]
_VEC19 = _VEC15[:7] + [(1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
                       (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


def lattice_vectors(q: int) -> np.ndarray:
    """int32 [q, 3] lattice vectors c_i in the library's direction order."""
    return np.array({15: _VEC15, 19: _VEC19}[int(q)], dtype=np.int32)


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), msg))
        self.status = status
        self.name = _STATUS.get(status, str(status))


class _Objective(C.Structure):
    _fields_ = [("kind", C.c_int32), ("weight", C.c_void_p), ("t_begin", C.c_int64),
                ("t_end", C.c_int64), ("scale", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("q", C.c_int32), ("storage", C.c_int32), ("tau", C.c_double),
                ("rho0", C.c_double), ("fp16_scale_log2", C.c_int32), ("n_iolets", C.c_int32),
                ("rho_mean", C.c_void_p), ("amp", C.c_void_p), ("period", C.c_void_p),
                ("phase", C.c_void_p), ("streaming", C.c_int32), ("iolet_kind", C.c_void_p),
                ("iolet_normal", C.c_void_p), ("velocity_weight", C.c_void_p),
                ("wall_q", C.c_void_p), ("site_order", C.c_int32)]


class _View(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("eye", C.c_double * 3),
                ("center", C.c_double * 3), ("up", C.c_double * 3), ("fov_y", C.c_double),
                ("dt", C.c_double), ("tf_scale", C.c_double), ("tf_offset", C.c_double),
                ("a_stop", C.c_double), ("filter", C.c_int32), ("skip_empty", C.c_int32),
                ("counters_d", C.c_void_p), ("lut", (C.c_float * 4) * 256)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load (building if needed) libhemelb_gb300.so; raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    # HEMELB_GB300_CHECKED=1: the build with range-checked table loads
    path = _build.CHECKED_LIB if os.environ.get("HEMELB_GB300_CHECKED") == "1" else _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise OSError("libhemelb_gb300.so is not built: %s" % path)
        _build.build()
    lib = C.CDLL(path)
    P, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    sig = {
        "lbm_links_build": [i32, i64, P, i64, P, P, P, P, P],
        "lbm_create": [P, P, i64, P, P, P, P],
        "lbm_destroy": [P],
        "lbm_last_error": [P],
        "lbm_set_stream": [P, P],
        "lbm_step": [P, i64],
        "lbm_step_driven": [P, i64, P, P],
        "lbm_get_time": [P, P],
        "lbm_set_time": [P, i64],
        "lbm_macros": [P, P, P, P],
        "lbm_mass": [P, P],
        "lbm_weighted_sum": [P, i32, P, P],
        "lbm_check_wait_timeout": [C.c_uint32, P, P],
        "lbm_set_stability_check": [P, i64, C.c_double],
        "lbm_check_guards": [P, P],
        "lbm_get_populations": [P, P],
        "lbm_get_populations_noalloc": [P, P],
        "lbm_set_populations": [P, P],
        "lbm_state_bytes": [P, P],
        "lbm_get_state": [P, P, C.c_size_t],
        "lbm_set_state": [P, P, C.c_size_t],
        "lbm_get_links": [P, P, P],
        "lbm_info": [P, P, P, P],
        "lbm_slab_chunks": [P, P],
        "lbm_objective_grad": [P, P, i64, i32, P, P, P, P, P, P],
        "lbm_revolve_steps": [i64, i32, P],
        "lbm_adjoint_counts": [P, P, P, P],
        "lbm_release_workspace": [P],
        "lbm_set_tau": [P, C.c_double],
        "lbm_set_iolets": [P, i32, P, P, P, P],
        "lbm_volume_create": [i32, i32, i32, P],
        "lbm_volume_destroy": [P],
        "lbm_volume_upload": [P, P, P],
        "lbm_volume_download": [P, P, P],
        "lbm_lattice_box": [P, P, P],
        "lbm_volume_from_lattice": [P, P, i32, P],
        "lbm_render": [P, P, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.lbm_destroy.restype = None
    lib.lbm_volume_destroy.restype = None
    lib.lbm_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(st: int, ctx=None):
    if st != 0:
        lib = load_library()
        msg = lib.lbm_last_error(ctx).decode(errors="replace")
        raise LbmError(st, msg)


def links_build(q: int, xyz, io_xyz=None, io_id=None, periodic=(0, 0, 0)):
    """Canonical neighbour table (int32 [q, n]) and link flags (uint8 [q, n])."""
    lib = load_library()
    xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
    n = xyz.shape[0]
    io_xyz = np.ascontiguousarray(np.zeros((0, 3)) if io_xyz is None else io_xyz,
                                  dtype=np.int32).reshape(-1, 3)
    io_id = np.ascontiguousarray(np.zeros(0) if io_id is None else io_id, dtype=np.int32)
    per = np.ascontiguousarray(periodic, dtype=np.int32)
    nbr = np.empty((q, n), np.int32)
    link = np.empty((q, n), np.uint8)
    _check(lib.lbm_links_build(int(q), n, _p(xyz), io_xyz.shape[0], _p(io_xyz), _p(io_id),
                               _p(per), _p(nbr), _p(link)))
    return nbr, link


def check_wait_timeout(limit: int = 4096, stream=None) -> bool:
    """Run the step kernels' bounded mbarrier wait on a barrier that nothing
    completes (``lbm_check_wait_timeout``); True when it gave up."""
    out = C.c_int32()
    _check(load_library().lbm_check_wait_timeout(int(limit), _stream_handle(stream), C.byref(out)))
    return bool(out.value)


def revolve_steps(nsteps: int, n_snap: int) -> int:
    """Forward steps of a checkpointed gradient (``lbm_revolve_steps``)."""
    out = C.c_int64()
    _check(load_library().lbm_revolve_steps(int(nsteps), int(n_snap), C.byref(out)))
    return out.value


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class Lattice:
    """One simulation (``lbm_create`` ... ``lbm_destroy``) on the current GPU."""

    def __init__(self, q: int, xyz, nbr, link, tau: float, storage: int = STORE_FP32,
                 rho0: float = 1.0, fp16_scale_log2: Optional[int] = None,
                 rho_mean: Sequence[float] = (), amp: Sequence[float] = None,
                 period: Sequence[float] = None, phase: Sequence[float] = None,
                 stream=None, streaming: int = STREAM_PULL, iolet_kind=None, iolet_normal=None,
                 velocity_weight=None, wall_q=None, site_order: int = ORDER_MORTON_RUNS):
        self._lib = load_library()
        self._ctx = C.c_void_p()
        k = len(rho_mean)
        z = [0.0] * k
        self._io = [np.ascontiguousarray(v, dtype=np.float64) for v in
                    (rho_mean, z if amp is None else amp, z if period is None else period,
                     z if phase is None else phase)]
        xyz = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
        nbr = np.ascontiguousarray(nbr, dtype=np.int32)
        link = np.ascontiguousarray(link, dtype=np.uint8)
        n = xyz.shape[0]
        if nbr.shape != (q, n) or link.shape != (q, n):
            raise ValueError("nbr and link must be [q, n]")
        self._kind = None if iolet_kind is None else np.ascontiguousarray(iolet_kind, dtype=np.int32)
        self._nrm = None if iolet_normal is None else np.ascontiguousarray(iolet_normal, dtype=np.float64)
        self._vw = None if velocity_weight is None else np.ascontiguousarray(velocity_weight, dtype=np.float64)
        self._wq = None if wall_q is None else np.ascontiguousarray(wall_q, dtype=np.float64)
        if self._wq is not None and self._wq.shape != (q, n):
            raise ValueError("wall_q must be [q, n]")
        if fp16_scale_log2 is None:
            # the scale S of the 16-bit forms: fp16 only needs the small
            # deviations kept out of its subnormal range; int16 resolves 2^-S
            # uniformly up to 32766 2^-S (22: deviations up to 7.8e-3)
            fp16_scale_log2 = 22 if int(storage) == STORE_I16 else 14
        prm = _Params(int(q), int(storage), float(tau), float(rho0), int(fp16_scale_log2), k,
                      *[(a.ctypes.data if k else None) for a in self._io], int(streaming),
                      None if self._kind is None else self._kind.ctypes.data,
                      None if self._nrm is None else self._nrm.ctypes.data,
                      None if self._vw is None else self._vw.ctypes.data,
                      None if self._wq is None else self._wq.ctypes.data, int(site_order))
        self.streaming = int(streaming)
        self.q, self.n, self.tau, self.storage, self.rho0 = int(q), n, float(tau), int(storage), float(rho0)
        self.n_iolets = k
        st = self._lib.lbm_create(C.byref(self._ctx), C.byref(prm), n, _p(xyz), _p(nbr), _p(link),
                                  _stream_handle(stream))
        _check(st, None)

    @classmethod
    def from_geometry(cls, geom, q: int, tau: float, storage: int = STORE_FP32, **kw):
        nbr, link = links_build(q, geom.xyz, geom.io_xyz, geom.io_id, geom.periodic)
        return cls(q, geom.xyz, nbr, link, tau, storage=storage, rho_mean=geom.rho_mean,
                   amp=geom.amp, period=geom.period, phase=geom.phase, **kw)

    # -- lifetime
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self._lib.lbm_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, st):
        _check(st, self._ctx)

    # -- calls
    def set_stream(self, stream):
        self._ck(self._lib.lbm_set_stream(self._ctx, _stream_handle(stream)))

    def step(self, nsteps: int = 1):
        self._ck(self._lib.lbm_step(self._ctx, int(nsteps)))

    def step_driven(self, rho_io, mass: bool = True):
        """Steps with caller-supplied iolet densities rho_io [nsteps, K] (host
        array, float64; may be a pinned torch tensor).  Returns the mass after
        each step (float64 [nsteps]) or None."""
        if hasattr(rho_io, "data_ptr"):
            nsteps = int(rho_io.shape[0])
            ptr = C.c_void_p(rho_io.data_ptr())
            keep = rho_io
        else:
            keep = np.ascontiguousarray(rho_io, dtype=np.float64).reshape(-1, max(self.n_iolets, 1))
            nsteps = keep.shape[0]
            ptr = _p(keep)
        out = np.empty(nsteps, np.float64) if mass else None
        self._ck(self._lib.lbm_step_driven(self._ctx, nsteps, ptr, _p(out)))
        del keep
        return out

    @property
    def time(self) -> int:
        t = C.c_int64()
        self._ck(self._lib.lbm_get_time(self._ctx, C.byref(t)))
        return t.value

    def set_time(self, t: int):
        self._ck(self._lib.lbm_set_time(self._ctx, int(t)))

    def macros(self, rho=None, u=None, wss=None, want=("rho", "u", "wss")):
        """rho [n], u [n, 3], wss [n] as float32 CUDA tensors (caller order)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if rho is None and "rho" in want:
            rho = torch.empty(self.n, dtype=torch.float32, device=dev)
        if u is None and "u" in want:
            u = torch.empty(self.n, 3, dtype=torch.float32, device=dev)
        if wss is None and "wss" in want:
            wss = torch.empty(self.n, dtype=torch.float32, device=dev)
        for t, shape in ((rho, (self.n,)), (u, (self.n, 3)), (wss, (self.n,))):
            if t is not None:
                if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() \
                        or tuple(t.shape) != shape:
                    raise ValueError("macros outputs must be contiguous float32 CUDA tensors")
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        self._ck(self._lib.lbm_macros(self._ctx, ptr(rho), ptr(u), ptr(wss)))
        return rho, u, wss

    def mass(self) -> float:
        m = C.c_double()
        self._ck(self._lib.lbm_mass(self._ctx, C.byref(m)))
        return m.value

    def weighted_sum(self, kind: int, weight=None) -> float:
        """sum_x weight[x] q(x) in float64 (q: OBJ_WSS wall shear stress,
        OBJ_DENSITY density); weight: [n] caller order (a CUDA float64 tensor,
        or anything numpy-like, copied to the device), None = all ones."""
        import torch
        w = None
        if weight is not None:
            w = weight if (hasattr(weight, "is_cuda") and weight.is_cuda and weight.dtype == torch.float64
                           and weight.is_contiguous()) else torch.as_tensor(
                np.ascontiguousarray(weight, dtype=np.float64)).cuda()
            if w.numel() != self.n:
                raise ValueError("weight must have n entries")
        out = C.c_double()
        self._ck(self._lib.lbm_weighted_sum(self._ctx, int(kind), None if w is None else C.c_void_p(w.data_ptr()),
                                            C.byref(out)))
        return out.value

    def get_populations(self) -> np.ndarray:
        f = np.empty((self.q, self.n), np.float64)
        self._ck(self._lib.lbm_get_populations(self._ctx, _p(f)))
        return f

    def get_populations_noalloc(self) -> np.ndarray:
        """As get_populations, staged in the library's static device array
        instead of a cudaMalloc buffer (q * n <= 2^20)."""
        f = np.empty((self.q, self.n), np.float64)
        self._ck(self._lib.lbm_get_populations_noalloc(self._ctx, _p(f)))
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (self.q, self.n):
            raise ValueError("populations must be [q, n]")
        self._ck(self._lib.lbm_set_populations(self._ctx, _p(f)))

    def state_bytes(self) -> int:
        b = C.c_size_t()
        self._ck(self._lib.lbm_state_bytes(self._ctx, C.byref(b)))
        return b.value

    def get_state(self) -> np.ndarray:
        buf = np.empty(self.state_bytes(), np.uint8)
        self._ck(self._lib.lbm_get_state(self._ctx, _p(buf), buf.nbytes))
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._ck(self._lib.lbm_set_state(self._ctx, _p(buf), buf.nbytes))

    def get_links(self) -> Tuple[np.ndarray, np.ndarray]:
        nbr = np.empty((self.q, self.n), np.int32)
        link = np.empty((self.q, self.n), np.uint8)
        self._ck(self._lib.lbm_get_links(self._ctx, _p(nbr), _p(link)))
        return nbr, link

    def set_stability_check(self, every: int, u_max: float = 0.3):
        """From now on lbm_step checks the state after every `every` steps (and
        after its last): LbmError LBM_ERR_UNSTABLE on a non-finite value or
        a site with rho <= 0 or |u| > u_max.  every = 0 turns it off."""
        self._ck(self._lib.lbm_set_stability_check(self._ctx, int(every), float(u_max)))

    def check_guards(self) -> bool:
        """True when every guard word after the planes of the population
        buffers is intact (no kernel wrote out of range)."""
        v = C.c_int32(0)
        self._ck(self._lib.lbm_check_guards(self._ctx, C.byref(v)))
        return bool(v.value)

    def set_tau(self, tau: float):
        self._ck(self._lib.lbm_set_tau(self._ctx, float(tau)))
        self.tau = float(tau)

    def set_iolets(self, rho_mean, amp, period, phase):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho_mean, amp, period, phase)]
        self._ck(self._lib.lbm_set_iolets(self._ctx, len(arrs[0]), *[_p(a) for a in arrs]))
        self._io = arrs

    def objective_grad(self, kind: int, weight, nsteps: int, t_begin: int, t_end: int,
                       scale: float = 1.0, n_snap: int = 16, want_df0: bool = False):
        """Run nsteps steps, return J and its gradient by the checkpointed
        discrete adjoint (``lbm_objective_grad``): a dict with J, dtau and
        per-iolet dmean, damp, dphase (float64), and dJ/df0 if asked."""
        w = np.ascontiguousarray(weight, dtype=np.float64)
        if w.shape != (self.n,):
            raise ValueError("weight must be [n]")
        obj = _Objective(int(kind), w.ctypes.data if self.n else None, int(t_begin), int(t_end),
                         float(scale))
        K = max(self.n_iolets, 1)
        J, dt = C.c_double(), C.c_double()
        dm, da, dp = np.zeros(K), np.zeros(K), np.zeros(K)
        df0 = np.zeros((self.q, self.n)) if want_df0 else None
        self._ck(self._lib.lbm_objective_grad(self._ctx, C.byref(obj), int(nsteps), int(n_snap),
                                              C.byref(J), C.byref(dt), _p(dm), _p(da), _p(dp),
                                              _p(df0)))
        out = dict(J=J.value, dtau=dt.value, dmean=dm[:self.n_iolets], damp=da[:self.n_iolets],
                   dphase=dp[:self.n_iolets])
        if want_df0:
            out["df0"] = df0
        return out

    def adjoint_counts(self):
        """(forward steps, adjoint steps) of the last objective_grad call."""
        f, a, ms = C.c_int64(), C.c_int64(), C.c_double()
        self._ck(self._lib.lbm_adjoint_counts(self._ctx, C.byref(f), C.byref(a), C.byref(ms)))
        return f.value, a.value

    def adjoint_sweep_ms(self) -> float:
        """Device time of the last objective_grad sweep (forward + adjoint)."""
        ms = C.c_double()
        self._ck(self._lib.lbm_adjoint_counts(self._ctx, None, None, C.byref(ms)))
        return ms.value

    def release_workspace(self):
        self._ck(self._lib.lbm_release_workspace(self._ctx))

    def info(self):
        n, npad, b = C.c_int64(), C.c_int64(), C.c_size_t()
        self._ck(self._lib.lbm_info(self._ctx, C.byref(n), C.byref(npad), C.byref(b)))
        return dict(n=n.value, npad=npad.value, device_bytes=b.value)

    def slab_chunks(self) -> int:
        """Slab chunks of the fused AA step pairs (0: steps run one by one)."""
        c = C.c_int32(0)
        self._ck(self._lib.lbm_slab_chunks(self._ctx, C.byref(c)))
        return int(c.value)

    def box(self):
        """Bounding box of the sites: (lo [3], dims [3]) as int tuples."""
        lo, dims = (C.c_int32 * 3)(), (C.c_int32 * 3)()
        self._ck(self._lib.lbm_lattice_box(self._ctx, lo, dims))
        return tuple(lo), tuple(dims)


# ---------------------------------------------------------------- rendering

class View:
    """Viewing and transfer-function parameters of ``lbm_render`` (steerable:
    ``orbit`` rotates the eye about the centre, ``zoom`` scales the field of
    view, ``tf_scale`` / ``tf_offset`` move the transfer function)."""

    def __init__(self, width: int, height: int, eye, center, up=(0.0, 0.0, 1.0), fov_y: float = 0.6,
                 dt: float = 0.5, tf_scale: float = 1.0, tf_offset: float = 0.0, lut=None,
                 a_stop: float = 0.99, filter: int = FILTER_TEXTURE, skip_empty: bool = True,
                 counters=None):
        self.width, self.height = int(width), int(height)
        self.eye = np.asarray(eye, np.float64).copy()
        self.center = np.asarray(center, np.float64).copy()
        self.up = np.asarray(up, np.float64).copy()
        self.fov_y, self.dt = float(fov_y), float(dt)
        self.tf_scale, self.tf_offset, self.a_stop = float(tf_scale), float(tf_offset), float(a_stop)
        self.lut = default_lut() if lut is None else np.asarray(lut, np.float32).reshape(256, 4)
        self.filter, self.skip_empty = int(filter), bool(skip_empty)
        # optional int64 CUDA tensor [2]: += samples composited, brick jumps
        self.counters = counters

    @classmethod
    def orbit(cls, center, distance: float, azimuth: float, elevation: float, width: int,
              height: int, **kw):
        """Eye on a sphere around center (angles in radians, z up)."""
        c = np.asarray(center, np.float64)
        d = np.array([math.cos(elevation) * math.cos(azimuth), math.cos(elevation) * math.sin(azimuth),
                      math.sin(elevation)])
        return cls(width, height, c + distance * d, c, up=(0.0, 0.0, 1.0), **kw)

    def zoom(self, factor: float) -> "View":
        """Narrow the field of view by factor (> 1 zooms in)."""
        self.fov_y = 2.0 * math.atan(math.tan(self.fov_y / 2.0) / float(factor))
        return self

    def _struct(self) -> _View:
        v = _View()
        v.width, v.height = self.width, self.height
        for name in ("eye", "center", "up"):
            arr = getattr(v, name)
            for a, x in enumerate(getattr(self, name)):
                arr[a] = float(x)
        v.fov_y, v.dt, v.tf_scale, v.tf_offset = self.fov_y, self.dt, self.tf_scale, self.tf_offset
        v.a_stop, v.filter, v.skip_empty = self.a_stop, self.filter, int(self.skip_empty)
        if self.counters is not None:
            c = self.counters
            if not c.is_cuda or c.numel() != 2 or c.element_size() != 8 or not c.is_contiguous():
                raise ValueError("counters must be a contiguous 2-element 64-bit CUDA tensor")
            v.counters_d = c.data_ptr()
        lut = np.ascontiguousarray(self.lut, dtype=np.float32)
        if lut.shape != (256, 4):
            raise ValueError("lut must be [256, 4]")
        C.memmove(C.addressof(v.lut), lut.ctypes.data, lut.nbytes)
        return v


def default_lut(alpha_max: float = 0.5) -> np.ndarray:
    """Blue-to-red RGBA table with opacity rising from 0 (value 0 is clear)."""
    s = np.arange(256, dtype=np.float64) / 255.0
    lut = np.zeros((256, 4), np.float32)
    lut[:, 0] = np.clip(1.5 * s, 0, 1)
    lut[:, 1] = np.clip(1.5 - np.abs(3.0 * s - 1.5), 0, 1)
    lut[:, 2] = np.clip(1.5 * (1.0 - s), 0, 1)
    lut[:, 3] = alpha_max * s * s
    return lut


class Volume:
    """A float voxel volume in a 3D texture (``lbm_volume_create``)."""

    def __init__(self, nx: int, ny: int, nz: int):
        self._lib = load_library()
        self._v = C.c_void_p()
        _check(self._lib.lbm_volume_create(int(nx), int(ny), int(nz), C.byref(self._v)))
        self.shape = (int(nz), int(ny), int(nx))

    @classmethod
    def for_lattice(cls, lattice: Lattice):
        """A volume covering the lattice's bounding box (and its origin)."""
        lo, dims = lattice.box()
        v = cls(max(dims[0], 1), max(dims[1], 1), max(dims[2], 1))
        v.origin = lo
        return v

    def close(self):
        if getattr(self, "_v", None) and self._v.value:
            self._lib.lbm_volume_destroy(self._v)
            self._v = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_dense(self, t):
        import torch
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != self.shape:
            raise ValueError("volume data must be a contiguous float32 CUDA tensor of shape %s"
                             % (self.shape,))

    def upload(self, vol, stream=None):
        """Copy a [nz, ny, nx] float32 CUDA tensor into the volume."""
        self._check_dense(vol)
        _check(self._lib.lbm_volume_upload(self._v, C.c_void_p(vol.data_ptr()), _stream_handle(stream)))

    def download(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        self._check_dense(out)
        _check(self._lib.lbm_volume_download(self._v, C.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    def from_lattice(self, lattice: Lattice, quantity: int = QTY_SPEED, origin=None):
        """Write a quantity of the lattice's current state (on its stream)."""
        org = getattr(self, "origin", (0, 0, 0)) if origin is None else origin
        o = (C.c_int32 * 3)(*[int(x) for x in org])
        lattice._ck(self._lib.lbm_volume_from_lattice(self._v, lattice._ctx, int(quantity), o))

    def render(self, view: View, out=None, stream=None):
        """RGBA image float32 [height, width, 4] (CUDA tensor)."""
        import torch
        if out is None:
            out = torch.empty(view.height, view.width, 4, dtype=torch.float32, device="cuda")
        if out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous() \
                or tuple(out.shape) != (view.height, view.width, 4):
            raise ValueError("out must be a contiguous float32 CUDA tensor [height, width, 4]")
        v = view._struct()
        _check(self._lib.lbm_render(self._v, C.byref(v), C.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out


def save_ppm(path: str, rgba, background=(0.0, 0.0, 0.0)):
    """Write an RGBA float image (array or tensor [H, W, 4]) over a background
    as a binary PPM file."""
    img = rgba.detach().cpu().numpy() if hasattr(rgba, "detach") else np.asarray(rgba)
    rgb = img[..., :3] + (1.0 - img[..., 3:4]) * np.asarray(background, np.float32)
    b = (np.clip(rgb, 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8)
    with open(path, "wb") as fh:
        fh.write(b"P6\n%d %d\n255\n" % (b.shape[1], b.shape[0]))
        fh.write(b.tobytes())


class HemeObjective:
    """Time-windowed objective J(tau, mean, amp, phase) of a simulation as a
    differentiable torch function.

    ``HemeObjective(lattice, kind, weight, nsteps, t_begin, t_end, ...)``
    snapshots the lattice's current state; calling it with torch tensors
    (tau: scalar; mean, amp, phase: [K]) restarts from that state, runs the
    forward solver and the discrete adjoint (``lbm_objective_grad``) in one
    go, and returns J as a float64 tensor whose ``backward`` delivers the
    adjoint gradient.  The solver state is not part of the graph.
    """

    def __init__(self, lattice: "Lattice", kind: int, weight, nsteps: int, t_begin: int,
                 t_end: int, scale: float = 1.0, n_snap: int = 16, period=None):
        self.L = lattice
        self.kind, self.nsteps = int(kind), int(nsteps)
        self.t_begin, self.t_end, self.scale, self.n_snap = int(t_begin), int(t_end), float(scale), int(n_snap)
        self.weight = np.ascontiguousarray(weight, dtype=np.float64)
        self.period = np.ascontiguousarray(lattice._io[2] if period is None else period, dtype=np.float64)
        self.state0 = lattice.get_state()
        self.t0 = lattice.time

    def evaluate(self, tau: float, mean, amp, phase):
        L = self.L
        L.set_state(self.state0)
        L.set_time(self.t0)
        L.set_tau(tau)
        L.set_iolets(mean, amp, self.period, phase)
        return L.objective_grad(self.kind, self.weight, self.nsteps, self.t_begin, self.t_end,
                                self.scale, self.n_snap)

    def __call__(self, tau, mean, amp, phase):
        import torch

        fn = _objective_function()
        return fn.apply(self, tau, mean, amp, phase)


_FN = None


def _objective_function():
    global _FN
    if _FN is not None:
        return _FN
    import torch

    class _HemeObjectiveFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, obj, tau, mean, amp, phase):
            r = obj.evaluate(float(tau.detach().cpu()), mean.detach().cpu().numpy(),
                             amp.detach().cpu().numpy(), phase.detach().cpu().numpy())
            f64 = dict(dtype=torch.float64)
            ctx.grads = (torch.tensor(r["dtau"], **f64), torch.as_tensor(r["dmean"], **f64),
                         torch.as_tensor(r["damp"], **f64), torch.as_tensor(r["dphase"], **f64))
            ctx.devs = [t.device for t in (tau, mean, amp, phase)]
            ctx.dtypes = [t.dtype for t in (tau, mean, amp, phase)]
            return torch.tensor(r["J"], dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            out = [None]
            for g, dev, dt in zip(ctx.grads, ctx.devs, ctx.dtypes):
                out.append((gJ.to(torch.float64) * g).to(device=dev, dtype=dt))
            return tuple(out)

    _FN = _HemeObjectiveFn
    return _FN
