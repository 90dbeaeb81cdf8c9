"""Seeded synthetic vessel geometries: the inputs of the lattice-Boltzmann path.

This module only decides *which voxels are fluid* and *which voxels outside the
fluid are inlet/outlet ("iolet") voxels*, and draws seeded random numbers.  It
holds none of the method's arithmetic (no lattice, no links, no collision): the
CUDA library and the FP64 oracle each build their own neighbour tables from the
site list produced here, so that both sides see identical inputs and nothing
else.

The paper evaluates on patient geometries (3D rotational angiography turned
into STL files, Section 4, Table II: 296,814 and 132,910 fluid sites).  Those
files are not available, so the shapes below stand in for them:

* ``tube``            straight cylinder, radius 8, length 64 (Poiseuille case),
* ``aneurysm``        quarter-arc tube of radius 20 with a fused sphere of radius
                      40 (saccular aneurysm) in a 256^3 box,
* ``vessel_tree``     seeded bifurcating tree, six generations, Murray's law,
                      in a 1024^3 box,
* ``periodic_box``, ``walled_box``, ``slab``, ``random_mask``: small closed or
                      periodic domains for invariants and brute-force checks.

Voxelisation rule (the same for every shape): a voxel with integer centre p is
fluid iff its squared distance to the shape is <= r^2, compared in float64.
Iolet voxels are non-fluid voxels just beyond an open end of the vessel, within
the end disk; a lattice link from a fluid site into such a voxel is an iolet
link, every other link into a non-fluid voxel is a wall link.

Caller order of the sites is the lexicographic (z, y, x) order of the voxels.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Geometry",
    "tube",
    "aneurysm",
    "vessel_tree",
    "periodic_box",
    "walled_box",
    "slab",
    "random_mask",
    "random_populations",
]


@dataclass
class Geometry:
    """A sparse fluid-site list plus its iolet voxels and iolet schedule.

    xyz:       int32 [N, 3] fluid voxel coordinates (caller order).
    io_xyz:    int32 [M, 3] non-fluid voxels that are iolet k = io_id[m].
    io_id:     int32 [M].
    periodic:  int32 [3], box extent per axis for periodic wrap, 0 = open.
    rho_mean, amp, period, phase: float64 [K] density schedule of iolet k,
               rho_k(t) = rho_mean + amp * sin(2 pi t / period + phase)
               (period 0 = constant).
    site_weight: optional float64 [N] objective weights (e.g. the aneurysm
               sphere sites for a wall-shear-stress objective).
    """

    name: str
    xyz: np.ndarray
    io_xyz: np.ndarray
    io_id: np.ndarray
    periodic: np.ndarray
    rho_mean: np.ndarray
    amp: np.ndarray
    period: np.ndarray
    phase: np.ndarray
    site_weight: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_iolets(self) -> int:
        return int(self.rho_mean.shape[0])


# --------------------------------------------------------------------------
# voxel-set helpers
# --------------------------------------------------------------------------

_KEY_BITS = 21
_KEY_OFF = 1 << 20  # coordinates may be slightly negative (iolet planes)


def _keys(xyz: np.ndarray) -> np.ndarray:
    """Lexicographic (z, y, x) integer key; monotone in caller order."""
    v = xyz.astype(np.int64) + _KEY_OFF
    return (v[:, 2] << (2 * _KEY_BITS)) | (v[:, 1] << _KEY_BITS) | v[:, 0]


def _unkeys(k: np.ndarray) -> np.ndarray:
    m = (1 << _KEY_BITS) - 1
    out = np.empty((k.shape[0], 3), dtype=np.int64)
    out[:, 0] = k & m
    out[:, 1] = (k >> _KEY_BITS) & m
    out[:, 2] = k >> (2 * _KEY_BITS)
    return (out - _KEY_OFF).astype(np.int32)


def _scan_box(lo: Sequence[int], hi: Sequence[int],
              pred: Callable[[np.ndarray, np.ndarray, np.ndarray], np.ndarray],
              chunk: int = 1 << 22) -> np.ndarray:
    """Keys of all integer voxels p in [lo, hi) (per axis) with pred(x,y,z)."""
    lo = [int(v) for v in lo]
    hi = [int(v) for v in hi]
    if any(h <= l for l, h in zip(lo, hi)):
        return np.empty(0, dtype=np.int64)
    nx, ny = hi[0] - lo[0], hi[1] - lo[1]
    xs = np.arange(lo[0], hi[0], dtype=np.float64)
    ys = np.arange(lo[1], hi[1], dtype=np.float64)
    X2, Y2 = np.meshgrid(xs, ys, indexing="xy")  # [ny, nx]
    X2 = X2.ravel()
    Y2 = Y2.ravel()
    slab_z = max(1, chunk // max(1, nx * ny))
    out: List[np.ndarray] = []
    for z0 in range(lo[2], hi[2], slab_z):
        zs = np.arange(z0, min(hi[2], z0 + slab_z), dtype=np.float64)
        X = np.tile(X2, zs.shape[0])
        Y = np.tile(Y2, zs.shape[0])
        Z = np.repeat(zs, X2.shape[0])
        m = pred(X, Y, Z)
        if m.any():
            p = np.stack([X[m], Y[m], Z[m]], axis=1).astype(np.int32)
            out.append(_keys(p))
    if not out:
        return np.empty(0, dtype=np.int64)
    return np.concatenate(out)


def _scan_all(scans) -> List[np.ndarray]:
    """_scan_box over a list of (lo, hi, predicate), on a few threads (the
    array operations release the interpreter lock); results in list order."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    workers = max(1, min(8, os.cpu_count() or 1, len(scans)))
    if workers == 1:
        return [_scan_box(lo, hi, pred) for lo, hi, pred in scans]
    with ThreadPoolExecutor(workers) as ex:
        return list(ex.map(lambda t: _scan_box(*t), scans))


def _finish(name: str, fluid_keys: List[np.ndarray], io_sets: List[np.ndarray],
            periodic=(0, 0, 0), rho_mean=(), amp=None, period=None, phase=None,
            meta=None) -> Geometry:
    # distinct fluid keys in ascending order (a sort and a neighbour test: on
    # tens of millions of keys much faster than np.unique's hashing path)
    fk = np.sort(np.concatenate(fluid_keys)) if fluid_keys else np.empty(0, np.int64)
    if fk.shape[0] > 1:
        fk = fk[np.concatenate(([True], fk[1:] != fk[:-1]))]
    # iolet voxels: drop those that are fluid; a voxel claimed by several
    # iolets goes to the lowest id
    if io_sets:
        ik = np.concatenate([np.asarray(s, dtype=np.int64) for s in io_sets])
        iid = np.concatenate([np.full(len(s), k, dtype=np.int32)
                              for k, s in enumerate(io_sets)])
    else:
        ik = np.empty(0, np.int64)
        iid = np.empty(0, np.int32)
    if fk.shape[0] and ik.shape[0]:
        pos = np.minimum(np.searchsorted(fk, ik), fk.shape[0] - 1)
        keep = fk[pos] != ik
        ik, iid = ik[keep], iid[keep]
    order = np.lexsort((iid, ik))
    ik, iid = ik[order], iid[order]
    first = np.ones(ik.shape[0], dtype=bool)
    first[1:] = ik[1:] != ik[:-1]
    ik, iid = ik[first], iid[first]
    order = np.lexsort((ik, iid))  # group by iolet id, then voxel order
    io_keys = [ik[order]]
    io_ids = [iid[order]]
    K = len(rho_mean)
    z = np.zeros(K, dtype=np.float64)
    g = Geometry(
        name=name,
        xyz=_unkeys(fk),
        io_xyz=_unkeys(np.concatenate(io_keys)) if io_keys else np.empty((0, 3), np.int32),
        io_id=np.concatenate(io_ids) if io_ids else np.empty(0, np.int32),
        periodic=np.asarray(periodic, dtype=np.int32),
        rho_mean=np.asarray(rho_mean, dtype=np.float64),
        amp=z.copy() if amp is None else np.asarray(amp, dtype=np.float64),
        period=z.copy() if period is None else np.asarray(period, dtype=np.float64),
        phase=z.copy() if phase is None else np.asarray(phase, dtype=np.float64),
        meta=dict(meta or {}),
    )
    return g


def _sites_where(g: Geometry, pred) -> np.ndarray:
    p = g.xyz.astype(np.float64)
    return pred(p[:, 0], p[:, 1], p[:, 2])


# --------------------------------------------------------------------------
# shapes
# --------------------------------------------------------------------------

def tube(radius: float = 8.0, length: int = 64, nx: int = 17, ny: int = 17,
         rho_in: float = 1.001, rho_out: float = 0.999) -> Geometry:
    """Straight cylinder along z, axis at the box centre, open at both ends.

    Fluid iff (x-cx)^2 + (y-cy)^2 <= r^2 for z in [0, length).  Inlet voxels
    are the disk at z = -1 (iolet 0), outlet voxels the disk at z = length
    (iolet 1).  With r = 8 in a 17x17x64 box this gives 12,608 fluid sites.
    """
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    r2 = float(radius) ** 2

    def disk(X, Y, Z):
        return (X - cx) ** 2 + (Y - cy) ** 2 <= r2

    fluid = _scan_box((0, 0, 0), (nx, ny, length), disk)
    inlet = _scan_box((0, 0, -1), (nx, ny, 0), disk)
    outlet = _scan_box((0, 0, length), (nx, ny, length + 1), disk)
    return _finish("tube_r%g_L%d" % (radius, length), [fluid], [inlet, outlet],
                   rho_mean=(rho_in, rho_out),
                   meta=dict(radius=radius, length=length, box=(nx, ny, length),
                             shape=dict(kind="cylinder_z", center=(cx, cy), r=float(radius))))


def aneurysm(tube_r: float = 20.0, arc_R: float = 150.0, sphere_r: float = 40.0,
             box: int = 256, arc_c=(40.0, 40.0, 128.0), rho_in: float = 1.0,
             amp_in: float = 0.001, period_in: float = 4000.0,
             rho_out: float = 1.0) -> Geometry:
    """Saccular aneurysm: a tube bent along a quarter circle plus a fused sphere.

    Centreline: arc of radius arc_R about arc_c in the plane z = arc_c[2],
    angle 0..pi/2, continued by straight segments to the box faces y = 0 (at
    angle 0) and x = 0 (at angle pi/2).  The sphere is centred at mid-arc on
    radius arc_R + tube_r + sphere_r/2 from the arc centre, so that it overlaps
    the outer tube wall by sphere_r/2.  Inlet (iolet 0): the end disk at
    y = -1, pulsatile rho = rho_in + amp_in sin(2 pi t / period_in).
    Outlet (iolet 1): the end disk at x = -1, constant rho_out.
    Objective weights mark the sphere sites that are outside the tube.
    """
    shape = dict(kind="aneurysm", tube_r=float(tube_r), arc_R=float(arc_R),
                 sphere_r=float(sphere_r), arc_c=tuple(float(v) for v in arc_c))
    fluid_pred, tube_d2, (sx, sy, sz), (e0, e1) = _aneurysm_parts(shape)
    ax, ay, az = arc_c
    r2 = tube_r ** 2

    fluid = _scan_box((0, 0, 0), (box, box, box), fluid_pred)
    inlet = _scan_box((0, -1, 0), (box, 0, box),
                      lambda X, Y, Z: (X - e0[0]) ** 2 + (Z - az) ** 2 <= r2)
    outlet = _scan_box((-1, 0, 0), (0, box, box),
                       lambda X, Y, Z: (Y - e1[1]) ** 2 + (Z - az) ** 2 <= r2)
    g = _finish("aneurysm_r%g_R%g_s%g" % (tube_r, arc_R, sphere_r), [fluid],
                [inlet, outlet], rho_mean=(rho_in, rho_out), amp=(amp_in, 0.0),
                period=(period_in, 0.0), phase=(0.0, 0.0),
                meta=dict(box=(box, box, box), sphere_c=(sx, sy, sz),
                          sphere_r=sphere_r, shape=shape))
    w = _sites_where(g, lambda X, Y, Z: (((X - sx) ** 2 + (Y - sy) ** 2 + (Z - sz) ** 2
                                          <= sphere_r ** 2)
                                         & (tube_d2(X, Y, Z) > r2)))
    g.site_weight = w.astype(np.float64)
    return g


def _aneurysm_parts(shape):
    """Inside predicate of the aneurysm shape, the squared distance to its
    tube centreline, the sphere centre and the two arc ends."""
    tube_r, arc_R, sphere_r = shape["tube_r"], shape["arc_R"], shape["sphere_r"]
    ax, ay, az = shape["arc_c"]
    r2 = tube_r ** 2
    s_dist = arc_R + tube_r + sphere_r / 2.0
    sx = ax + s_dist * math.cos(math.pi / 4)
    sy = ay + s_dist * math.sin(math.pi / 4)
    sz = az
    e0 = (ax + arc_R, ay)          # arc end at angle 0, straight part toward y=0
    e1 = (ax, ay + arc_R)          # arc end at angle pi/2, straight part toward x=0

    def tube_d2(X, Y, Z):
        dx, dy = X - ax, Y - ay
        rr = np.sqrt(dx * dx + dy * dy)
        th = np.arctan2(dy, dx)
        on_arc = (th >= 0.0) & (th <= math.pi / 2)
        d_arc = np.where(on_arc, (rr - arc_R) ** 2 + (Z - az) ** 2, np.inf)
        # straight segment 0: x = e0.x, y in [-inf, e0.y]
        d_s0 = np.where(Y <= e0[1], (X - e0[0]) ** 2 + (Z - az) ** 2, np.inf)
        d_s1 = np.where(X <= e1[0], (Y - e1[1]) ** 2 + (Z - az) ** 2, np.inf)
        return np.minimum(d_arc, np.minimum(d_s0, d_s1))

    def fluid_pred(X, Y, Z):
        in_tube = tube_d2(X, Y, Z) <= r2
        in_sph = (X - sx) ** 2 + (Y - sy) ** 2 + (Z - sz) ** 2 <= sphere_r ** 2
        return in_tube | in_sph

    return fluid_pred, tube_d2, (sx, sy, sz), (e0, e1)


def _perp_basis(d: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    h = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = h - np.dot(h, d) * d
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    return e1, e2


def _tree_segments(seed: int, generations: int, root_r: float, length_factor: float,
                   root_start, murray_exp: float = 3.0):
    """Seeded binary tree: list of (start, dir, radius, length, gen, is_leaf)."""
    rng = np.random.default_rng(seed)
    segs = []
    queue = [(np.asarray(root_start, dtype=np.float64), np.array([0.0, 0.0, 1.0]),
              float(root_r), 0)]
    while queue:
        nxt = []
        for start, d, r, gen in queue:
            L = length_factor * r
            leaf = gen == generations - 1
            segs.append((start, d, r, L, gen, leaf))
            if leaf:
                continue
            end = start + L * d
            a = rng.uniform(0.7, 1.0)
            th1 = math.radians(rng.uniform(25.0, 45.0))
            th2 = math.radians(rng.uniform(25.0, 45.0))
            phi = rng.uniform(0.0, 2.0 * math.pi)
            r1 = r / (1.0 + a ** murray_exp) ** (1.0 / murray_exp)
            r2 = a * r1
            e1, e2 = _perp_basis(d)
            m = math.cos(phi) * e1 + math.sin(phi) * e2
            d1 = math.cos(th1) * d + math.sin(th1) * m
            d2 = math.cos(th2) * d - math.sin(th2) * m
            nxt.append((end, d1 / np.linalg.norm(d1), r1, gen + 1))
            nxt.append((end, d2 / np.linalg.norm(d2), r2, gen + 1))
        queue = nxt
    return segs


def _tree_layout(shape):
    """Segments of the tree shape, shifted so that the tree is centred in x
    and y in its box: list of (start, dir, radius, length, gen, is_leaf)."""
    segs = _tree_segments(shape["seed"], shape["generations"], shape["root_r"],
                          shape["length_factor"], (0.0, 0.0, 0.0))
    box = shape["box"]
    lo = np.min([np.minimum(s[0], s[0] + s[3] * s[1]) - s[2] for s in segs], axis=0)
    hi = np.max([np.maximum(s[0], s[0] + s[3] * s[1]) + s[2] for s in segs], axis=0)
    shift = np.array([math.floor(box / 2.0 - (lo[0] + hi[0]) / 2.0),
                      math.floor(box / 2.0 - (lo[1] + hi[1]) / 2.0), 0.0])
    return [(s[0] + shift,) + tuple(s[1:]) for s in segs]


def vessel_tree(seed: int = 1906, generations: int = 6, root_r: float = 48.0,
                length_factor: float = 5.5, box: int = 1024,
                rho_in: float = 1.001, rho_out: float = 1.0) -> Geometry:
    """Seeded random bifurcating vessel tree (binary, ``generations`` levels).

    Root: radius root_r, starting at z = 0 along +z, its (x, y) chosen so that
    the tree's bounding box is centred in x and y.  At each
    bifurcation a ~ U(0.7, 1.0) sets the asymmetry; the children radii follow
    Murray's law with exponent 3, r1 = r / (1 + a^3)^(1/3), r2 = a r1; branch
    angles U(25, 45) degrees on either side of the parent axis in a plane of
    random azimuth U(0, 2 pi).  Every branch has length length_factor * r.
    Fluid = union of flat-ended cylinders plus a sphere of the parent radius
    at every bifurcation point, clipped to the box.  Iolet 0 is the root's
    start disk (inlet, rho_in); iolets 1..2^(g-1) are the leaf end disks
    (outlets, rho_out), numbered in breadth-first order.  With the defaults
    (length 5.5 r) the whole tree lies inside the 1024^3 box.
    """
    shape = dict(kind="tree", seed=int(seed), generations=int(generations), root_r=float(root_r),
                 length_factor=float(length_factor), box=int(box))
    segs = _tree_layout(shape)
    scans = []  # (lo, hi, predicate) per cylinder and per bifurcation sphere

    def clip_lo_hi(lo, hi):
        lo = np.maximum(np.floor(lo), 0).astype(int)
        hi = np.minimum(np.ceil(hi) + 1, box).astype(int)
        return lo, hi

    for start, d, r, L, gen, leaf in segs:
        end = start + L * d
        lo, hi = clip_lo_hi(np.minimum(start, end) - r - 1, np.maximum(start, end) + r + 1)

        def cyl(X, Y, Z, start=start, d=d, r=r, L=L):
            px, py, pz = X - start[0], Y - start[1], Z - start[2]
            s = px * d[0] + py * d[1] + pz * d[2]
            qx, qy, qz = px - s * d[0], py - s * d[1], pz - s * d[2]
            return (s >= 0.0) & (s <= L) & (qx * qx + qy * qy + qz * qz <= r * r)

        scans.append((lo, hi, cyl))
        if not leaf:
            lo, hi = clip_lo_hi(end - r - 1, end + r + 1)

            def sph(X, Y, Z, c=end, r=r):
                return (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r

            scans.append((lo, hi, sph))

    fluid_keys = _scan_all(scans)

    def end_disk(c, n, r):
        lo = np.floor(c - r - 3).astype(int)
        hi = np.ceil(c + r + 3).astype(int) + 1

        def pred(X, Y, Z):
            px, py, pz = X - c[0], Y - c[1], Z - c[2]
            s = px * n[0] + py * n[1] + pz * n[2]
            qx, qy, qz = px - s * n[0], py - s * n[1], pz - s * n[2]
            return (s > 0.0) & (s <= 2.0) & (qx * qx + qy * qy + qz * qz <= r * r)

        return _scan_box(lo, hi, pred)

    io_sets = []
    s0, d0, r0 = segs[0][0], segs[0][1], segs[0][2]
    io_sets.append(end_disk(s0, -d0, r0))
    leaves = [s for s in segs if s[5]]
    for start, d, r, L, gen, leaf in leaves:
        io_sets.append(end_disk(start + L * d, d, r))
    K = len(io_sets)
    rho_mean = [rho_in] + [rho_out] * (K - 1)
    g = _finish("vessel_tree_s%d_g%d_r%g" % (seed, generations, root_r), fluid_keys,
                io_sets, rho_mean=rho_mean,
                meta=dict(box=(box, box, box), segments=len(segs), leaves=len(leaves), shape=shape))
    return g


def periodic_box(nx: int, ny: int, nz: int) -> Geometry:
    """Every voxel of an nx*ny*nz box is fluid and every axis wraps around."""
    fluid = _scan_box((0, 0, 0), (nx, ny, nz), lambda X, Y, Z: np.ones_like(X, dtype=bool))
    return _finish("periodic_%dx%dx%d" % (nx, ny, nz), [fluid], [],
                   periodic=(nx, ny, nz), rho_mean=())


def walled_box(nx: int, ny: int, nz: int) -> Geometry:
    """A closed box: every link leaving it is a wall link, no iolets."""
    fluid = _scan_box((0, 0, 0), (nx, ny, nz), lambda X, Y, Z: np.ones_like(X, dtype=bool))
    return _finish("walled_%dx%dx%d" % (nx, ny, nz), [fluid], [], rho_mean=())


def slab(nx: int, ny: int, h: int, rho_in: float = 1.001,
         rho_out: float = 0.999) -> Geometry:
    """Plane channel: fluid z in [0, h), periodic in y, walls at z = -1 and
    z = h (halfway walls at z = -1/2 and h - 1/2), inlet plane x = -1
    (iolet 0), outlet plane x = nx (iolet 1)."""
    allp = lambda X, Y, Z: np.ones_like(X, dtype=bool)
    fluid = _scan_box((0, 0, 0), (nx, ny, h), allp)
    inlet = _scan_box((-1, 0, 0), (0, ny, h), allp)
    outlet = _scan_box((nx, 0, 0), (nx + 1, ny, h), allp)
    return _finish("slab_%dx%dx%d" % (nx, ny, h), [fluid], [inlet, outlet],
                   periodic=(0, ny, 0), rho_mean=(rho_in, rho_out),
                   meta=dict(h=h, nx=nx))


def random_mask(shape=(6, 6, 6), p: float = 0.6, seed: int = 0, n_iolets: int = 2,
                periodic: bool = False, p_io: float = 0.3) -> Geometry:
    """A seeded random fluid mask in a small box (for brute-force checks).

    Each voxel is fluid with probability p.  Non-fluid voxels inside the box
    and on its one-voxel skin become iolet k (k uniform in [0, n_iolets)) with
    probability p_io, otherwise they are walls.  With periodic=True the box
    wraps around and only interior non-fluid voxels can be iolets.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    m = rng.random((nz, ny, nx)) < p
    zz, yy, xx = np.nonzero(m)
    fluid = _keys(np.stack([xx, yy, zz], 1).astype(np.int32))
    lo = (0, 0, 0) if periodic else (-1, -1, -1)
    hi = (nx, ny, nz) if periodic else (nx + 1, ny + 1, nz + 1)
    io_sets = [[] for _ in range(n_iolets)]
    if n_iolets:
        for z in range(lo[2], hi[2]):
            for y in range(lo[1], hi[1]):
                for x in range(lo[0], hi[0]):
                    inside = 0 <= x < nx and 0 <= y < ny and 0 <= z < nz
                    if inside and m[z, y, x]:
                        continue
                    if rng.random() < p_io:
                        io_sets[int(rng.integers(0, n_iolets))].append((x, y, z))
    io = [_keys(np.asarray(s, dtype=np.int32).reshape(-1, 3)) for s in io_sets]
    rho_mean = 1.0 + 0.002 * (rng.random(n_iolets) - 0.5)
    amp = 0.001 * rng.random(n_iolets)
    period = rng.uniform(20.0, 60.0, n_iolets)
    phase = rng.uniform(0.0, 2 * math.pi, n_iolets)
    return _finish("random_%dx%dx%d_p%g_s%d" % (nx, ny, nz, p, seed), [fluid], io,
                   periodic=shape if periodic else (0, 0, 0), rho_mean=rho_mean,
                   amp=amp, period=period, phase=phase)


def random_populations(q: int, n: int, seed: int, amplitude: float = 1e-3,
                       rho0: float = 1.0) -> np.ndarray:
    """Seeded float64 [q, n] populations: (1 + amplitude * U(-1, 1)) times a
    per-direction base value rho0 / q.  These are raw random inputs, not an
    equilibrium; both sides receive the same array."""
    rng = np.random.default_rng(seed)
    base = rho0 / q
    return base * (1.0 + amplitude * (2.0 * rng.random((q, n)) - 1.0))


# --------------------------------------------------------------------------
# wall positions along the lattice links (for interpolated walls)
# --------------------------------------------------------------------------

Q_QUANTUM = 2.0 ** -24  # wall fractions are multiples of this


def _quantise(qv: np.ndarray) -> np.ndarray:
    k = np.clip(np.round(qv / Q_QUANTUM), 1, 1 / Q_QUANTUM)
    return k * Q_QUANTUM


def _quad_interval(alpha, beta, gamma):
    """Interval [a, b] of s with alpha s^2 + beta s + gamma <= 0 (alpha >= 0);
    empty intervals come back with a > b."""
    a = np.full(alpha.shape, np.inf)
    b = np.full(alpha.shape, -np.inf)
    lin = alpha <= 0.0
    a[lin & (gamma <= 0.0)] = -np.inf
    b[lin & (gamma <= 0.0)] = np.inf
    disc = beta * beta - 4.0 * alpha * gamma
    ok = ~lin & (disc >= 0.0)
    sq = np.sqrt(np.where(ok, disc, 0.0))
    a[ok] = (-beta[ok] - sq[ok]) / (2.0 * alpha[ok])
    b[ok] = (-beta[ok] + sq[ok]) / (2.0 * alpha[ok])
    return a, b


def _cylinder_interval(p, c, start, d, r, L):
    """s-interval where p + s c lies in the capped cylinder (axis start + t d,
    t in [0, L], radius r)."""
    w = p - start
    wd, cd = w @ d, c @ d
    wp = w - wd[:, None] * d
    cp = c - cd[:, None] * d
    a, b = _quad_interval((cp * cp).sum(1), 2.0 * (wp * cp).sum(1), (wp * wp).sum(1) - r * r)
    with np.errstate(divide="ignore", invalid="ignore"):
        t0, t1 = (0.0 - wd) / cd, (L - wd) / cd
    par = cd == 0.0
    lo = np.where(par, np.where((wd >= 0) & (wd <= L), -np.inf, np.inf), np.minimum(t0, t1))
    hi = np.where(par, np.where((wd >= 0) & (wd <= L), np.inf, -np.inf), np.maximum(t0, t1))
    return np.maximum(a, lo), np.minimum(b, hi)


def _sphere_interval(p, c, centre, r):
    w = p - centre
    return _quad_interval((c * c).sum(1), 2.0 * (w * c).sum(1), (w * w).sum(1) - r * r)


def _union_exit(link_id, a, b, n_links):
    """First exit s >= 0 from the union of the intervals of each link,
    starting inside at s = 0 (NaN where no interval contains 0)."""
    order = np.argsort(link_id, kind="stable")
    link_id, a, b = link_id[order], a[order], b[order]
    out = np.full(n_links, np.nan)
    if link_id.size == 0:
        return out
    starts = np.flatnonzero(np.r_[True, link_id[1:] != link_id[:-1]])
    ids = link_id[starts]
    cur = np.maximum.reduceat(np.where((a <= 0.0) & (b >= 0.0), b, -np.inf), starts)
    for _ in range(8):
        nxt = np.maximum.reduceat(np.where((a <= np.repeat(cur, np.diff(np.r_[starts, a.size])))
                                           & (b >= 0.0), b, -np.inf), starts)
        nxt = np.maximum(nxt, cur)
        if np.array_equal(nxt, cur):
            break
        cur = nxt
    out[ids] = np.where(np.isfinite(cur) & (cur >= 0.0), cur, np.nan)
    return out


def _bisect_exit(pred, p, c, samples=16, iters=30):
    """First s in (0, 1] where pred turns false along p + s c (1 if never)."""
    lo = np.zeros(p.shape[0])
    hi = np.ones(p.shape[0])
    found = np.zeros(p.shape[0], dtype=bool)
    for j in range(1, samples + 1):
        s = j / samples
        q = p + s * c
        out = ~pred(q[:, 0], q[:, 1], q[:, 2]) & ~found
        hi[out] = s
        lo[out] = (j - 1) / samples
        found |= out
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        q = p + mid[:, None] * c
        ins = pred(q[:, 0], q[:, 1], q[:, 2])
        lo = np.where(ins & found, mid, lo)
        hi = np.where(~ins & found, mid, hi)
    return np.where(found, hi, 1.0)


def wall_fractions(g: Geometry, vectors, link) -> np.ndarray:
    """Fraction of each wall link that lies in the fluid, from the analytic
    shape the geometry was voxelised from: for a fluid site p and a wall link
    along the lattice vector c (link[i][x] == 1), the first s in (0, 1] where
    p + s c leaves the shape, rounded to a multiple of 2^-24 (the wall crosses
    the link at p + s c).  float64 [q, n]; 0.5 (the half-way wall) for links
    that are not walls, for shapes without a description, and where the
    shape does not contain p.  ``vectors`` [q, 3] are the lattice vectors in
    the link table's direction order."""
    e = np.asarray(vectors, dtype=np.float64).reshape(-1, 3)
    link = np.asarray(link)
    qn = e.shape[0]
    out = np.full((qn, g.n), 0.5)
    shape = g.meta.get("shape")
    if shape is None or g.n == 0:
        return out
    ii, xx = np.nonzero(link == 1)
    if ii.size == 0:
        return out
    p = g.xyz[xx].astype(np.float64)
    c = e[ii]
    kind = shape["kind"]
    if kind == "cylinder_z":
        cx, cy = shape["center"]
        r = shape["r"]
        a, b = _quad_interval(c[:, 0] ** 2 + c[:, 1] ** 2,
                              2.0 * ((p[:, 0] - cx) * c[:, 0] + (p[:, 1] - cy) * c[:, 1]),
                              (p[:, 0] - cx) ** 2 + (p[:, 1] - cy) ** 2 - r * r)
        sv = np.where((a <= 0.0) & (b >= 0.0), b, np.nan)
    elif kind == "aneurysm":
        pred = _aneurysm_parts(shape)[0]
        sv = _bisect_exit(pred, p, c)
    elif kind == "tree":
        segs = _tree_layout(shape)
        ids, As, Bs = [], [], []
        for start, d, r, L, gen, leaf in segs:
            end = start + L * d
            lo = np.minimum(start, end) - r - 2.0
            hi = np.maximum(start, end) + r + 2.0
            sel = np.flatnonzero(np.all((p >= lo) & (p <= hi), axis=1))
            if sel.size:
                a, b = _cylinder_interval(p[sel], c[sel], start, d, r, L)
                ids.append(sel); As.append(a); Bs.append(b)
            if not leaf:
                sel = np.flatnonzero(np.all((p >= end - r - 2.0) & (p <= end + r + 2.0), axis=1))
                if sel.size:
                    a, b = _sphere_interval(p[sel], c[sel], end, r)
                    ids.append(sel); As.append(a); Bs.append(b)
        if ids:
            sv = _union_exit(np.concatenate(ids), np.concatenate(As), np.concatenate(Bs), ii.size)
        else:
            sv = np.full(ii.size, np.nan)
    else:
        return out
    sv = np.where(np.isnan(sv), 0.5, np.minimum(sv, 1.0))
    out[ii, xx] = _quantise(sv)
    return out
