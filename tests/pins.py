"""Checks that pin the FP64 oracle to facts outside itself.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError when the
oracle disagrees with a closed form, an invariant, a textbook special case or
a brute-force computation.  The same functions run against the real oracle
(they must pass) and against copies of it with a planted mistake (at least
one of them must fail), see test_oracle_mutants.py.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np

from paper_1906_11925_gb300 import geometry as G

TAU_EXACT_BB = 0.5 + math.sqrt(3.0 / 16.0)  # halfway bounce-back has zero slip here


# ---------------------------------------------------------------- lattice

def _rational_weights(vecs):
    """Weights of a three-shell 3D velocity set, by speed shell, from the
    isotropy conditions sum w = 1, sum w c_x^2 = 1/3 and
    sum w c_x^2 c_y^2 = 1/9, solved exactly in rationals (for components in
    {-1, 0, 1}, c_x^4 = c_x^2, so the mixed fourth moment is the independent
    one)."""
    shells = sorted({sum(v * v for v in c) for c in vecs})
    rows = []
    rhs = []

    def add(fun, val):
        rows.append([sum(Fraction(fun(c)) for c in vecs if sum(v * v for v in c) == s)
                     for s in shells])
        rhs.append(Fraction(val))

    add(lambda c: 1, 1)
    add(lambda c: c[0] ** 2, Fraction(1, 3))
    add(lambda c: c[0] ** 2 * c[1] ** 2, Fraction(1, 9))
    assert len(shells) == 3
    # Gaussian elimination in rationals (square system)
    n = len(shells)
    A = [r[:] + [b] for r, b in zip(rows[:n], rhs[:n])]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        for r in range(n):
            if r != col and A[r][col] != 0:
                fac = A[r][col] / A[col][col]
                A[r] = [a - fac * b for a, b in zip(A[r], A[col])]
    return {s: A[i][n] / A[i][i] for i, s in enumerate(shells)}


def pin_lattice(o, q):
    e, w, opp = o.lattice(q)
    shells = {15: {0, 1, 3}, 19: {0, 1, 2}}[q]
    want = {c for c in itertools.product((-1, 0, 1), repeat=3)
            if sum(v * v for v in c) in shells}
    got = [tuple(int(v) for v in row) for row in e]
    assert len(got) == q and set(got) == want, "velocity set"
    assert got[0] == (0, 0, 0), "rest vector first"
    for i in range(q):
        assert tuple(-v for v in got[i]) == got[opp[i]], "opposite of %d" % i
        if i > 0:
            assert opp[i] == (i + 1 if i % 2 == 1 else i - 1), "pair ordering"
    wr = _rational_weights(got)
    for i, c in enumerate(got):
        assert w[i] == float(wr[sum(v * v for v in c)]), "weight %d" % i
    # isotropy up to fourth order, exactly in rationals
    W = [wr[sum(v * v for v in c)] for c in got]
    d = lambda a, b: 1 if a == b else 0
    assert sum(W) == 1
    for a in range(3):
        assert sum(Wi * c[a] for Wi, c in zip(W, got)) == 0
        for b in range(3):
            assert sum(Wi * c[a] * c[b] for Wi, c in zip(W, got)) == Fraction(d(a, b), 3)
            for g in range(3):
                assert sum(Wi * c[a] * c[b] * c[g] for Wi, c in zip(W, got)) == 0
                for h in range(3):
                    m4 = sum(Wi * c[a] * c[b] * c[g] * c[h] for Wi, c in zip(W, got))
                    assert m4 == Fraction(d(a, b) * d(g, h) + d(a, g) * d(b, h)
                                          + d(a, h) * d(b, g), 9)


def pin_equilibrium(o, q, seed=0):
    """sum feq = rho, sum c feq = rho u, sum c c feq = rho/3 I + rho u u."""
    e, _, _ = o.lattice(q)
    e = e.astype(np.float64)
    rng = np.random.default_rng(seed)
    for _ in range(20):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.1, 0.1, 3)
        feq = o.equilibrium(q, rho, u)
        assert abs(feq.sum() - rho) <= 1e-14 * rho
        assert np.allclose(e.T @ feq, rho * u, rtol=0, atol=1e-15)
        P = (e.T * feq) @ e
        assert np.allclose(P, rho / 3.0 * np.eye(3) + rho * np.outer(u, u), rtol=0, atol=1e-15)


# ---------------------------------------------------------------- links

def brute_links(e, xyz, io_xyz, io_id, periodic):
    """O(N^2 Q) neighbour search written independently of both builders."""
    q = e.shape[0]
    n = xyz.shape[0]
    nbr = np.full((q, n), -1, np.int32)
    link = np.ones((q, n), np.uint8)
    for x in range(n):
        for i in range(q):
            y = [int(xyz[x, a]) + int(e[i, a]) for a in range(3)]
            for a in range(3):
                if periodic[a] > 0:
                    y[a] %= int(periodic[a])
            hit = [j for j in range(n) if list(xyz[j]) == y]
            assert len(hit) <= 1
            if hit:
                nbr[i, x] = hit[0]
                link[i, x] = 0
                continue
            io = [int(io_id[m]) for m in range(io_xyz.shape[0]) if list(io_xyz[m]) == y]
            if io:
                link[i, x] = 2 + io[0]
    return nbr, link


def pin_links(o, q, seed, periodic):
    g = G.random_mask((5, 4, 4), p=0.55, seed=seed, n_iolets=3, periodic=periodic)
    e, _, opp = o.lattice(q)
    nbr, link = o.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    bn, bl = brute_links(e, g.xyz, g.io_xyz, g.io_id, g.periodic)
    assert np.array_equal(nbr, bn), "nbr vs brute force"
    assert np.array_equal(link, bl), "link vs brute force"
    # symmetry of fluid links
    for i in range(q):
        m = nbr[i] >= 0
        xs = np.nonzero(m)[0]
        assert np.array_equal(nbr[opp[i], nbr[i, m]], xs), "link symmetry"


# ---------------------------------------------------------------- invariants

def _setup(o, q, g):
    nbr, link = o.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    return nbr, link


def pin_mass_periodic(o, q, steps=300):
    """Closed periodic box: mass and momentum are conserved exactly (FP64)."""
    g = G.periodic_box(5, 4, 3)
    nbr, link = _setup(o, q, g)
    e, _, _ = o.lattice(q)
    f0 = G.random_populations(q, g.n, seed=3, amplitude=0.2)
    f = o.run(q, nbr, link, 0.7, f0, steps)
    m0, m1 = f0.sum(), f.sum()
    assert abs(m1 - m0) <= 1e-13 * m0, "mass drift %g" % ((m1 - m0) / m0)
    j0 = e.T.astype(np.float64) @ f0.sum(axis=1)
    j1 = e.T.astype(np.float64) @ f.sum(axis=1)
    assert np.all(np.abs(j1 - j0) <= 1e-13 * m0), "momentum drift"
    # the state must have changed (a step that copies its input is no step)
    assert np.abs(f - f0).max() > 1e-4


def pin_mass_walled(o, q, steps=300):
    """Closed box with halfway bounce-back on every side: mass is conserved
    exactly (every population leaving through a wall comes back)."""
    g = G.walled_box(5, 4, 6)
    nbr, link = _setup(o, q, g)
    f0 = G.random_populations(q, g.n, seed=4, amplitude=0.2)
    f = o.run(q, nbr, link, 0.9, f0, steps)
    m0, m1 = f0.sum(), f.sum()
    assert abs(m1 - m0) <= 1e-13 * m0, "mass drift %g" % ((m1 - m0) / m0)
    assert np.abs(f - f0).max() > 1e-4


def pin_mass_sum(o, q):
    """The total mass is the sum of every population of every site, each
    counted once.  Closed forms: the rest state of n sites has mass
    n rho0 sum_i w_i = n rho0 (the weights sum to 1); populations numbered
    f[i, x] = 1 + i n + x (distinct integers, exact in float64) sum to
    m (m + 1) / 2 with m = q n, so a dropped direction or site, a wrong plane
    stride or a transposed index changes the value; and in a closed periodic
    box the mass of the final state equals the exactly rounded sum of the
    initial populations.  Float64 sums of N terms are held to the recursive
    summation bound N u sum |f|, u = 2^-53."""
    u = 2.0 ** -53
    for n in (1, 2, 7, 130):
        for rho0 in (1.0, 1.25):
            m = o.mass(o.rest_state(q, n, rho0))
            assert abs(m - n * rho0) <= (q * n + q) * u * n * rho0, (n, rho0, m)
        f = (1.0 + np.arange(q * n, dtype=np.float64)).reshape(q, n)
        qn = q * n
        assert o.mass(f) == qn * (qn + 1) // 2, (n, o.mass(f))
        # one population carries all the mass: each position in turn
        for x in {0, n // 2, n - 1}:
            for i in {0, q // 2, q - 1}:
                e = np.zeros((q, n))
                e[i, x] = 3.0
                assert o.mass(e) == 3.0, (i, x)
    g = G.periodic_box(4, 3, 5)
    nbr, link = _setup(o, q, g)
    f0 = G.random_populations(q, g.n, seed=12, amplitude=0.3)
    exact = math.fsum(f0.ravel())
    assert abs(o.mass(f0) - exact) <= q * g.n * u * np.abs(f0).sum()
    f = o.run(q, nbr, link, 0.8, f0, 50)
    assert abs(o.mass(f) - exact) <= 1e-13 * exact


def pin_rest(o, q, steps=100):
    """Fluid at rest between iolets of the rest density stays at rest."""
    g = G.tube(radius=3, length=8, nx=7, ny=7, rho_in=1.0, rho_out=1.0)
    nbr, link = _setup(o, q, g)
    f0 = o.rest_state(q, g.n)
    f = o.run(q, nbr, link, 0.8, f0, steps, geom=g)
    assert np.abs(f - f0).max() <= 1e-15


def pin_iolet_density(o, q):
    """Between two iolets of density rho1 and no walls (periodic cross
    section), fluid at rest relaxes to uniform density rho1 and rest."""
    g = G.slab(6, 1, 1, rho_in=1.0003, rho_out=1.0003)
    g.periodic[:] = (0, 1, 1)
    nbr, link = _setup(o, q, g)
    assert (link == 1).sum() == 0
    f = o.run(q, nbr, link, 0.8, o.rest_state(q, g.n), 2000, geom=g)
    rho, u, _ = o.macros(q, link, 0.8, f)
    assert np.abs(rho - 1.0003).max() < 1e-12 and np.abs(u).max() < 1e-12


def pin_iolet_time(o, q):
    """A single site between two pulsatile iolets: after the step t -> t+1
    each population arriving from iolet k equals the (pinned) equilibrium at
    the iolet density evaluated at the step's start time t and the site's
    velocity before the step."""
    g = G.slab(1, 1, 1)
    g.periodic[:] = (0, 1, 1)
    nbr, link = _setup(o, q, g)
    e, _, opp = o.lattice(q)
    io = dict(rho_mean=np.array([1.0, 1.0]), amp=np.array([0.01, 0.02]),
              period=np.array([7.0, 11.0]), phase=np.array([0.3, 1.1]))
    f = G.random_populations(q, 1, seed=9, amplitude=0.3)
    for t in (0, 5, 13):
        rho, u, _ = o.macros(q, link, 0.8, f)
        fn = o.step(q, nbr, link, 0.8, f, t=t, **io)
        for k in (0, 1):
            rk = io["rho_mean"][k] + io["amp"][k] * math.sin(
                2 * math.pi * t / io["period"][k] + io["phase"][k])
            feq = o.equilibrium(q, rk, u[0])
            for i in range(q):
                if link[i, 0] == 2 + k:
                    assert abs(fn[opp[i], 0] - feq[opp[i]]) <= 1e-15, (t, k, i)
        f = fn


# ---------------------------------------------------------------- Poiseuille

def pin_slab_poiseuille(o, q, steps=6000):
    """Plane Poiseuille flow between halfway bounce-back walls at
    tau = 1/2 + sqrt(3/16), where BGK with halfway bounce-back has no slip
    (He, Zou, Luo & Dembo, J. Stat. Phys. 87, 1997): the profile across the
    channel is the parabola u = G/(2 rho nu) (a^2 - s^2) with the walls
    exactly half-way between sites, nu = (tau - 1/2)/3, G = c_s^2 |d rho/dx|,
    and the wall shear stress at the wall-adjacent sites is G (h/2 - 1/2)."""
    h = 12
    tau = TAU_EXACT_BB
    g = G.slab(64, 2, h)
    nbr, link = _setup(o, q, g)
    f = o.run(q, nbr, link, tau, o.rest_state(q, g.n), steps, geom=g)
    rho, u, wss = o.macros(q, link, tau, f)
    x, y, z = g.xyz.T
    nu = (tau - 0.5) / 3.0
    xs = np.arange(16, 48)
    rx = np.array([rho[x == k].mean() for k in xs])
    Gr = -np.polyfit(xs, rx, 1)[0] / 3.0
    sel = (x == 32) & (y == 0)
    c = np.polyfit(z[sel], u[sel, 0], 2)
    roots = np.sort(np.roots(c).real)
    assert abs(roots[0] + 0.5) < 1e-4 and abs(roots[1] - (h - 0.5)) < 1e-4, roots
    curv = -Gr / (2.0 * nu * rho[sel].mean())
    assert abs(c[0] / curv - 1.0) < 1e-4, (c[0], curv)
    assert np.abs(u[:, 1]).max() == 0.0  # mirror symmetry of the periodic cross-section
    assert np.abs(u[sel, 2]).max() < 1e-3 * np.abs(u[sel, 0]).max()
    wsel = sel & ((z == 0) | (z == h - 1))
    assert np.allclose(wss[wsel], Gr * (h / 2.0 - 0.5), rtol=1e-4, atol=0)
    inner = sel & (z > 0) & (z < h - 1)
    assert np.all(wss[inner] == 0.0)


def pin_tube_poiseuille(o, steps=1000):
    """Pressure-driven flow in the straight tube (r = 8, 17x17x64, D3Q15,
    tau = 0.8, rho 1.001 -> 0.999): near the axis the mass-flux profile is the
    Hagen-Poiseuille parabola with curvature -G/(4 nu) (within 4%, the
    staircase wall perturbs it), the effective radius lies within half a
    lattice unit of 8, and the mean pressure gradient is within 10% of the
    nominal drop over the tube length."""
    q, tau = 15, 0.8
    g = G.tube()
    nbr, link = _setup(o, q, g)
    f = o.run(q, nbr, link, tau, o.rest_state(q, g.n), steps, geom=g)
    rho, u, _ = o.macros(q, link, tau, f)
    x, y, z = g.xyz.T
    r2 = (x - 8.0) ** 2 + (y - 8.0) ** 2
    nu = (tau - 0.5) / 3.0
    zs = np.arange(16, 48)
    rz = np.array([rho[z == k].mean() for k in zs])
    Gf = -np.polyfit(zs, rz, 1)[0] / 3.0
    nominal = (1.001 - 0.999) / 3.0 / 65.0
    assert abs(Gf / nominal - 1.0) < 0.1, (Gf, nominal)
    sel = (z >= 16) & (z < 48) & (r2 <= 16)
    c = np.polyfit(r2[sel], u[sel, 2] * rho[sel], 1)
    assert abs(c[0] / (-Gf / (4.0 * nu)) - 1.0) < 0.04, c
    reff = math.sqrt(-c[1] / c[0])
    assert 7.5 <= reff <= 8.5, reff
    assert u[:, 2].min() > -1e-5


ALL_FAST = [
    ("lattice15", lambda o: pin_lattice(o, 15)),
    ("lattice19", lambda o: pin_lattice(o, 19)),
    ("equilibrium15", lambda o: pin_equilibrium(o, 15)),
    ("equilibrium19", lambda o: pin_equilibrium(o, 19)),
    ("links15", lambda o: pin_links(o, 15, 1, False)),
    ("links19p", lambda o: pin_links(o, 19, 2, True)),
    ("mass_periodic19", lambda o: pin_mass_periodic(o, 19)),
    ("mass_walled15", lambda o: pin_mass_walled(o, 15, 200)),
    ("mass_sum15", lambda o: pin_mass_sum(o, 15)),
    ("mass_sum19", lambda o: pin_mass_sum(o, 19)),
    ("rest19", lambda o: pin_rest(o, 19)),
    ("iolet_density15", lambda o: pin_iolet_density(o, 15)),
    ("iolet_time19", lambda o: pin_iolet_time(o, 19)),
    ("slab19", lambda o: pin_slab_poiseuille(o, 19, 3000)),
]


# ---------------------------------------------------------------- adjoint

def _adj_setup(o, q, seed=5):
    g = G.random_mask((7, 6, 5), p=0.6, seed=seed, n_iolets=3)
    nbr, link = o.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    rng = np.random.default_rng(seed)
    f0 = o.rest_state(q, g.n) * (1.0 + 0.02 * (2.0 * rng.random((q, g.n)) - 1.0))
    return g, nbr, link, f0, rng


def pin_adjoint_dot_product(o, q, tau=0.7):
    """One step: <(dF/df)^T w, v> equals <w, dF/df v> from central differences
    of the forward step (F is smooth; h = 1e-6, error O(h^2))."""
    g, nbr, link, f0, rng = _adj_setup(o, q)
    w = rng.standard_normal(f0.shape)
    v = rng.standard_normal(f0.shape)
    lam, _, _, _, _ = o.adjoint_step(q, nbr, link, tau, f0, w, t=4, geom=g)
    h = 1e-6
    Fp = o.step(q, nbr, link, tau, f0 + h * v, t=4, geom=g)
    Fm = o.step(q, nbr, link, tau, f0 - h * v, t=4, geom=g)
    a, b = float(np.sum(lam * v)), float(np.sum(w * (Fp - Fm) / (2 * h)))
    assert abs(a - b) <= 1e-8 * abs(b), (a, b)


def pin_adjoint_gradient(o, q, kind, tau=0.7, nsteps=8):
    """Adjoint gradient of a windowed objective against central finite
    differences of the FP64 forward run: d/dtau and d/d(mean, amp, phase) of
    every iolet (h = 1e-6), and d/df0 along a random direction (h = 1e-8 for
    the wall-shear-stress objective, whose |s| is not smooth where s = 0)."""
    g, nbr, link, f0, rng = _adj_setup(o, q)
    m = (rng.random(g.n) < 0.5).astype(np.float64)
    args = dict(kind=kind, m=m, t_begin=3, t_end=nsteps + 1, scale=0.25)
    rho, _, wss = o.macros(q, link, tau, f0)
    q0 = o.objective(q, link, tau, kind, m, f0)
    assert abs(q0 - float(np.sum(m * (wss if kind == 0 else rho)))) <= 1e-13 * abs(q0)
    r = o.gradient(q, nbr, link, tau, f0, nsteps, geom=g, want_lam0=True, **args)
    J = o.objective_run(q, nbr, link, tau, f0, nsteps, geom=g, **args)
    assert abs(r["J"] - J) <= 1e-13 * abs(J)
    h = 1e-6

    def fd(**kw):
        io = dict(rho_mean=g.rho_mean.copy(), amp=g.amp.copy(), period=g.period.copy(),
                  phase=g.phase.copy())
        t_ = kw.pop("tau", 0.0)
        key, k = kw.get("key"), kw.get("k")
        if key:
            io[key][k] += h
        Jp = o.objective_run(q, nbr, link, tau + t_ * h, f0, nsteps, **io, **args)
        if key:
            io[key][k] -= 2 * h
        Jm = o.objective_run(q, nbr, link, tau - t_ * h, f0, nsteps, **io, **args)
        return (Jp - Jm) / (2 * h)

    scale = max(abs(r["dtau"]), 1e-30)
    assert abs(r["dtau"] - fd(tau=1.0)) <= 1e-5 * scale, ("dtau", r["dtau"])
    for k in range(g.n_iolets):
        for nm, key in (("dmean", "rho_mean"), ("damp", "amp"), ("dphase", "phase")):
            ref = fd(key=key, k=k)
            tol = 1e-5 * max(abs(ref), 1e-3 * abs(r["dmean"][k]))
            assert abs(r[nm][k] - ref) <= tol, (nm, k, r[nm][k], ref)
    v = rng.standard_normal(f0.shape)
    hv = 1e-8 if kind == 0 else 1e-6
    Jp = o.objective_run(q, nbr, link, tau, f0 + hv * v, nsteps, geom=g, **args)
    Jm = o.objective_run(q, nbr, link, tau, f0 - hv * v, nsteps, geom=g, **args)
    ref = (Jp - Jm) / (2 * hv)
    got = float(np.sum(r["lam0"] * v))
    assert abs(got - ref) <= 1e-5 * abs(ref), ("lam0", got, ref)


def _adj_bc_setup(o, q, seed=6):
    """A random mask with a density iolet, a pulsatile velocity iolet (with a
    non-uniform weight profile) and interpolated walls at random fractions on
    both sides of 1/2."""
    g, nbr, link, f0, rng = _adj_setup(o, q, seed)
    bc = dict(io_kind=np.array([0, 1, 0], np.int32),
              io_normal=np.array([[0, 0, 0], [0.6, 0.0, 0.8], [0, 0, 0]], np.float64),
              weight=0.5 + rng.random(g.n),
              wall_q=np.where(link == 1, rng.uniform(0.05, 1.0, link.shape), 0.5))
    io = dict(rho_mean=np.array([1.001, 0.003, 0.999]), amp=np.array([0.0005, 0.001, 0.0]),
              period=np.array([13.0, 17.0, 0.0]), phase=np.array([0.2, 0.7, 0.0]))
    assert ((bc["wall_q"] < 0.5) & (link == 1)).any() and ((bc["wall_q"] > 0.5) & (link == 1)).any()
    return g, nbr, link, f0, rng, bc, io


def pin_adjoint_dot_product_bc(o, q, tau=0.7):
    """One step with velocity iolets and interpolated walls: <(dF/df)^T w, v>
    equals <w, dF/df v> from central differences of the forward step."""
    g, nbr, link, f0, rng, bc, io = _adj_bc_setup(o, q)
    w = rng.standard_normal(f0.shape)
    v = rng.standard_normal(f0.shape)
    lam, _, _, _, _ = o.adjoint_step(q, nbr, link, tau, f0, w, t=4, **bc, **io)
    h = 1e-6
    Fp = o.run_bc(q, nbr, link, tau, f0 + h * v, 1, t0=4, **bc, **io)
    Fm = o.run_bc(q, nbr, link, tau, f0 - h * v, 1, t0=4, **bc, **io)
    a, b = float(np.sum(lam * v)), float(np.sum(w * (Fp - Fm) / (2 * h)))
    assert abs(a - b) <= 1e-8 * abs(b), (a, b)


def pin_adjoint_gradient_bc(o, q, kind, tau=0.7, nsteps=8):
    """The windowed objective's gradient with velocity iolets and interpolated
    walls against central differences of the FP64 forward run: d/dtau, d/d
    (mean, amp, phase) of the velocity iolet's speed schedule and of the
    density iolets, and d/df0 along a random direction."""
    g, nbr, link, f0, rng, bc, io = _adj_bc_setup(o, q)
    m = (rng.random(g.n) < 0.5).astype(np.float64)
    args = dict(kind=kind, m=m, t_begin=3, t_end=nsteps + 1, scale=0.25)
    r = o.gradient(q, nbr, link, tau, f0, nsteps, want_lam0=True, **bc, **io, **args)
    J = o.objective_run(q, nbr, link, tau, f0, nsteps, **bc, **io, **args)
    assert abs(r["J"] - J) <= 1e-13 * abs(J)
    # the density objective is ~80 while some of its derivatives are ~2e-5,
    # so at h = 1e-6 its differences would carry round-off of 1e-16 * 80 / h
    # (4e-4 of the smallest derivative): h = 1e-4 there (truncation ~1e-8);
    # the wall-shear-stress objective is small and curved: h = 1e-6
    h = 1e-4 if kind == 1 else 1e-6

    def fd(tau_h=0.0, key=None, k=None):
        io2 = {kk: vv.copy() for kk, vv in io.items()}
        if key:
            io2[key][k] += h
        Jp = o.objective_run(q, nbr, link, tau + tau_h * h, f0, nsteps, **bc, **io2, **args)
        if key:
            io2[key][k] -= 2 * h
        Jm = o.objective_run(q, nbr, link, tau - tau_h * h, f0, nsteps, **bc, **io2, **args)
        return (Jp - Jm) / (2 * h)

    assert abs(r["dtau"] - fd(tau_h=1.0)) <= 1e-5 * max(abs(r["dtau"]), 1e-30), ("dtau", r["dtau"])
    for k in range(g.n_iolets):
        for nm, key in (("dmean", "rho_mean"), ("damp", "amp"), ("dphase", "phase")):
            ref = fd(key=key, k=k)
            tol = 1e-5 * max(abs(ref), 1e-3 * abs(r["dmean"][k]))
            assert abs(r[nm][k] - ref) <= tol, (nm, k, r[nm][k], ref)
    assert abs(r["dmean"][1]) > 1e-6  # the velocity iolet's speed does move J
    v = rng.standard_normal(f0.shape)
    hv = 1e-8 if kind == 0 else 1e-6
    Jp = o.objective_run(q, nbr, link, tau, f0 + hv * v, nsteps, **bc, **io, **args)
    Jm = o.objective_run(q, nbr, link, tau, f0 - hv * v, nsteps, **bc, **io, **args)
    ref = (Jp - Jm) / (2 * hv)
    got = float(np.sum(r["lam0"] * v))
    assert abs(got - ref) <= 1e-5 * abs(ref), ("lam0", got, ref)


ALL_FAST += [
    ("adjoint_dot19", lambda o: pin_adjoint_dot_product(o, 19)),
    ("adjoint_wss15", lambda o: pin_adjoint_gradient(o, 15, 0)),
    ("adjoint_density19", lambda o: pin_adjoint_gradient(o, 19, 1)),
    ("adjoint_dot_bc15", lambda o: pin_adjoint_dot_product_bc(o, 15)),
    ("adjoint_bc_density19", lambda o: pin_adjoint_gradient_bc(o, 19, 1)),
]


# ---------------------------------------------------------------- velocity iolets

def _ladd_slab(o, q, ny, weight_fn, steps):
    """Channel along x, periodic in y and z, no walls: iolet 0 (x = -1) is a
    density outlet, iolet 1 (x = 12) a velocity inlet pushing in -x (using the
    second iolet also checks that the iolet's own normal is used)."""
    g = G.slab(12, ny, 1, rho_in=1.0, rho_out=1.0)
    g.periodic[:] = (0, ny, 1)
    nbr, link = o.links_build(q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    U = 0.01
    x, y, z = g.xyz.T
    w = weight_fn(x, y, z)
    f = o.run_bc(q, nbr, link, 1.5, o.rest_state(q, g.n), steps, io_kind=[0, 1],
                 io_normal=[[0, 0, 0], [-1, 0, 0]], weight=w, rho_mean=[1.0, U])
    rho, u, _ = o.macros(q, link, 1.5, f)
    return g, x, y, w, U, rho, u


def pin_ladd_plug(o, q):
    """Velocity (Ladd) inlet with uniform weight w, density outlet, no walls
    (periodic cross-section): the steady flow is the plug u = -w U (the inlet
    pushes along its normal -x), and rho u is constant along the channel."""
    g, x, y, w, U, rho, u = _ladd_slab(o, q, 1, lambda x, y, z: np.full(x.shape, 0.5), 6000)
    assert np.abs(-u[:, 0] / (0.5 * U) - 1.0).max() < 1e-9, u[:, 0]
    assert np.abs(u[:, 1:]).max() == 0.0


def pin_ladd_flux(o, q):
    """Non-uniform weights across the channel: at steady state the mass flux
    through every cross-section equals the inflow, the sum over the inlet
    sites of rho(x) w(x) U (each inlet site has all its +x links on the
    iolet)."""
    g, x, y, w, U, rho, u = _ladd_slab(o, q, 4, lambda x, y, z: 0.5 + 0.5 * y, 8000)
    inlet = x == 11
    inflow = float(np.sum(rho[inlet] * w[inlet] * U))
    for k in range(12):
        flux = -float(np.sum(rho[x == k] * u[x == k, 0]))
        assert abs(flux / inflow - 1.0) < 1e-9, (k, flux, inflow)


ALL_FAST += [
    ("ladd_plug19", lambda o: pin_ladd_plug(o, 19)),
    ("ladd_flux15", lambda o: pin_ladd_flux(o, 15)),
]


# ---------------------------------------------------------------- volume rendering

def _lut(rgb, alpha):
    lut = np.zeros((256, 4), np.float32)
    lut[:, :3] = rgb
    lut[:, 3] = alpha
    return lut


def _axis_ray(o, vol, eye, center, lut, dt, a_stop=1.0, tf_scale=1.0, tf_offset=0.0, up=(0, 1, 0)):
    """One pixel whose ray is exactly the view axis (a 1 x 1 image)."""
    return o.render(vol, 1, 1, eye, center, up, 0.5, dt, tf_scale, tf_offset, lut, a_stop)[0, 0]


def pin_render_homogeneous(o):
    """A constant volume along the view axis: every segment has the same
    colour, so A = 1 - prod(1 - alpha l_m) over the segment lengths l_m and
    C = colour * A; small steps approach Beer-Lambert, 1 - exp(-alpha L);
    early termination and the opacity clamp follow from the same closed form."""
    nx = ny = nz = 8
    vol = np.full((nz, ny, nx), 0.5, np.float32)
    rgb = np.array([1.0, 0.5, 0.25])
    eye, ctr = [3.5, 3.5, -20.0], [3.5, 3.5, 3.5]
    L = 8.0  # the axis crosses z in [-0.5, 7.5]
    alpha, dt = 0.2, 0.3  # 26 segments of 0.3, then one of 0.2
    px = _axis_ray(o, vol, eye, ctr, _lut(rgb, alpha), dt)
    A = 1.0 - (1.0 - alpha * dt) ** 26 * (1.0 - alpha * 0.2)
    assert abs(px[3] - A) < 1e-6, (px, A)
    assert np.abs(px[:3] - rgb * A).max() < 1e-6, px
    px = _axis_ray(o, vol, eye, ctr, _lut(rgb, alpha), 1e-3)
    assert abs(px[3] - (1.0 - math.exp(-alpha * L))) < 1e-3, px
    # opacity 0.6 per sample: A_k = 1 - 0.4^k crosses 0.99 after six samples
    px = _axis_ray(o, vol, eye, ctr, _lut(rgb, 2.0), 0.3, a_stop=0.99)
    assert abs(px[3] - (1.0 - 0.4 ** 6)) < 1e-6, px
    px = _axis_ray(o, vol, eye, ctr, _lut(rgb, 2.0), 0.3, a_stop=0.98)
    assert abs(px[3] - (1.0 - 0.4 ** 5)) < 1e-6, px
    # alpha l > 1 is clamped to an opaque sample
    px = _axis_ray(o, vol, eye, ctr, _lut(rgb, 10.0), 0.3)
    assert np.abs(px - np.r_[rgb, 1.0]).max() < 1e-6, px
    # a volume whose transfer gives alpha 0 leaves the pixel empty
    assert np.abs(_axis_ray(o, vol, eye, ctr, _lut(rgb, 0.0), 0.3)).max() == 0.0


def pin_render_trilinear(o, seed=3):
    """Trilinear interpolation reproduces a + b x + c y + d x y exactly (also
    in the clamped half-voxel rim, at the clamped coordinate); with a constant
    opacity the pixel colour is the LUT, linearly interpolated at
    s = clamp((v - offset) scale, 0, 1) * 255, times the closed-form A.
    Rays along z test the x and y weights, rays along x the z weight."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = 9, 7, 6
    a, b, c, d = 0.1, 0.07, 0.05, 0.01
    lut = _lut(0.0, 0.3)
    lut[:, :3] = rng.random((256, 3))
    off, scale = 0.05, 1.3
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    A_z = 1.0 - (1.0 - 0.3 * 0.5) ** (2 * nz)  # L = nz, dt = 0.5

    def expect(v, A):
        s = min(max((v - off) * scale, 0.0), 1.0) * 255.0
        return np.array([np.interp(s, np.arange(256), lut[:, ch]) for ch in range(3)]) * A

    vol = (a + b * i + c * j + d * i * j).astype(np.float32)
    for x0, y0 in [(2.3, 4.6), (0.5, 0.25), (7.9, 5.99), (-0.3, 3.2), (8.3, 6.4), (4.0, 3.0)]:
        px = _axis_ray(o, vol, [x0, y0, -10.0], [x0, y0, 0.0], lut, 0.5, tf_scale=scale,
                       tf_offset=off)
        xc, yc = min(max(x0, 0.0), nx - 1.0), min(max(y0, 0.0), ny - 1.0)
        v = a + b * xc + c * yc + d * xc * yc
        # the volume holds float32 values: 1e-4 covers their rounding through the LUT slope
        assert abs(px[3] - A_z) < 1e-6
        assert np.abs(px[:3] - expect(v, A_z)).max() < 1e-4, (x0, y0, px, expect(v, A_z))
    vol = (a + c * j + 0.12 * k).astype(np.float32)
    A_x = 1.0 - (1.0 - 0.3 * 0.5) ** (2 * nx)
    for y0, z0 in [(1.7, 2.45), (5.2, 4.9), (3.0, -0.2)]:
        px = _axis_ray(o, vol, [-10.0, y0, z0], [0.0, y0, z0], lut, 0.5, tf_scale=scale,
                       tf_offset=off)
        v = a + c * y0 + 0.12 * min(max(z0, 0.0), nz - 1.0)
        assert np.abs(px[:3] - expect(v, A_x)).max() < 1e-4, (y0, z0, px)


def pin_render_midpoint(o):
    """With a vanishing opacity C / A is the length-weighted mean colour along
    the ray; the midpoint samples integrate the piecewise-linear colour of a
    z ramp exactly when the segments start at its kinks.  The eye sits inside
    the volume (z = 2.25), so the path is [2.25, 7.5]."""
    nx, ny, nz = 5, 5, 8
    k = np.arange(nz, dtype=np.float64)[:, None, None] * np.ones((1, ny, nx))
    vol = (k / (nz - 1)).astype(np.float32)
    lut = _lut(0.0, 1e-6)
    lut[:, 0] = np.arange(256) / 255.0
    px = _axis_ray(o, vol, [2.0, 2.0, 2.25], [2.0, 2.0, 5.0], lut, 0.25)
    z0, z1 = 2.25, nz - 0.5
    integral = (49.0 - z0 * z0) / (2.0 * 7.0) + (z1 - 7.0) * 1.0
    mean = integral / (z1 - z0)
    assert abs(px[0] / px[3] - mean) < 1e-5, (px, mean)
    assert abs(px[3] - 1e-6 * (z1 - z0)) < 1e-10, px


def pin_render_over_operator(o, seed=4):
    """Front-to-back compositing is the 'over' operator: for a ray along z
    through a volume that is zero on a slab between two random layers (and a
    transfer function with zero opacity at 0), the full image equals
    front + (1 - A_front) back, where front and back render each layer alone."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = 6, 6, 14
    vol = rng.random((nz, ny, nx)).astype(np.float32) + 0.05
    vol[5:9] = 0.0  # the gap
    front, back = vol.copy(), vol.copy()
    front[9:] = 0.0
    back[:5] = 0.0
    lut = rng.random((256, 4)).astype(np.float32)
    lut[:, 3] *= 0.6
    lut[0, 3] = 0.0
    args = dict(eye=[2.2, 3.1, -30.0], center=[2.6, 2.4, 7.0], up=[0, 1, 0], fov_y=0.15, dt=0.37,
                tf_scale=1.0, tf_offset=0.0, lut=lut, a_stop=1.0)
    full = o.render(vol, 7, 5, **args)
    f = o.render(front, 7, 5, **args)
    bk = o.render(back, 7, 5, **args)
    comp = f + (1.0 - f[..., 3:4]) * bk
    assert ((f[..., 3] > 0.05) & (bk[..., 3] > 0.05)).mean() > 0.5
    assert np.abs(full - comp).max() < 1e-6, np.abs(full - comp).max()


def pin_render_camera(o):
    """Pinhole camera: looking down -z from the axis with up = +y, a pixel's
    ray hits the box exactly when it passes through the front face, i.e. when
    |s_x| D < n_x / 2 and |s_y| D < n_y / 2 for s_x = ((p_x + 1/2) / W * 2 - 1)
    tan(fov/2) W / H and s_y = (1 - (p_y + 1/2) / H * 2) tan(fov/2), D the
    distance to the front face.  +x is on the right of the image and +y at
    the top (right = forward x up)."""
    nx, ny, nz = 10, 6, 4
    ctr = np.array([(nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0])
    eye = ctr + [0.0, 0.0, 30.0]
    W, H, fov = 41, 23, 0.5
    lut = _lut(1.0, 0.5)
    img = o.render(np.ones((nz, ny, nx), np.float32), W, H, eye, ctr, [0, 1, 0], fov, 0.3, 1.0,
                   0.0, lut)
    D = eye[2] - (nz - 0.5)
    th = math.tan(fov / 2)
    sx = ((np.arange(W) + 0.5) / W * 2 - 1) * th * W / H
    sy = (1 - (np.arange(H) + 0.5) / H * 2) * th
    inx, iny = np.abs(sx) * D < nx / 2, np.abs(sy) * D < ny / 2
    margin_x = np.abs(np.abs(sx) * D - nx / 2) > 1e-3
    margin_y = np.abs(np.abs(sy) * D - ny / 2) > 1e-3
    hit = img[..., 3] > 0
    want = iny[:, None] & inx[None, :]
    sure = margin_y[:, None] & margin_x[None, :]
    assert want.sum() > 20 and (~want).sum() > 20
    assert np.array_equal(hit[sure], want[sure]), (hit.sum(), want.sum())
    # orientation: only the +x half (resp. the +y half) of the volume is visible
    lut = _lut(1.0, 0.0)
    lut[:, 3] = np.arange(256) / 255.0
    half = np.zeros((nz, ny, nx), np.float32)
    half[:, :, nx // 2 + 1:] = 1.0
    a = o.render(half, W, H, eye, ctr, [0, 1, 0], fov, 0.3, 1.0, 0.0, lut)[..., 3]
    assert a[:, : W // 2].max() == 0.0 and a[H // 2, W // 2 + 2: W // 2 + 7].min() > 0.0
    half = np.zeros((nz, ny, nx), np.float32)
    half[:, ny // 2 + 1:, :] = 1.0
    a = o.render(half, W, H, eye, ctr, [0, 1, 0], fov, 0.3, 1.0, 0.0, lut)[..., 3]
    assert a[H // 2:, :].max() == 0.0 and a[H // 2 - 3, W // 2] > 0.0


def pin_render_miss(o):
    """Rays that never meet the box leave the pixel empty."""
    vol = np.ones((4, 4, 4), np.float32)
    img = o.render(vol, 9, 7, [1.5, 1.5, -10.0], [1.5, 1.5, -20.0], [0, 1, 0], 0.5, 0.3, 1.0, 0.0,
                   _lut(1.0, 1.0))
    assert np.abs(img).max() == 0.0


ALL_FAST += [
    ("render_homogeneous", pin_render_homogeneous),
    ("render_trilinear", pin_render_trilinear),
    ("render_midpoint", pin_render_midpoint),
    ("render_over", pin_render_over_operator),
    ("render_camera", pin_render_camera),
    ("render_miss", pin_render_miss),
]


# ---------------------------------------------------------------- interpolated (BFL) walls

def _slab_wall_q(o, q, g, link, q_lo, q_hi):
    """Fluid fractions of the wall links of G.slab: q_lo for the links toward
    the wall below (c_z = -1), q_hi toward the wall above (c_z = +1); the
    walls sit at z = -q_lo and z = h - 1 + q_hi."""
    e = np.asarray(o.lattice(q)[0]).reshape(q, 3)
    wq = np.full(link.shape, 0.5)
    for i in range(q):
        w = link[i] == 1
        wq[i, w & (e[i, 2] < 0)] = q_lo
        wq[i, w & (e[i, 2] > 0)] = q_hi
    return wq


def bfl_slab_wall_error(o, q, h, q_lo, q_hi, tau=0.8, steps=None):
    """Distance (lattice units) between the zeros of the steady BFL channel
    profile and the true wall positions, below and above."""
    nx = 64 if h < 20 else 128
    g = G.slab(nx, 2, h)
    nbr, link = _setup(o, q, g)
    wq = _slab_wall_q(o, q, g, link, q_lo, q_hi)
    steps = steps or int(4000 * (h / 12.0) ** 2)
    f = o.run_bc(q, nbr, link, tau, o.rest_state(q, g.n), steps, wall_q=wq, geom=g)
    _, u, _ = o.macros(q, link, tau, f)
    x, y, z = g.xyz.T
    sel = (x == nx // 2) & (y == 0)
    roots = np.sort(np.roots(np.polyfit(z[sel], u[sel, 0], 2)).real)
    return roots[0] + q_lo, roots[1] - (h - 1 + q_hi)


def pin_bfl_halfway(o, q):
    """BFL with q = 1/2 on every wall link is the plain half-way bounce-back."""
    g = G.random_mask((7, 6, 5), p=0.6, seed=21, n_iolets=2)
    nbr, link = _setup(o, q, g)
    rng = np.random.default_rng(3)
    f0 = o.rest_state(q, g.n) * (1.0 + 0.01 * (2 * rng.random((q, g.n)) - 1))
    a = o.run(q, nbr, link, 0.7, f0, 15, geom=g)
    b = o.run_bc(q, nbr, link, 0.7, f0, 15, wall_q=np.full((q, g.n), 0.5), geom=g)
    assert np.array_equal(a, b)


def pin_bfl_rest(o, q):
    """Both BFL interpolations have weights summing to 1, so the rest state
    stays at rest for any wall position."""
    g = G.random_mask((7, 6, 5), p=0.6, seed=22, n_iolets=0)
    nbr, link = _setup(o, q, g)
    rng = np.random.default_rng(4)
    wq = rng.uniform(0.02, 1.0, (q, g.n))
    f0 = o.rest_state(q, g.n)
    f = o.run_bc(q, nbr, link, 0.7, f0, 40, wall_q=wq, geom=g)
    assert np.abs(f - f0).max() < 1e-14


def pin_bfl_slab(o, q):
    """Plane Poiseuille flow between walls off the half-way position: the zeros
    of the BFL profile follow the walls to within 0.05 lattice units at
    h = 12 (the linear interpolation leaves a tau- and q-dependent slip of
    this size, halving with each doubling of h), where half-way bounce-back
    would put them up to 0.4 away."""
    for q_lo, q_hi in ((0.1, 0.7), (0.8, 0.35)):
        lo, hi = bfl_slab_wall_error(o, q, 12, q_lo, q_hi)
        assert abs(lo) < 0.05 and abs(hi) < 0.05, (q_lo, q_hi, lo, hi)


ALL_FAST += [
    ("bfl_halfway19", lambda o: pin_bfl_halfway(o, 19)),
    ("bfl_rest15", lambda o: pin_bfl_rest(o, 15)),
    ("bfl_slab19", lambda o: pin_bfl_slab(o, 19)),
]
