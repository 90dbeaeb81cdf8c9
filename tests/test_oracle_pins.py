"""The FP64 oracle against closed forms, invariants and brute force (CPU)."""
import os

import numpy as np
import pytest

import oracle
import pins


@pytest.fixture(scope="module")
def o():
    return oracle.default()


@pytest.mark.parametrize("q", [15, 19])
def test_lattice_isotropy(o, q):
    pins.pin_lattice(o, q)


@pytest.mark.parametrize("q", [15, 19])
def test_equilibrium_moments(o, q):
    pins.pin_equilibrium(o, q)


@pytest.mark.parametrize("q,seed,periodic", [(15, 1, False), (15, 5, True),
                                             (19, 2, True), (19, 7, False)])
def test_links_brute_force(o, q, seed, periodic):
    pins.pin_links(o, q, seed, periodic)


@pytest.mark.parametrize("q", [15, 19])
def test_mass_momentum_periodic(o, q):
    pins.pin_mass_periodic(o, q, steps=1000)


@pytest.mark.parametrize("q", [15, 19])
def test_mass_walled(o, q):
    pins.pin_mass_walled(o, q, steps=1000)


@pytest.mark.parametrize("q", [15, 19])
def test_mass_sum(o, q):
    pins.pin_mass_sum(o, q)


@pytest.mark.parametrize("q", [15, 19])
def test_rest_state(o, q):
    pins.pin_rest(o, q)


@pytest.mark.parametrize("q", [15, 19])
def test_iolet_density(o, q):
    pins.pin_iolet_density(o, q)


@pytest.mark.parametrize("q", [15, 19])
def test_iolet_time_index(o, q):
    pins.pin_iolet_time(o, q)


@pytest.mark.parametrize("q", [15, 19])
def test_slab_poiseuille(o, q):
    pins.pin_slab_poiseuille(o, q)


def test_tube_poiseuille(o):
    pins.pin_tube_poiseuille(o)


def test_links_duplicate_rejected(o):
    with pytest.raises(ValueError):
        o.links_build(15, np.array([[0, 0, 0], [0, 0, 0]]))


def test_empty_geometry(o):
    nbr, link = o.links_build(19, np.zeros((0, 3), np.int32))
    assert nbr.shape == (19, 0) and link.shape == (19, 0)
    f = o.run(19, nbr, link, 0.8, np.zeros((19, 0)), 3)
    assert f.shape == (19, 0)
    assert o.mass(f) == 0.0


@pytest.mark.parametrize("q", [15, 19])
def test_adjoint_dot_product(o, q):
    pins.pin_adjoint_dot_product(o, q)


@pytest.mark.parametrize("q", [15, 19])
@pytest.mark.parametrize("kind", [0, 1])
def test_adjoint_gradient_vs_central_differences(o, q, kind):
    pins.pin_adjoint_gradient(o, q, kind)


@pytest.mark.parametrize("q", [15, 19])
def test_velocity_iolet_plug_flow(o, q):
    pins.pin_ladd_plug(o, q)


@pytest.mark.parametrize("q", [15, 19])
def test_velocity_iolet_flux_balance(o, q):
    pins.pin_ladd_flux(o, q)


@pytest.mark.parametrize("name", ["homogeneous", "trilinear", "midpoint", "over", "camera", "miss"])
def test_render(o, name):
    dict(pins.ALL_FAST)["render_" + name](o)


@pytest.mark.parametrize("q", [15, 19])
def test_bfl_halfway_and_rest(o, q):
    pins.pin_bfl_halfway(o, q)
    pins.pin_bfl_rest(o, q)


@pytest.mark.parametrize("q", [15, 19])
def test_bfl_slab(o, q):
    pins.pin_bfl_slab(o, q)


def test_bfl_second_order():
    """Doubling the channel width (at fixed tau) halves the wall-position
    error in lattice units: BFL is second-order accurate."""
    o = oracle.default()
    e12 = pins.bfl_slab_wall_error(o, 19, 12, 0.1, 0.7)
    e24 = pins.bfl_slab_wall_error(o, 19, 24, 0.1, 0.7)
    for a, b in zip(e12, e24):
        assert 1.7 < a / b < 2.4, (e12, e24)


@pytest.mark.parametrize("q", [15, 19])
def test_adjoint_dot_product_with_velocity_iolets_and_bfl(o, q):
    pins.pin_adjoint_dot_product_bc(o, q)


@pytest.mark.parametrize("q,kind", [(15, 0), (19, 1), (19, 0), (15, 1)])
def test_adjoint_gradient_with_velocity_iolets_and_bfl(o, q, kind):
    pins.pin_adjoint_gradient_bc(o, q, kind)
