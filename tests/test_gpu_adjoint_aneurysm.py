"""Wall-shear-stress gradients on the saccular aneurysm (641,833 sites, D3Q15,
tau = 0.55, pulsatile inlet 1 + 0.001 sin(2 pi t / 4000), outlet 1.0,
objective = sphere-wall WSS averaged over a window of late states,
gradient with respect to tau and the inlet amplitude and phase, 64 snapshots).

1. 400 steps (window: the last 200 states) against FP64 oracle central
   differences with h = 1e-6 on every parameter.
2. The full 4000 steps (window: the last 2000 states) against central
   differences of the GPU forward solver itself (a property that holds at
   any size: the adjoint is the derivative of the implemented step).
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

Q, TAU, NSNAP = 15, 0.55, 64


@pytest.fixture(scope="module")
def aneurysm():
    g = G.aneurysm()
    nbr, link = lbm.links_build(Q, g.xyz, g.io_xyz, g.io_id, g.periodic)
    return g, nbr, link


def lattice(g, nbr, link):
    return lbm.Lattice(Q, g.xyz, nbr, link, TAU, rho_mean=g.rho_mean, amp=g.amp, period=g.period,
                       phase=g.phase)


def test_aneurysm_wss_gradient_vs_oracle_central_differences(aneurysm):
    g, nbr, link = aneurysm
    nsteps, tb, te, scale = 400, 201, 401, 1.0 / 200
    L = lattice(g, nbr, link)
    got = L.objective_grad(lbm.OBJ_WSS, g.site_weight, nsteps, tb, te, scale=scale, n_snap=NSNAP)
    fw, ad = L.adjoint_counts()
    assert fw == lbm.revolve_steps(nsteps, NSNAP) and ad == nsteps
    o = oracle.default()
    f0 = o.rest_state(Q, g.n)
    h = 1e-6

    def J(tau=TAU, amp=None, phase=None):
        a = g.amp.copy() if amp is None else amp
        p = g.phase.copy() if phase is None else phase
        return o.objective_run(Q, nbr, link, tau, f0, nsteps, lbm.OBJ_WSS, g.site_weight, tb, te,
                               scale=scale, rho_mean=g.rho_mean, amp=a, period=g.period, phase=p)

    J0 = J()
    d_tau = (J(tau=TAU + h) - J(tau=TAU - h)) / (2 * h)
    ap, am = g.amp.copy(), g.amp.copy()
    ap[0] += h
    am[0] -= h
    d_amp = (J(amp=ap) - J(amp=am)) / (2 * h)
    pp, pm = g.phase.copy(), g.phase.copy()
    pp[0] += h
    pm[0] -= h
    d_phase = (J(phase=pp) - J(phase=pm)) / (2 * h)
    errs = dict(J=abs(got["J"] / J0 - 1), dtau=abs(got["dtau"] / d_tau - 1),
                damp=abs(got["damp"][0] / d_amp - 1), dphase=abs(got["dphase"][0] / d_phase - 1))
    print("aneurysm 400 steps: J", got["J"], J0, "dtau", got["dtau"], d_tau, "damp", got["damp"][0],
          d_amp, "dphase", got["dphase"][0], d_phase, errs)
    for k, v in errs.items():
        assert v <= 2e-3, (k, v)


def test_aneurysm_full_run_gradient_vs_gpu_central_differences(aneurysm):
    g, nbr, link = aneurysm
    nsteps, tb, te, scale = 4000, 2001, 4001, 1.0 / 2000
    L = lattice(g, nbr, link)
    state0 = L.get_state()
    got = L.objective_grad(lbm.OBJ_WSS, g.site_weight, nsteps, tb, te, scale=scale, n_snap=NSNAP)
    fw, ad = L.adjoint_counts()
    assert fw == lbm.revolve_steps(nsteps, NSNAP) == 9790

    def J(tau=TAU, amp=None, phase=None):
        L.set_state(state0)
        L.set_time(0)
        L.set_tau(tau)
        L.set_iolets(g.rho_mean, g.amp if amp is None else amp, g.period,
                     g.phase if phase is None else phase)
        r = L.objective_grad(lbm.OBJ_WSS, g.site_weight, nsteps, tb, te, scale=scale, n_snap=NSNAP)
        return r["J"]

    assert J() == got["J"]  # bitwise reproducible
    # the fp32 forward is rounding-noisy in tau below h ~ 3e-4 over 4000 steps
    ht, ha, hp = 1e-3, 1e-6, 1e-3
    d_tau = (J(tau=TAU + ht) - J(tau=TAU - ht)) / (2 * ht)
    d_amp = (J(amp=g.amp + [ha, 0]) - J(amp=g.amp - [ha, 0])) / (2 * ha)
    d_phase = (J(phase=g.phase + [hp, 0]) - J(phase=g.phase - [hp, 0])) / (2 * hp)
    errs = dict(dtau=abs(got["dtau"] / d_tau - 1), damp=abs(got["damp"][0] / d_amp - 1),
                dphase=abs(got["dphase"][0] / d_phase - 1))
    print("aneurysm 4000 steps: J", got["J"], "dtau", got["dtau"], d_tau, "damp", got["damp"][0],
          d_amp, "dphase", got["dphase"][0], d_phase, errs)
    for k, v in errs.items():
        assert v <= 5e-3, (k, v)
