"""The checked build (libhemelb_gb300_checked.so: every table entry a step
kernel loads is range-checked and an out-of-range one would set the error
word that lbm_mass reports): on the paper-sized aneurysm in all four storage
and streaming forms, and on random masks with velocity iolets and
interpolated walls, it meets no out-of-range entry and gives the states of
the release build bit for bit.  Each build runs in a child process of its
own (the binding loads one library per process)."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import hashlib, json, sys
import numpy as np
sys.path.insert(0, %r)
import bench
from paper_1906_11925_gb300 import geometry as G, lbm
out = {"lib": lbm.load_library()._name}
g = bench.make_geometry("aneurysm")
nbr, link = lbm.links_build(15, g.xyz, g.io_xyz, g.io_id, g.periodic)
for storage in (lbm.STORE_FP32, lbm.STORE_FP16):
    for streaming in (lbm.STREAM_PULL, lbm.STREAM_AA):
        L = lbm.Lattice(15, g.xyz, nbr, link, 0.55, storage=storage, streaming=streaming,
                        rho_mean=g.rho_mean, amp=g.amp, period=g.period, phase=g.phase, stream=0)
        L.step(45)
        out["aneurysm_%%d_%%d" %% (storage, streaming)] = [hashlib.sha256(L.get_state().tobytes()).hexdigest(), L.mass()]
        L.close()
for q in (15, 19):
    m = G.random_mask((12, 11, 10), p=0.6, seed=95 + q, n_iolets=2)
    nb, lk = lbm.links_build(q, m.xyz, m.io_xyz, m.io_id, m.periodic)
    rng = np.random.default_rng(q)
    wq = np.round(rng.uniform(0.0, 1.0, (q, m.n)) * 2 ** 24).clip(1) / 2 ** 24
    kw = dict(rho_mean=[1.002, 0.02], amp=[0.001, 0.0], period=[17.0, 0.0], phase=[0.3, 0.0],
              iolet_kind=[0, 1], iolet_normal=[[0, 0, 0], [0.6, 0.0, 0.8]], stream=0)
    for streaming, wall_q in ((lbm.STREAM_PULL, wq), (lbm.STREAM_PULL, None), (lbm.STREAM_AA, None)):
        L = lbm.Lattice(q, m.xyz, nb, lk, 0.7, streaming=streaming, wall_q=wall_q, **kw)
        L.step(37)
        out["mask_%%d_%%d_%%d" %% (q, streaming, wall_q is not None)] = [hashlib.sha256(L.get_state().tobytes()).hexdigest(), L.mass()]
        L.close()
print(json.dumps(out))
""" % ROOT


def run(checked: bool):
    env = dict(os.environ, HEMELB_GB300_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_matches_release_and_finds_no_bad_entry():
    rel, chk = run(False), run(True)
    assert rel.pop("lib").endswith("libhemelb_gb300.so")
    assert chk.pop("lib").endswith("libhemelb_gb300_checked.so")
    assert len(rel) == 10
    assert rel == chk
