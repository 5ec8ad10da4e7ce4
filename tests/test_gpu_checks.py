"""The debug build with device-side index checks (-DMSM_CHECKS=1).

Memory checkers are not available on this machine, so the library has a debug
build whose kernels test their data-dependent indices (candidate ranges read
from cell_start, bucket slots, the sort permutation, grid indices of the
interpolation) before each access; a failed test sets MSM_DEV_CHECK in the
status word and skips the access. This test builds that library and runs it,
in a fresh process (the binding loads one library per process), on small
cases of every boundary kind (with the per-atom and, where the plan allows
them, the cluster-pair short-range kernel and the spectral level method), a
tilted cell, a dense cluster and a batch:
no check may fire, and the outputs must match the FP64 oracle as in the
other parity tests.
"""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import oracle as O
from paper_2510_05961_gb300 import SHORT_CLUSTER, Batch, Plan, _lib
from paper_2510_05961_gb300 import workloads as W
O.build()
dev = torch.device("cuda", 0)

def rel_rms(a, b):
    a = np.asarray(a, np.float64).reshape(len(a), -1); b = np.asarray(b, np.float64).reshape(len(b), -1)
    return float(np.sqrt(((a - b) ** 2).sum(1).mean() / max((b ** 2).sum(1).mean(), 1e-300)))

def cluster():
    rng = np.random.default_rng(6100)
    v = rng.normal(size=(2000, 3))
    v *= (3.0 * rng.uniform(size=(2000, 1)) ** (1 / 3)) / np.linalg.norm(v, axis=1, keepdims=True)
    q = rng.normal(0.0, 0.5, size=2000); q -= q.mean()
    return W.Workload("cluster", (v + 30.0).astype(np.float32), q.astype(np.float32), (60.0,) * 3, (0, 0, 0), 2.0, 8.0, 4)

def tilted():
    L = 20.0
    A = np.array([[L, 0, 0], [0.4 * L, L, 0], [0.1 * L, -0.2 * L, L]])
    rng = np.random.default_rng(6200)
    frac = rng.uniform(0, 1, (1500, 3))
    q = np.where(np.arange(1500) % 2 == 0, 1.0, -1.0)
    return A, (frac @ A).astype(np.float32), q.astype(np.float32)

out = {"lib": __import__("os").environ["MSM_GB300_LIB"], "cases": []}
cases = [W.random_box(3000, seed=6301), W.random_box(1200, seed=6302, pbc=(1, 1, 0)),
         W.random_box(900, seed=6303, pbc=(0, 0, 1)), W.open_cluster(n=500, side=24.0, seed=6304), cluster(),
         W.random_box(40, density=0.08, seed=6305)]
for w in cases:
    ref = O.msm(O.plan_for(w), w.pos.astype(np.float64), w.q.astype(np.float64))
    for sb, lm in ((256, 0), (SHORT_CLUSTER, 0), (256, 1)):
        plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, w.levels, max_atoms=w.n, device=dev)
        try:
            plan.set_tuning(32, sb)
            plan.set_level_method(lm)
        except Exception:
            continue  # outside the cluster kernel's or the spectral method's preconditions
        pos = torch.from_numpy(w.pos).to(dev); q = torch.from_numpy(w.q).to(dev)
        E, phi, F = plan.forward(pos, q, forces=True, virial=True)
        gp, gq, Wv = plan.backward(torch.ones(1, dtype=torch.float64, device=dev))
        torch.cuda.synchronize()
        st = plan.status()
        out["cases"].append({"name": "%s/%d/%d" % (w.name, sb, lm), "status": st,
                             "eE": abs(E.item() - ref["E"]) / abs(ref["E"]),
                             "eF": rel_rms(F.cpu().numpy(), ref["F"]), "ephi": rel_rms(phi.cpu().numpy(), ref["phi"]),
                             "eW": float(np.abs(Wv.cpu().numpy() - ref["W"]).max() / np.abs(ref["W"]).max())})
A, pos_t, q_t = tilted()
plan = Plan(A.reshape(9), (1, 1, 1), 0.0, 6.0, 4, 0, (16, 16, 16), max_atoms=len(q_t), device=dev)
E, phi, F = plan.forward(torch.from_numpy(pos_t).to(dev), torch.from_numpy(q_t).to(dev), forces=True, virial=True)
torch.cuda.synchronize()
ref = O.msm(O.make_plan(A, (1, 1, 1), 0, 6.0, 4, grid_override=(16, 16, 16)), pos_t.astype(np.float64),
            q_t.astype(np.float64))
out["cases"].append({"name": "tilted", "status": plan.status(), "eE": abs(E.item() - ref["E"]) / abs(ref["E"]),
                     "eF": rel_rms(F.cpu().numpy(), ref["F"]), "ephi": rel_rms(phi.cpu().numpy(), ref["phi"]), "eW": 0.0})
systems = W.batch_systems(nsys=9, seed=6306, nmax=400)
batch = Batch(systems, device=dev)
pos = torch.from_numpy(np.concatenate([s.pos for s in systems])).to(dev)
q = torch.from_numpy(np.concatenate([s.q for s in systems])).to(dev)
E, phi, F = batch.forward(pos, q, forces=True, virial=True)
batch.backward(torch.ones(len(systems), dtype=torch.float64, device=dev))
torch.cuda.synchronize()
out["batch_status"] = batch.status()
E = E.cpu().numpy()
ok = []
for s, w in enumerate(systems):
    ref = O.msm(O.plan_for(w), w.pos.astype(np.float64), w.q.astype(np.float64))
    floor = 1e-7 * 0.5 * float(np.abs(w.q.astype(np.float64) * ref["phi"]).sum())
    ok.append(bool(abs(E[s] - ref["E"]) <= 1e-5 * abs(ref["E"]) + floor))
out["batch_ok"] = ok
print("RESULT " + json.dumps(out))
'''


def test_checked_build_runs_clean():
    from paper_2510_05961_gb300 import _lib, build
    lib = build.build(checks=True)
    env = dict(os.environ, MSM_GB300_LIB=lib)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1][7:])
    assert res["lib"].endswith("libmsm_gb300_checks.so")
    for c in res["cases"]:
        assert c["status"] & _lib.MSM_DEV_CHECK == 0, c
        assert c["status"] & _lib.MSM_DEV_ERRORS == 0, c
        assert c["eE"] <= 1e-5 and c["eF"] <= 1e-4 and c["ephi"] <= 1e-4 and c["eW"] <= 1e-4, c
    assert res["batch_status"] & _lib.MSM_DEV_ERRORS == 0
    assert all(res["batch_ok"]), res["batch_ok"]
