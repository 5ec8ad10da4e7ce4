"""Dynamic cells (msm_plan_set_cell): one plan, its cell changed between calls.

The plan keeps its grid counts M and stencil sizes; the stencils for the new
spacings h_1 = L / M are recomputed on the device (periodic, p = 4) or on the
host (every other setting). Each cell is checked against the
FP64 oracle planned for that cell with the same M (grid_override), with the
parity tolerances; a compression beyond the plan's stencil radius is refused;
returning to the creation cell reproduces a fresh plan.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05961_gb300 import Plan, build  # noqa: E402
from paper_2510_05961_gb300 import _lib as L  # noqa: E402
from paper_2510_05961_gb300 import workloads as W  # noqa: E402
from msm_testutil import expected_for  # noqa: E402

E_TOL = 1e-5
F_TOL = 1e-4
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    import oracle as O
    O.build()


def rel_rms(a, b):
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    return float(np.sqrt(((a - b) ** 2).sum(1).mean() / max((b ** 2).sum(1).mean(), 1e-300)))


def run(plan, pos, q):
    E, phi, F = plan.forward(torch.from_numpy(pos).to(DEV), torch.from_numpy(q).to(DEV), forces=True, virial=True)
    gp, gq, Wv = plan.backward(torch.ones(1, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    assert plan.status() == expected_for(plan.params.pbc, q)
    return dict(E=float(E.cpu()[0]), phi=phi.cpu().numpy(), F=F.cpu().numpy(), W=Wv.cpu().numpy())


def oracle_for(cell, w, M, pos):
    import oracle as O
    P = O.make_plan(cell, w.pbc, w.h, w.a, w.p, w.levels, tuple(M), w.qi_mode)
    return O.msm(P, pos.astype(np.float64), w.q.astype(np.float64), forces=True, virial=True)


CASES = {
    # device path: periodic, p = 4, raw-sample balls on every level
    "periodic_p4_20001": lambda: W.random_box(20001, seed=91),
    "periodic_p4_3000": lambda: W.random_box(3000, seed=92),
    # host path: omega'-convolved stencils (p = 6), folded or dense boxes (open, slab, wire, exact interpolation)
    "periodic_p6_3000": lambda: W.random_box(3000, seed=96, p=6, h=1.5, a=6.0),
    "slab_3000": lambda: W.random_box(3000, seed=97, pbc=(1, 1, 0)),
    "wire_1500": lambda: W.random_box(1500, seed=95, pbc=(0, 0, 1)),
    "open_1500": lambda: W.random_box(1500, seed=98, pbc=(0, 0, 0)),
    "periodic_qi1_400": lambda: dataclasses.replace(W.random_box(400, seed=99, h=2.0, a=4.0), qi_mode=1),
}


@pytest.mark.parametrize("key", list(CASES))
def test_cell_changes_match_oracle(key):
    import oracle as O
    w = CASES[key]()
    M = [O.plan_for(w).M[d] for d in range(3)]
    base = np.array(w.cell, np.float64)
    # built for the most compressed cell it will serve
    plan = Plan(tuple(base * 0.97), w.pbc, w.h, w.a, w.p, w.levels, tuple(M), max_atoms=w.n, device=DEV,
                qi_mode=w.qi_mode)
    for s in [(1.0, 1.0, 1.0), (1.04, 0.99, 1.02), (0.97, 0.97, 0.97), (1.1, 1.1, 1.1)]:
        cell = base * np.array(s)
        pos = (w.pos.astype(np.float64) * np.array(s)).astype(np.float32)
        plan.set_cell(cell)
        info = plan.info()
        assert np.allclose(info["h1"], cell / np.array(M))
        r = run(plan, pos, w.q)
        ref = oracle_for(cell, w, M, pos)
        assert abs(r["E"] - ref["E"]) <= E_TOL * abs(ref["E"]), (s, r["E"], ref["E"])
        assert rel_rms(r["F"], ref["F"]) <= F_TOL, s
        assert rel_rms(r["phi"], ref["phi"]) <= F_TOL, s
        assert np.abs(r["W"] - ref["W"]).max() <= F_TOL * np.abs(ref["W"]).max(), s


def test_compression_beyond_capacity_is_refused_and_creation_cell_is_reproduced():
    import oracle as O
    w = W.random_box(8000, seed=93)
    M = [O.plan_for(w).M[d] for d in range(3)]
    base = np.array(w.cell, np.float64)
    plan = Plan(tuple(base), w.pbc, w.h, w.a, w.p, w.levels, tuple(M), max_atoms=w.n, device=DEV)
    r0 = run(plan, w.pos, w.q)
    with pytest.raises(L.MsmError) as e:
        plan.set_cell(base * 0.8)
    assert e.value.code == L.MSM_ERR_CAPACITY
    plan.set_cell(base * 1.05)
    run(plan, (w.pos.astype(np.float64) * 1.05).astype(np.float32), w.q)
    plan.set_cell(base)
    r1 = run(plan, w.pos, w.q)
    assert r1["E"] == pytest.approx(r0["E"], rel=1e-6)
    assert np.allclose(r1["F"], r0["F"], rtol=1e-4, atol=1e-5 * np.abs(r0["F"]).max())
    assert np.allclose(r1["W"], r0["W"], rtol=1e-5, atol=1e-6 * np.abs(r0["W"]).max())


def test_non_orthorhombic_cell_is_refused():
    w = W.random_box(500, seed=94)
    plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, w.levels, max_atoms=w.n, device=DEV)
    c = np.diag(np.array(w.cell, np.float64))
    c[0, 1] = 0.5
    with pytest.raises(L.MsmError) as e:
        plan.set_cell(c)
    assert e.value.code == L.MSM_ERR_UNSUPPORTED
