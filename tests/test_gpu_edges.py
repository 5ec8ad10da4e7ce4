"""Edge-case inputs against the oracle.

- Sites exactly on level-1 grid points and binning-cell faces: an undisplaced
  rock-salt lattice with spacing a0/2 = h_1 (the planner's grid for h = 2 A on
  a 16 A cell), periodic, slab and open. Along open axes the crystal has a
  layer of sites on both faces (s = 0 and s = 1, x = L). These are the ties the
  FP32 binning contract (c = min((int)(s C), C - 1)) and the vanishing B-spline
  end values Phi_p(+-p/2) = 0 (Sec. 3.3's index set of the interpolation)
  settle; the binning must be bit-exact and every output within the parity
  tolerances.
- A clustered input: 5000 atoms in a ball of radius 3 A inside a 60 A open
  box (about 44 atoms / A^3; up to 1383 atoms in one binning cell, against
  about 2 at the benchmark density), so the stable rank within a cell is long;
  binning bit-exact and full parity.
Both cases run with the per-atom and the cluster-pair short-range kernels.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05961_gb300 import SHORT_CLUSTER, Plan, build  # noqa: E402
from paper_2510_05961_gb300 import workloads as W  # noqa: E402
from msm_testutil import expected_status  # noqa: E402

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


def run_and_compare(w, short_block=256):
    import oracle as O
    plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, w.levels, w.grid_override, max_atoms=w.n, device=DEV)
    plan.set_tuning(32, short_block)
    pos = torch.from_numpy(w.pos).to(DEV)
    q = torch.from_numpy(w.q).to(DEV)
    E, phi, F = plan.forward(pos, q, forces=True, virial=True)
    gp, gq, Wv = plan.backward(torch.ones(1, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    assert plan.status() == expected_status(w)
    P = O.plan_for(w)
    cid, start, perm, st = O.bin_atoms(P, w.pos, w.q)
    assert st == 0
    assert np.array_equal(plan.debug_array(0).cpu().numpy(), start)
    assert np.array_equal(plan.debug_array(1).cpu().numpy(), perm)
    assert np.array_equal(plan.debug_array(4).cpu().numpy(), cid[perm])
    ref = O.msm(P, w.pos.astype(np.float64), w.q.astype(np.float64), forces=True, virial=True)
    assert abs(float(E.cpu()[0]) - ref["E"]) <= E_TOL * abs(ref["E"])
    assert rel_rms(phi.cpu().numpy(), ref["phi"]) <= F_TOL
    assert rel_rms(F.cpu().numpy(), ref["F"]) <= F_TOL
    assert rel_rms(gq.cpu().numpy(), ref["phi"]) <= F_TOL
    assert rel_rms(gp.cpu().numpy(), -ref["F"]) <= F_TOL
    assert np.abs(Wv.cpu().numpy() - ref["W"]).max() <= F_TOL * np.abs(ref["W"]).max()
    return P


@pytest.mark.parametrize("short_block", [256, SHORT_CLUSTER], ids=["per_atom", "cluster"])
@pytest.mark.parametrize("pbc", [(1, 1, 1), (1, 1, 0), (0, 0, 0)], ids=["periodic", "slab", "open"])
def test_lattice_on_grid_points_and_cell_faces(pbc, short_block):
    w = W.lattice_on_grid(pbc=pbc)
    P = run_and_compare(w, short_block)
    # the sites really are on grid points and cell faces
    u = w.pos.astype(np.float64) / np.array([P.h1[d] for d in range(3)])
    assert np.array_equal(u, np.round(u))
    edge = np.array([P.edge[d] for d in range(3)])
    assert (np.abs(w.pos / edge - np.round(w.pos / edge)) == 0).mean() > 0.4
    for d in range(3):
        if not pbc[d]:
            assert (w.pos[:, d] == np.float32(w.cell[d])).any() and (w.pos[:, d] == 0).any()


@pytest.mark.parametrize("short_block", [256, SHORT_CLUSTER], ids=["per_atom", "cluster"])
def test_clustered_input(short_block):
    rng = np.random.default_rng(6100)
    n, R, side = 5000, 3.0, 60.0
    v = rng.normal(size=(n, 3))
    v *= (R * rng.uniform(size=(n, 1)) ** (1 / 3)) / np.linalg.norm(v, axis=1, keepdims=True)
    pos = (v + side / 2).astype(np.float32)
    q = rng.normal(0.0, 0.5, size=n)
    q -= q.mean()
    w = W.Workload("cluster_ball", pos, q.astype(np.float32), (side,) * 3, (0, 0, 0), 2.0, 8.0, 4)
    run_and_compare(w, short_block)
