"""The cluster-pair short-range kernel (MSM_SHORT_CLUSTER) against the oracle
and against the per-atom kernel.

Both kernels sum the same pairs of Eq. U_zero (every atom j and periodic image
with 0 < |d| < a) in different orders, so each output must match the FP64
oracle within the parity tolerances, and the two kernels must agree atom by
atom to FP32 summation-order rounding: |delta phi_i| and |delta F_i| at most
1e-5 (|x_i| + rms x), which a pair missing from either kernel (a term of about
|q_j| / r) exceeds by orders of magnitude. Boundary kinds: periodic, slabs open
along z and x, wires along z and y (p = 6), open, the water box (p = 6), p = 8,
rock salt, charges on a plane; a batch of systems; plans outside the kernel's
preconditions refuse the setting.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05961_gb300 import SHORT_CLUSTER, Batch, Plan, build  # noqa: E402
from paper_2510_05961_gb300 import workloads as W  # noqa: E402
from msm_testutil import expected_status  # noqa: E402

E_TOL = 1e-5
F_TOL = 1e-4
PAIR_TOL = 1e-5
DEV = torch.device("cuda", 0)

CASES = {
    "periodic_20001": lambda: W.random_box(20001, seed=31),
    "slab_3000": lambda: W.random_box(3000, seed=33, pbc=(1, 1, 0)),
    "slab_open_x_2000": lambda: W.random_box(2000, seed=45, pbc=(0, 1, 1)),
    "wire_z_2000": lambda: W.random_box(2000, seed=46, pbc=(0, 0, 1)),
    "wire_y_1200_p6": lambda: W.random_box(1200, seed=47, pbc=(0, 1, 0), p=6, h=1.5, a=6.0),
    "open_c1": lambda: W.open_cluster(),
    "water_600": lambda: W.water_box(nmol=600, L=26.2, seed=32),
    "open_p8": lambda: W.open_cluster(n=700, side=24.0, seed=37, h=1.6, a=6.0, p=8, levels=0),
    "rocksalt_6": lambda: W.rocksalt(ncell=6, seed=36),
    "sheet_slab": lambda: W.sheet(periodic=True, p=4, h=1.0),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    import oracle as O
    O.build()


def rel_rms(a, b):
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    return float(np.sqrt(((a - b) ** 2).sum(1).mean() / max((b ** 2).sum(1).mean(), 1e-300)))


def run(w, short_block):
    plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, w.levels, w.grid_override, max_atoms=w.n, device=DEV)
    plan.set_tuning(32, short_block)
    assert plan.info()["short_block"] == short_block
    pos = torch.from_numpy(w.pos).to(DEV)
    q = torch.from_numpy(w.q).to(DEV)
    E, phi, F = plan.forward(pos, q, forces=True, virial=True)
    gp, gq, Wv = plan.backward(torch.ones(1, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    assert plan.status() == expected_status(w)
    return dict(E=float(E.cpu()[0]), phi=phi.cpu().numpy().astype(np.float64),
                F=F.cpu().numpy().astype(np.float64), W=Wv.cpu().numpy(), dpos=gp.cpu().numpy(),
                dq=gq.cpu().numpy())


def per_atom_close(a, b, tol):
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    scale = np.sqrt((b ** 2).sum(1).mean())
    err = np.linalg.norm(a - b, axis=1)
    bound = tol * (np.linalg.norm(b, axis=1) + scale)
    return bool((err <= bound).all()), float((err / bound).max())


@pytest.mark.parametrize("key", list(CASES))
def test_cluster_kernel_matches_oracle_and_per_atom_kernel(key):
    import oracle as O
    w = CASES[key]()
    rc = run(w, SHORT_CLUSTER)
    ra = run(w, 256)
    ref = O.msm(O.plan_for(w), w.pos.astype(np.float64), w.q.astype(np.float64), forces=True, virial=True)
    assert abs(rc["E"] - ref["E"]) <= E_TOL * abs(ref["E"]), (rc["E"], ref["E"])
    assert rel_rms(rc["F"], ref["F"]) <= F_TOL
    assert rel_rms(rc["phi"], ref["phi"]) <= F_TOL
    assert rel_rms(rc["dq"], ref["phi"]) <= F_TOL
    assert rel_rms(rc["dpos"], -ref["F"]) <= F_TOL
    assert np.abs(rc["W"] - ref["W"]).max() <= F_TOL * np.abs(ref["W"]).max(), (rc["W"], ref["W"])
    ok, worst = per_atom_close(rc["phi"], ra["phi"], PAIR_TOL)
    assert ok, ("phi", worst)
    ok, worst = per_atom_close(rc["F"], ra["F"], PAIR_TOL)
    assert ok, ("F", worst)
    assert abs(rc["E"] - ra["E"]) <= PAIR_TOL * abs(ra["E"])
    assert np.abs(rc["W"] - ra["W"]).max() <= 2 * PAIR_TOL * np.abs(ra["W"]).max()


def test_cluster_kernel_is_reproducible():
    w = CASES["periodic_20001"]()
    r1 = run(w, SHORT_CLUSTER)
    r2 = run(w, SHORT_CLUSTER)
    assert r1["E"] == r2["E"]
    assert np.array_equal(r1["phi"], r2["phi"]) and np.array_equal(r1["F"], r2["F"])
    assert np.array_equal(r1["W"], r2["W"])


def test_cluster_kernel_batch():
    import oracle as O
    systems = W.batch_systems(nsys=12, seed=64, nmin=1500, nmax=4000)
    batch = Batch(systems, device=DEV)
    batch.set_tuning(32, SHORT_CLUSTER)
    pos = torch.from_numpy(np.concatenate([s.pos for s in systems])).to(DEV)
    q = torch.from_numpy(np.concatenate([s.q for s in systems])).to(DEV)
    E, phi, F = batch.forward(pos, q, forces=True, virial=True)
    gp, gq, Wb = batch.backward(torch.ones(len(systems), dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    assert batch.status() == expected_status(systems)
    E, F, Wb = E.cpu().numpy(), F.cpu().numpy(), Wb.cpu().numpy()
    off = 0
    for s, sw in enumerate(systems):
        ref = O.msm(O.plan_for(sw), sw.pos.astype(np.float64), sw.q.astype(np.float64), forces=True, virial=True)
        floor = 1e-7 * 0.5 * float(np.abs(sw.q.astype(np.float64) * ref["phi"]).sum())
        assert abs(E[s] - ref["E"]) <= E_TOL * abs(ref["E"]) + floor, s
        assert rel_rms(F[off:off + sw.n], ref["F"]) <= F_TOL, s
        assert np.abs(Wb[s] - ref["W"]).max() <= F_TOL * np.abs(ref["W"]).max(), s
        off += sw.n


def test_plans_outside_the_preconditions_refuse():
    # a periodic cell shorter than a + 2 e_z along z, and a tilted cell
    small = W.random_box(40, density=0.08, seed=34)
    plan = Plan(small.cell, small.pbc, small.h, small.a, small.p, max_atoms=small.n, device=DEV)
    with pytest.raises(Exception):
        plan.set_tuning(32, SHORT_CLUSTER)
    assert plan.info()["short_block"] in (128, 256)
    A = np.array([[30.0, 0, 0], [6.0, 30.0, 0], [0, 0, 30.0]])
    tilted = Plan(A.reshape(9), (1, 1, 1), 0.0, 6.0, 4, 0, (16, 16, 16), max_atoms=100, device=DEV)
    with pytest.raises(Exception):
        tilted.set_tuning(32, SHORT_CLUSTER)
