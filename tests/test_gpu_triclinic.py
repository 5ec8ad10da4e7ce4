"""Tilted (triclinic) periodic cells on the GPU against the FP64 oracle.

The cell rows a, b, c need not be orthogonal: binning follows the FP32
contract s = A^-T r bit for bit, the short-range kernel visits the cells
within the cutoff's fractional reach, the stencils follow the cell's metric
(dense boxes on every level) and the grid gradients map through A^-1 diag(M).
Tolerances as in the other parity tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05961_gb300 import Plan, build  # noqa: E402
from msm_testutil import expected_for, expected_status  # noqa: E402

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


def tilted(kind, n, seed, density=0.1):
    """Atoms uniform in a tilted cell of the given volume; +/-1 charges."""
    rng = np.random.default_rng(seed)
    L = (n / density) ** (1.0 / 3.0)
    if kind == "sheared":
        A = np.array([[L, 0, 0], [0.5 * L, L, 0], [0.2 * L, -0.3 * L, L]])
    elif kind == "monoclinic":
        c = L / np.sin(np.radians(105.0))
        A = np.array([[L, 0, 0], [0, L, 0], [c * np.cos(np.radians(105.0)), 0, L]])
    else:  # hexagonal
        A = np.array([[L, 0, 0], [-0.5 * L, np.sqrt(3) / 2 * L, 0], [0, 0, L / (np.sqrt(3) / 2)]])
    s = rng.uniform(0, 1, (n, 3))
    pos = (s @ A).astype(np.float32)
    q = np.concatenate([np.ones(n // 2), -np.ones(n - n // 2)]).astype(np.float32)
    rng.shuffle(q)
    return A, pos, q


CASES = [("sheared", 3000, 51, 4, 6.0, 16), ("monoclinic", 6000, 52, 6, 7.0, 16), ("hexagonal", 4000, 53, 4, 6.0, 16),
         ("sheared", 20000, 54, 4, 8.0, 32)]


@pytest.mark.parametrize("kind,n,seed,p,a,M", CASES)
def test_tilted_cell_matches_oracle(kind, n, seed, p, a, M):
    import oracle as O
    A, pos, q = tilted(kind, n, seed)
    plan = Plan(A.reshape(9), (1, 1, 1), 0.0, a, p, 0, (M, M, M), max_atoms=n, device=DEV)
    P = O.make_plan(A, (1, 1, 1), 0, a, p, grid_override=(M, M, M))
    assert P.tri == 1
    info = plan.info()
    assert list(info["R"]) == [P.R[d] for d in range(3)] and list(info["C"]) == [P.C[d] for d in range(3)]
    # binning: bit-exact with the oracle's FP32 contract
    cid, start, perm, st = O.bin_atoms(P, pos, q)
    tp, tq = torch.from_numpy(pos).to(DEV), torch.from_numpy(q).to(DEV)
    E, phi, F = plan.forward(tp, tq, forces=True, virial=True)
    gp, gq, Wv = plan.backward(torch.ones(1, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    assert plan.status() == expected_for((1, 1, 1), q)
    assert np.array_equal(plan.debug_array(0).cpu().numpy(), start)
    assert np.array_equal(plan.debug_array(1).cpu().numpy(), perm)
    ref = O.msm(P, pos.astype(np.float64), q.astype(np.float64), forces=True, virial=True)
    assert abs(float(E.cpu()[0]) - ref["E"]) <= E_TOL * abs(ref["E"])
    assert rel_rms(F.cpu().numpy(), ref["F"]) <= F_TOL
    assert rel_rms(phi.cpu().numpy(), ref["phi"]) <= F_TOL
    assert rel_rms(gp.cpu().numpy(), -ref["F"]) <= F_TOL
    Wr = ref["W"]
    assert np.abs(Wv.cpu().numpy() - Wr).max() <= F_TOL * np.abs(Wr).max()


def test_tilted_cell_field_and_force_gradients():
    # msm_field and the force vector-Jacobian product (L = sum u . F) in a tilted cell:
    # dL/dq = -D_u phi and dL/dr = D_u F, central differences of the FP64 oracle along u
    import oracle as O
    from paper_2510_05961_gb300 import msm_outputs
    A, pos, q = tilted("sheared", 3000, 55)
    plan = Plan(A.reshape(9), (1, 1, 1), 0.0, 6.0, 4, 0, (16, 16, 16), max_atoms=len(q), device=DEV)
    tp, tq = torch.from_numpy(pos).to(DEV), torch.from_numpy(q).to(DEV)
    plan.forward(tp, tq, forces=True)
    P = O.make_plan(A, (1, 1, 1), 0, 6.0, 4, grid_override=(16, 16, 16))
    pd, qd = pos.astype(np.float64), q.astype(np.float64)
    ref = O.msm(P, pd, qd, forces=True, virial=False)
    assert rel_rms(plan.field().cpu().numpy(), ref["F"] / qd[:, None]) <= F_TOL
    u = np.random.default_rng(56).normal(size=pos.shape)
    x = tp.clone().requires_grad_(True)
    y = tq.clone().requires_grad_(True)
    E, phi, F = msm_outputs(x, y, plan)
    (torch.from_numpy(u.astype(np.float32)).to(DEV) * F).sum().backward()
    torch.cuda.synchronize()
    eps = 1e-4
    rp = O.msm(P, pd + eps * u, qd, forces=True, virial=False)
    rm = O.msm(P, pd - eps * u, qd, forces=True, virial=False)
    assert rel_rms(y.grad.cpu().numpy(), -(rp["phi"] - rm["phi"]) / (2 * eps)) <= F_TOL
    assert rel_rms(x.grad.cpu().numpy(), (rp["F"] - rm["F"]) / (2 * eps)) <= F_TOL


def test_tilted_cell_dynamic_cell():
    # a plan built for a tilted cell takes later cells (strained, re-tilted, rectangular) within its
    # capacity; each against the oracle planned for that cell with the same grid counts
    import oracle as O
    from paper_2510_05961_gb300 import _lib as L
    A, pos, q = tilted("sheared", 3000, 57)
    plan = Plan((A * 0.96).reshape(9), (1, 1, 1), 0.0, 6.0, 4, 0, (16, 16, 16), max_atoms=len(q), device=DEV)
    frac = pos.astype(np.float64) @ np.linalg.inv(A)
    for B in (A, A @ (np.eye(3) + np.array([[0.02, 0.01, 0], [0, -0.01, 0.02], [0, 0, 0.03]])).T,
              np.diag(np.diag(A)) * 1.0):
        plan.set_cell(B)
        pb = (frac @ B).astype(np.float32)
        tp, tq = torch.from_numpy(pb).to(DEV), torch.from_numpy(q).to(DEV)
        E, phi, F = plan.forward(tp, tq, forces=True, virial=True)
        gp, gq, Wv = plan.backward(torch.ones(1, dtype=torch.float64, device=DEV))
        torch.cuda.synchronize()
        assert plan.status() == expected_for((1, 1, 1), q)
        P = O.make_plan(B, (1, 1, 1), 0, 6.0, 4, grid_override=(16, 16, 16))
        ref = O.msm(P, pb.astype(np.float64), q.astype(np.float64), forces=True, virial=True)
        assert abs(float(E.cpu()[0]) - ref["E"]) <= E_TOL * abs(ref["E"])
        assert rel_rms(F.cpu().numpy(), ref["F"]) <= F_TOL
        assert np.abs(Wv.cpu().numpy() - ref["W"]).max() <= F_TOL * np.abs(ref["W"]).max()
    with pytest.raises(L.MsmError) as e:
        plan.set_cell(A * 0.8)
    assert e.value.code == L.MSM_ERR_CAPACITY


def test_batch_mixing_tilted_and_rectangular_cells():
    # one batch with tilted and rectangular cells: every system against the oracle
    import dataclasses

    import oracle as O
    from paper_2510_05961_gb300 import Batch
    from paper_2510_05961_gb300 import workloads as W
    systems, refs = [], []
    for k, (kind, n, seed) in enumerate([("sheared", 1500, 61), ("hexagonal", 900, 62), (None, 1200, 63),
                                         ("monoclinic", 700, 64)]):
        if kind is None:
            w = W.random_box(n, seed=seed, h=2.0, a=6.0)
            w = dataclasses.replace(w, grid_override=(16, 16, 16), h=0.0)
            A = np.diag(w.cell)
            pos, q = w.pos, w.q
        else:
            A, pos, q = tilted(kind, n, seed)
            w = W.Workload(name=kind, pos=pos, q=q, cell=tuple(A.reshape(9)), pbc=(1, 1, 1), h=0.0, a=6.0, p=4,
                           grid_override=(16, 16, 16))
        systems.append(w)
        P = O.make_plan(A, (1, 1, 1), 0, 6.0, 4, grid_override=(16, 16, 16))
        refs.append(O.msm(P, pos.astype(np.float64), q.astype(np.float64), forces=True, virial=True))
    batch = Batch(systems, device=DEV)
    tp = torch.from_numpy(np.concatenate([s.pos for s in systems])).to(DEV)
    tq = torch.from_numpy(np.concatenate([s.q for s in systems])).to(DEV)
    E, phi, F = batch.forward(tp, tq, forces=True, virial=True)
    _, _, Wb = batch.backward(torch.ones(len(systems), dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    assert batch.status() == expected_status(systems)
    E, F, Wb = E.cpu().numpy(), F.cpu().numpy(), Wb.cpu().numpy()
    off = 0
    for s, (w, r) in enumerate(zip(systems, refs)):
        assert abs(E[s] - r["E"]) <= E_TOL * abs(r["E"]) + 1e-7 * 0.5 * float(np.abs(w.q * r["phi"]).sum())
        assert rel_rms(F[off:off + w.n], r["F"]) <= F_TOL
        assert np.abs(Wb[s] - r["W"]).max() <= F_TOL * np.abs(r["W"]).max()
        off += w.n
