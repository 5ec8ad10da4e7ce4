"""The autotuner and every launch shape it chooses among.

Each (anterpolation tile z-extent, short-range kernel: 128 or 256 threads per
block of the per-atom kernel, or the cluster-pair kernel) pair is forced on a
single system and on a batch and checked against the oracle with the parity
tolerances; msm_autotune must pick valid shapes and leave results unchanged.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05961_gb300 import SHORT_CLUSTER, Batch, Plan, build  # noqa: E402
from paper_2510_05961_gb300 import workloads as W  # noqa: E402

DEV = torch.device("cuda", 0)
F_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    import oracle as O
    O.build()


def rel_rms(a, b):
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    return float(np.sqrt(((a - b) ** 2).sum(1).mean() / max((b ** 2).sum(1).mean(), 1e-300)))


def _ref(w):
    import oracle as O
    return O.msm(O.plan_for(w), w.pos.astype(np.float64), w.q.astype(np.float64), forces=True, virial=True)


@pytest.mark.parametrize("tz", [16, 32, 64])
@pytest.mark.parametrize("nb", [128, 256, SHORT_CLUSTER])
def test_every_shape_matches_oracle(tz, nb):
    w = W.random_box(9000, seed=61)
    ref = _ref(w)
    plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, max_atoms=w.n, device=DEV)
    plan.set_tuning(tz, nb)
    info = plan.info()
    assert (info["anterp_tz"], info["short_block"]) == (tz, nb)
    pos, q = torch.from_numpy(w.pos).to(DEV), torch.from_numpy(w.q).to(DEV)
    E, phi, F = plan.forward(pos, q, forces=True, virial=True)
    gp, gq, Wv = plan.backward(torch.ones(1, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    assert abs(float(E.cpu()[0]) - ref["E"]) <= 1e-5 * abs(ref["E"])
    assert rel_rms(F.cpu().numpy(), ref["F"]) <= F_TOL
    assert rel_rms(phi.cpu().numpy(), ref["phi"]) <= F_TOL
    assert np.abs(Wv.cpu().numpy() - ref["W"]).max() <= F_TOL * np.abs(ref["W"]).max()


def test_autotune_single_and_batch():
    w = W.random_box(20001, seed=62)
    ref = _ref(w)
    plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, max_atoms=w.n, device=DEV)
    pos, q = torch.from_numpy(w.pos).to(DEV), torch.from_numpy(w.q).to(DEV)
    choice = plan.autotune(pos, q)
    assert choice["anterp_tz"] in (16, 32, 64) and choice["short_block"] in (128, 256, SHORT_CLUSTER)
    E, phi, F = plan.forward(pos, q, forces=True)
    torch.cuda.synchronize()
    assert abs(float(E.cpu()[0]) - ref["E"]) <= 1e-5 * abs(ref["E"])
    assert rel_rms(F.cpu().numpy(), ref["F"]) <= F_TOL

    systems = W.batch_systems(nsys=40, seed=63, nmax=800)
    batch = Batch(systems, device=DEV)
    bpos = torch.from_numpy(np.concatenate([s.pos for s in systems])).to(DEV)
    bq = torch.from_numpy(np.concatenate([s.q for s in systems])).to(DEV)
    bchoice = batch.autotune(bpos, bq)
    # small periodic cubes of the batch are outside the cluster kernel's preconditions
    assert bchoice["anterp_tz"] in (16, 32, 64) and bchoice["short_block"] in (128, 256)
    for tz, nb in ((bchoice["anterp_tz"], bchoice["short_block"]), (16, 128), (64, 256)):
        batch.set_tuning(tz, nb)
        Eb, phib, Fb = batch.forward(bpos, bq, forces=True)
        torch.cuda.synchronize()
        Eb, Fb = Eb.cpu().numpy(), Fb.cpu().numpy()
        off = 0
        for s, sw in enumerate(systems):
            r = _ref(sw)
            floor = 1e-7 * 0.5 * float(np.abs(sw.q.astype(np.float64) * r["phi"]).sum())
            assert abs(Eb[s] - r["E"]) <= 1e-5 * abs(r["E"]) + floor
            assert rel_rms(Fb[off:off + sw.n], r["F"]) <= F_TOL
            off += sw.n
    with pytest.raises(Exception):
        batch.set_tuning(24, 256)
