"""The spectral level method (MSM_LEVELS_SPECTRAL): the level stencils applied
as products with their discrete Fourier transforms between FFTs of the level
grids, and the grid virial by Parseval's identity.

On a periodic grid the stencil sum of Eq. action_of_K_as_convolution is a
circular convolution with the folded stencil, so both methods apply the same
operator; every output must match the FP64 oracle within the parity
tolerances, every level's grid potential e^l must match the oracle's to 1e-4
of the largest level-1 entry, and the two methods must agree to FP32 rounding
(potentials and forces to 1e-5 relative RMS, the virial to 1e-5 of its largest
entry). Cases: random periodic boxes (cubic, and a rectangular cell with three
different spacings), the water box (p = 6), rock salt, p = 8; the virial when
the forward skipped it; dynamic cells on a spectral plan and a switch after a
device-path cell change; the autotuner; refusals on plans that do not allow it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05961_gb300 import LEVELS_BALL, LEVELS_SPECTRAL, Batch, Plan, build  # noqa: E402
from paper_2510_05961_gb300 import workloads as W  # noqa: E402
from msm_testutil import expected_status  # noqa: E402

E_TOL = 1e-5
F_TOL = 1e-4
AGREE = 1e-5
DEV = torch.device("cuda", 0)


def rect_box(seed=71):
    """Periodic rectangular cell 60 x 48 x 54 A on a 32^3 grid (spacings 1.875, 1.5, 1.6875 A)."""
    rng = np.random.default_rng(seed)
    cell = (60.0, 48.0, 54.0)
    n = 12000
    pos = (rng.uniform(size=(n, 3)) * np.array(cell)).astype(np.float32)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0).astype(np.float32)
    w = W.Workload("rect_12000", pos, q, cell, (1, 1, 1), 0.0, 8.0, 4)
    w.grid_override = (32, 32, 32)
    return w


CASES = {
    "periodic_20001": lambda: W.random_box(20001, seed=31),
    "rect_12000": rect_box,
    "water_600": lambda: W.water_box(nmol=600, L=26.2, seed=32),
    "rocksalt_6": lambda: W.rocksalt(ncell=6, seed=36),
    "periodic_p8": lambda: W.random_box(6000, seed=72, p=8, h=1.6, a=7.0),
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


def make_plan(w, method):
    plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, w.levels, w.grid_override, max_atoms=w.n, device=DEV)
    assert plan.info()["spectral_ok"]
    plan.set_level_method(method)
    assert plan.info()["level_method"] == method
    return plan


def run(w, method, virial_in_forward=True, plan=None):
    plan = plan or make_plan(w, method)
    pos = torch.from_numpy(w.pos).to(DEV)
    q = torch.from_numpy(w.q).to(DEV)
    E, phi, F = plan.forward(pos, q, forces=True, virial=virial_in_forward)
    levels = []
    for l in range(1, plan.info()["ncomp"] + 1):
        levels.append(plan.debug_array(3, l).cpu().numpy().copy())
    gp, gq, Wv = plan.backward(torch.ones(1, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    assert plan.status() == expected_status(w)
    return dict(plan=plan, E=float(E.cpu()[0]), phi=phi.cpu().numpy(), F=F.cpu().numpy(), W=Wv.cpu().numpy(),
                dpos=gp.cpu().numpy(), dq=gq.cpu().numpy(), elev=levels)


def oracle(w):
    import oracle as O
    P = O.plan_for(w)
    return P, O.msm(P, w.pos.astype(np.float64), w.q.astype(np.float64), forces=True, virial=True, grids=True)


def check_oracle(r, ref):
    assert abs(r["E"] - ref["E"]) <= E_TOL * abs(ref["E"]), (r["E"], ref["E"])
    assert rel_rms(r["F"], ref["F"]) <= F_TOL
    assert rel_rms(r["phi"], ref["phi"]) <= F_TOL
    assert rel_rms(r["dq"], ref["phi"]) <= F_TOL
    assert rel_rms(r["dpos"], -ref["F"]) <= F_TOL
    assert np.abs(r["W"] - ref["W"]).max() <= F_TOL * np.abs(ref["W"]).max(), (r["W"], ref["W"])


@pytest.mark.parametrize("key", list(CASES))
def test_spectral_matches_oracle_and_ball_method(key):
    w = CASES[key]()
    P, ref = oracle(w)
    rs = run(w, LEVELS_SPECTRAL)
    rb = run(w, LEVELS_BALL)
    check_oracle(rs, ref)
    escale = np.abs(ref["elev"][0]).max()
    for l in range(1, P.ncomp + 1):
        eo = ref["elev"][l - 1].reshape(-1)
        assert np.abs(rs["elev"][l - 1] - eo).max() <= 1e-4 * escale, ("e", l)
        assert np.abs(rs["elev"][l - 1] - rb["elev"][l - 1]).max() <= AGREE * escale, ("e vs ball", l)
    assert rel_rms(rs["phi"], rb["phi"]) <= AGREE
    assert rel_rms(rs["F"], rb["F"]) <= AGREE
    assert abs(rs["E"] - rb["E"]) <= AGREE * abs(rb["E"])
    assert np.abs(rs["W"] - rb["W"]).max() <= AGREE * np.abs(rb["W"]).max(), (rs["W"], rb["W"])


def test_spectral_virial_without_forward_virial():
    w = CASES["periodic_20001"]()
    P, ref = oracle(w)
    r = run(w, LEVELS_SPECTRAL, virial_in_forward=False)
    check_oracle(r, ref)


def _oracle_for(cell, w, M, pos):
    import oracle as O
    P = O.make_plan(cell, w.pbc, w.h, w.a, w.p, w.levels, tuple(M), w.qi_mode)
    return O.msm(P, pos.astype(np.float64), w.q.astype(np.float64), forces=True, virial=True)


def _run_cell(plan, pos, q):
    E, phi, F = plan.forward(torch.from_numpy(pos).to(DEV), torch.from_numpy(q).to(DEV), forces=True, virial=True)
    gp, gq, Wv = plan.backward(torch.ones(1, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    return dict(E=float(E.cpu()[0]), phi=phi.cpu().numpy(), F=F.cpu().numpy(), W=Wv.cpu().numpy(),
                dpos=gp.cpu().numpy(), dq=gq.cpu().numpy())


@pytest.mark.parametrize("make", [lambda: W.random_box(8000, seed=73),
                                  lambda: W.random_box(3000, seed=76, p=6, h=1.5, a=6.0)], ids=["p4_device", "p6_host"])
def test_spectral_dynamic_cell(make):
    """Cell changes on a plan running the spectral method: periodic p = 4 plans recompute the spectra on
    the device from the raw samples (separable sums, FP32), others on the host (FP64)."""
    import oracle as O
    w = make()
    M = [O.plan_for(w).M[d] for d in range(3)]
    base = np.array(w.cell, np.float64)
    # built for the most compressed cell it will serve (the plan keeps its stencil sizes)
    plan = Plan(tuple(base * 0.97), w.pbc, w.h, w.a, w.p, w.levels, tuple(M), max_atoms=w.n, device=DEV)
    plan.set_level_method(LEVELS_SPECTRAL)
    for f in ((1.0, 1.0, 1.0), (1.04, 0.99, 1.02), (0.97, 0.97, 0.97)):
        cell = base * np.array(f)
        pos = (w.pos.astype(np.float64) * np.array(f)).astype(np.float32)
        plan.set_cell(cell)
        check_oracle(_run_cell(plan, pos, w.q), _oracle_for(cell, w, M, pos))
    # a cell change under the ball method, then the switch: the spectra followed the cell
    plan.set_level_method(LEVELS_BALL)
    cell = base * 1.03
    pos = (w.pos.astype(np.float64) * 1.03).astype(np.float32)
    plan.set_cell(cell)
    plan.set_level_method(LEVELS_SPECTRAL)
    check_oracle(_run_cell(plan, pos, w.q), _oracle_for(cell, w, M, pos))


def test_autotune_picks_a_level_method():
    w = W.random_box(20001, seed=62)
    P, ref = oracle(w)
    plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, max_atoms=w.n, device=DEV)
    pos, q = torch.from_numpy(w.pos).to(DEV), torch.from_numpy(w.q).to(DEV)
    choice = plan.autotune(pos, q)
    assert choice["level_method"] in (LEVELS_BALL, LEVELS_SPECTRAL)
    r = run(w, None, plan=plan)
    check_oracle(r, ref)


def test_plans_without_the_spectral_method_refuse():
    for w in (W.random_box(3000, seed=33, pbc=(1, 1, 0)), W.open_cluster(), W.random_box(2000, seed=46, pbc=(0, 0, 1))):
        plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, w.levels, w.grid_override, max_atoms=w.n, device=DEV)
        assert not plan.info()["spectral_ok"]
        with pytest.raises(Exception):
            plan.set_level_method(LEVELS_SPECTRAL)
        assert plan.info()["level_method"] == LEVELS_BALL
    A = np.array([[30.0, 0, 0], [6.0, 30.0, 0], [0, 0, 30.0]])
    tilted = Plan(A.reshape(9), (1, 1, 1), 0.0, 6.0, 4, 0, (16, 16, 16), max_atoms=100, device=DEV)
    with pytest.raises(Exception):
        tilted.set_level_method(LEVELS_SPECTRAL)
    batch = Batch([W.random_box(500, seed=74), W.random_box(700, seed=75)], device=DEV)
    assert batch is not None  # batches keep the ball and box kernels (no level-method call)


def test_spectral_vjps_field_and_end_to_end_match_ball_method():
    """The calls that run the grid chain again (msm_force_vjp, msm_potential_vjp) or
    end to end (msm_evaluate_host), and msm_field, on a spectral plan agree with the
    ball method's to FP32 rounding."""
    w = CASES["periodic_20001"]()
    pos = torch.from_numpy(w.pos).to(DEV)
    q = torch.from_numpy(w.q).to(DEV)
    rng = np.random.default_rng(77)
    u = torch.from_numpy(rng.normal(size=(w.n, 3)).astype(np.float32)).to(DEV)
    g = torch.from_numpy(rng.normal(size=w.n).astype(np.float32)).to(DEV)
    out = {}
    for m in (LEVELS_BALL, LEVELS_SPECTRAL):
        plan = make_plan(w, m)
        plan.forward(pos, q, forces=True, virial=True)
        fld = plan.field().cpu().numpy()
        fq, fp = plan.force_vjp(u)
        plan.forward(pos, q, forces=True, virial=True)
        pq, pp = plan.potential_vjp(g)
        torch.cuda.synchronize()
        host = plan.evaluate_host(torch.from_numpy(w.pos), torch.from_numpy(w.q))
        out[m] = dict(field=fld, fq=fq.cpu().numpy(), fp=fp.cpu().numpy(), pq=pq.cpu().numpy(),
                      pp=pp.cpu().numpy(), host=host)
    b, s = out[LEVELS_BALL], out[LEVELS_SPECTRAL]
    for key in ("field", "fq", "fp", "pq", "pp"):
        assert rel_rms(s[key], b[key]) <= AGREE, key
    hb, hs = b["host"], s["host"]
    assert abs(float(hs[0]) - float(hb[0])) <= AGREE * abs(float(hb[0]))
    for i in (1, 2):
        assert rel_rms(np.asarray(hs[i]), np.asarray(hb[i])) <= AGREE, i
    assert np.abs(np.asarray(hs[3]) - np.asarray(hb[3])).max() <= AGREE * np.abs(np.asarray(hb[3])).max()


def test_spectral_plan_in_a_cuda_graph():
    """Forward (forces, virial) and backward of a spectral plan captured in a CUDA graph
    and replayed twice with a new input set copied into the captured buffers: every
    replay against the oracle on its inputs."""
    import oracle as O
    w = CASES["periodic_20001"]()
    plan = make_plan(w, LEVELS_SPECTRAL)
    pos = torch.from_numpy(w.pos).to(DEV)
    q = torch.from_numpy(w.q).to(DEV)
    gE = torch.ones(1, dtype=torch.float64, device=DEV)
    side = torch.cuda.Stream(DEV)
    side.wait_stream(torch.cuda.current_stream(DEV))
    with torch.cuda.stream(side):
        for _ in range(2):
            plan.forward(pos, q, forces=True, virial=True)
            plan.backward(gE)
    torch.cuda.current_stream(DEV).wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        E, phi, F = plan.forward(pos, q, forces=True, virial=True)
        gp, gq, Wv = plan.backward(gE)
    for seed in (81, 82):
        w2 = W.redraw(w, seed)
        pos.copy_(torch.from_numpy(w2.pos))
        q.copy_(torch.from_numpy(w2.q))
        graph.replay()
        torch.cuda.synchronize()
        ref = O.msm(O.plan_for(w2), w2.pos.astype(np.float64), w2.q.astype(np.float64), forces=True, virial=True)
        r = dict(E=float(E.cpu()[0]), phi=phi.cpu().numpy(), F=F.cpu().numpy(), W=Wv.cpu().numpy(),
                 dpos=gp.cpu().numpy(), dq=gq.cpu().numpy())
        check_oracle(r, ref)
