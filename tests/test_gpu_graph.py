"""The batched forward + backward as the benchmark times it: captured once in a
CUDA graph and replayed.

The 512-system batch (log-uniform 20-4000 atoms, open / slab / periodic;
batched evaluation of independent systems, Sec. 4.1) is captured the way the
benchmark captures it (launch shapes tuned first, warm-up on a side stream,
then one forward with forces and virial and one backward with dL/dE = 1 into
static output buffers). The graph is replayed twice; before each replay a
different seeded input set of the same shapes is copied into the captured
position and charge buffers. After each replay every system's E, phi, F,
dE/dq, dE/dr and W is compared with the FP64 oracle on that replay's inputs:
this covers the reuse of the static buffers across replays, the fork/join of
the library's second stream inside the capture and the workspace state left
by the previous replay. Tolerances as in the other parity tests (relative
energy 1e-5 with the FP32 rounding floor 1e-7 sum |q phi| / 2 for energies
that cancel, relative RMS 1e-4 for per-atom outputs, 1e-4 of the largest
virial entry).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05961_gb300 import Batch, build  # noqa: E402
from paper_2510_05961_gb300 import workloads as W  # noqa: E402
from msm_testutil import expected_status  # noqa: E402

E_TOL = 1e-5
F_TOL = 1e-4
DEV = torch.device("cuda", 0)


def rel_rms(a, b):
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    return float(np.sqrt(((a - b) ** 2).sum(1).mean() / max((b ** 2).sum(1).mean(), 1e-300)))


def check_against_oracle(systems, E, phi, F, gp, gq, Wb):
    import oracle as O
    off = 0
    for s, w in enumerate(systems):
        n = w.n
        ref = O.msm(O.plan_for(w), w.pos.astype(np.float64), w.q.astype(np.float64), forces=True, virial=True)
        floor = 1e-7 * 0.5 * float(np.abs(w.q.astype(np.float64) * ref["phi"]).sum())
        assert abs(E[s] - ref["E"]) <= E_TOL * abs(ref["E"]) + floor, (s, E[s], ref["E"])
        assert rel_rms(phi[off:off + n], ref["phi"]) <= F_TOL, s
        assert rel_rms(F[off:off + n], ref["F"]) <= F_TOL, s
        assert rel_rms(gq[off:off + n], ref["phi"]) <= F_TOL, s
        assert rel_rms(gp[off:off + n], -ref["F"]) <= F_TOL, s
        assert np.abs(Wb[s] - ref["W"]).max() <= F_TOL * np.abs(ref["W"]).max(), s
        off += n


def test_graph_replays_match_oracle():
    build.build()
    import oracle as O
    O.build()
    systems = W.batch_systems()
    nsys = len(systems)
    ntot = sum(s.n for s in systems)
    batch = Batch(systems, device=DEV)
    pos = torch.from_numpy(np.concatenate([s.pos for s in systems])).to(DEV)
    q = torch.from_numpy(np.concatenate([s.q for s in systems])).to(DEV)
    g = torch.ones(nsys, dtype=torch.float64, device=DEV)
    out_f = (torch.empty(nsys, dtype=torch.float64, device=DEV), torch.empty(ntot, dtype=torch.float32, device=DEV),
             torch.empty((ntot, 3), dtype=torch.float32, device=DEV))
    out_b = (torch.empty((ntot, 3), dtype=torch.float32, device=DEV),
             torch.empty(ntot, dtype=torch.float32, device=DEV),
             torch.empty(9 * nsys, dtype=torch.float64, device=DEV))

    def step():
        batch.forward(pos, q, forces=True, virial=True, phi=True, out=out_f)
        batch.backward(g, out=out_b)

    batch.autotune(pos, q)
    side = torch.cuda.Stream(DEV)
    side.wait_stream(torch.cuda.current_stream(DEV))
    with torch.cuda.stream(side):
        for _ in range(3):
            step()
    torch.cuda.current_stream(DEV).wait_stream(side)
    torch.cuda.synchronize(DEV)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        step()
    for seed in (7101, 7102):
        inputs = [W.redraw(w, seed * 1000 + s) for s, w in enumerate(systems)]
        pos.copy_(torch.from_numpy(np.concatenate([w.pos for w in inputs])))
        q.copy_(torch.from_numpy(np.concatenate([w.q for w in inputs])))
        graph.replay()
        torch.cuda.synchronize(DEV)
        assert batch.status() == expected_status(inputs)
        E, phi, F = (t.cpu().numpy() for t in out_f)
        gp, gq, Wb = (t.cpu().numpy() for t in out_b)
        check_against_oracle(inputs, E, phi, F, gp, gq, Wb.reshape(nsys, 3, 3))
