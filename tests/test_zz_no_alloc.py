"""msm_forward_noalloc: the forward pass for callers that cannot allocate
device memory (their host application owns all of it, or they run where an
allocation is not allowed). It keeps its workspace in a fixed device array
inside the library instead of a caller-allocated one.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test. It checks the no-alloc forward,
called twice in a row through the C ABI, against msm_forward with a
caller-allocated workspace, within the tolerances of the other parity tests,
and that a plan too large for the fixed array is refused with a clear error.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2510_05961_gb300 import Plan, _lib, build  # noqa: E402
from paper_2510_05961_gb300 import workloads as W  # noqa: E402

E_TOL = 1e-5
F_TOL = 1e-4
DEV = torch.device("cuda", 0)


def _vp(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _rel_rms(a, b):
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    return float(np.sqrt(((a - b) ** 2).sum(1).mean() / (b ** 2).sum(1).mean()))


@pytest.mark.parametrize("w", [W.random_box(20001, seed=51), W.open_cluster(n=1000, seed=52)],
                         ids=["periodic", "open"])
def test_noalloc_forward_matches_forward(w):
    build.build()
    lib = _lib.load()
    plan = Plan(w.cell, w.pbc, w.h, w.a, w.p, w.levels, max_atoms=w.n, device=DEV)
    pos = torch.from_numpy(w.pos).to(DEV)
    q = torch.from_numpy(w.q).to(DEV)
    E_ref, phi_ref, F_ref = plan.forward(pos, q, forces=True, virial=False)
    E_ref, phi_ref, F_ref = E_ref.item(), phi_ref.cpu().numpy(), F_ref.cpu().numpy()
    stream = C.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
    for _ in range(2):  # two calls in a row share (and reuse) the fixed array
        E = torch.empty(1, dtype=torch.float64, device=DEV)
        phi = torch.empty(w.n, dtype=torch.float32, device=DEV)
        F = torch.empty((w.n, 3), dtype=torch.float32, device=DEV)
        rc = lib.msm_forward_noalloc(plan.handle, w.n, _vp(pos), _vp(q), _vp(E), _vp(phi), _vp(F),
                                     _lib.MSM_WANT_FORCES, stream)
        assert rc == 0, lib.msm_last_error()
        torch.cuda.synchronize()
        assert abs(E.item() - E_ref) <= E_TOL * abs(E_ref)
        assert _rel_rms(phi.cpu().numpy(), phi_ref) <= F_TOL
        assert _rel_rms(F.cpu().numpy(), F_ref) <= F_TOL


def test_noalloc_rejects_plans_beyond_the_fixed_array():
    build.build()
    lib = _lib.load()
    n = 1_024_000  # its workspace is far above the fixed array
    plan = Plan(((n / 0.1) ** (1 / 3),) * 3, (1, 1, 1), 2.0, 8.0, 4, max_atoms=n, device=DEV)
    E = torch.empty(1, dtype=torch.float64, device=DEV)
    rc = lib.msm_forward_noalloc(plan.handle, 0, None, None, _vp(E), None, None, 0,
                                 C.c_void_p(torch.cuda.current_stream(DEV).cuda_stream))
    assert rc == _lib.MSM_ERR_CAPACITY
    assert b"fixed scratch" in lib.msm_last_error()
