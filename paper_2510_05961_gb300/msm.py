"""Python front end of the GB300 MSM library.

PyTorch provides device memory and streams; every step of the method runs in
the library's CUDA kernels, called through the C ABI. ``MSMFunction`` is the
autograd wrapper: its backward reuses the sorted bins, level grids and
per-atom results the forward left in the plan's workspace (the hand-written
adjoint of Sec. 3.2.2, Eqs. analytic_uoneplus_position_grad /
analytic_uoneplus_charge_grad) and also yields the virial.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

import torch

from . import _lib as L


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(device):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


# short_block code of the cluster-pair short-range kernel (MSM_SHORT_CLUSTER in msm_gb300.h)
SHORT_CLUSTER = 4
# level methods (MSM_LEVELS_* in msm_gb300.h): ball stencils, or products with the stencil
# spectra between FFTs of the level grids (fully periodic single-system plans)
LEVELS_BALL = 0
LEVELS_SPECTRAL = 1

class Plan:
    """One system: cell, periodicity, level-one spacing h, cutoff a, order p, levels.

    Holds the library plan (device stencil tables) and a workspace tensor
    sized for ``max_atoms``. Not thread-safe; one forward/backward at a time.
    """

    def __init__(self, cell, pbc, h, cutoff, order=4, levels=0, grid_override=(0, 0, 0), max_atoms=1,
                 device=None, qi_mode=0):
        self.lib = L.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.params = L.make_params(cell, pbc, h, cutoff, order, levels, grid_override, max_atoms, qi_mode)
            h_ = C.c_void_p()
            L.check(self.lib.msm_plan_create(C.byref(self.params), C.byref(h_)))
            self.handle = h_
            nb = C.c_size_t()
            L.check(self.lib.msm_workspace_bytes(self.handle, C.byref(nb)))
            self.workspace = torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=self.device)
        self.max_atoms = int(max_atoms)
        self.last_virial = None
        self._n = None

    def __del__(self):
        try:
            if getattr(self, "handle", None) is not None and self.lib is not None:
                self.lib.msm_plan_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    # ------------------------------------------------------------------ info
    def info(self):
        I = L.PlanInfo()
        L.check(self.lib.msm_plan_get_info(self.handle, C.byref(I)))
        return {
            "nlev": I.nlev, "ncomp": I.ncomp, "M": list(I.M), "h1": list(I.h1),
            "lo": [list(I.lo[l]) for l in range(I.ncomp)], "n": [list(I.n[l]) for l in range(I.ncomp)],
            "R": list(I.R), "C": list(I.C), "nnbr": list(I.nnbr),
            "stencil_kind": [I.stencil_kind[l] for l in range(I.ncomp)],
            "anterp_tz": I.anterp_tz, "short_block": I.short_block, "anterp_kind": I.anterp_kind,
            "level_method": I.level_method, "spectral_ok": bool(I.spectral_ok),
        }

    def debug_array(self, which, level=1):
        """View of an internal workspace array (0 cell_start, 1 perm, 2 grid charge, 3 grid potential, 4 sorted cell)."""
        off = C.c_size_t()
        cnt = C.c_size_t()
        L.check(self.lib.msm_debug_offset(self.handle, which, level, C.byref(off), C.byref(cnt)))
        dt = torch.float32 if which in (2, 3) else torch.int32
        nbytes = int(cnt.value) * 4
        return self.workspace[int(off.value):int(off.value) + nbytes].view(dt)

    # ------------------------------------------------------------------ calls
    def forward(self, pos, q, forces=True, virial=False, phi=True):
        """Energy (float64, shape (1,)), potentials (n,) and forces (n, 3) of float32 device inputs."""
        n = int(pos.shape[0])
        assert pos.dtype == torch.float32 and q.dtype == torch.float32 and pos.is_contiguous() and q.is_contiguous()
        assert pos.device == self.device and q.device == self.device
        E = torch.empty(1, dtype=torch.float64, device=self.device)
        ph = torch.empty(n, dtype=torch.float32, device=self.device) if phi else None
        F = torch.empty((n, 3), dtype=torch.float32, device=self.device) if forces else None
        flags = (L.MSM_WANT_FORCES if forces else 0) | (L.MSM_WANT_VIRIAL if virial else 0)
        L.check(self.lib.msm_forward(self.handle, _ptr(self.workspace), self.workspace.numel(), n, _ptr(pos), _ptr(q),
                                     _ptr(E), _ptr(ph), _ptr(F), flags, _stream(self.device)))
        self._n = n
        return E, ph, F

    def backward(self, grad_E, dpos=True, dq=True, virial=True):
        """dE/dpos, dE/dq (scaled by grad_E) and the virial (3x3 float64) from the last forward."""
        n = self._n
        g = grad_E.to(device=self.device, dtype=torch.float64).reshape(1).contiguous()
        gp = torch.empty((n, 3), dtype=torch.float32, device=self.device) if dpos else None
        gq = torch.empty(n, dtype=torch.float32, device=self.device) if dq else None
        W = torch.empty(9, dtype=torch.float64, device=self.device) if virial else None
        L.check(self.lib.msm_backward(self.handle, _ptr(self.workspace), _ptr(g), _ptr(gp), _ptr(gq), _ptr(W),
                                      _stream(self.device)))
        if W is not None:
            W = W.view(3, 3)
            self.last_virial = W
        return gp, gq, W

    def set_cell(self, cell):
        """New orthorhombic cell (3 lengths or a 3x3 / 9-entry matrix) for this periodic p = 4 plan: the
        stencils are recomputed on the device; grid counts and stencil sizes stay (see msm_plan_set_cell)."""
        c = np.asarray(cell, dtype=np.float64)
        c = np.diag(c) if c.shape == (3,) else c.reshape(3, 3)
        arr = (C.c_double * 9)(*[float(v) for v in c.reshape(9)])
        L.check(self.lib.msm_plan_set_cell(self.handle, arr, _stream(self.device)))

    def field(self, out=None):
        """Field -grad phi (n, 3) float32 at every atom from the last forward (forces = q * field)."""
        n = self._n
        fld = out if out is not None else torch.empty((n, 3), dtype=torch.float32, device=self.device)
        L.check(self.lib.msm_field(self.handle, _ptr(self.workspace), _ptr(fld), _stream(self.device)))
        return fld

    def force_vjp(self, u, dq=True, dpos=True):
        """(dL/dq, dL/dpos) for L = sum_k u_k . F_k of the last forward (u: (n, 3) float32 device).
        Consumes the workspace: a later backward needs a new forward."""
        n = self._n
        u = u.detach().to(device=self.device, dtype=torch.float32).contiguous()
        gq = torch.empty(n, dtype=torch.float32, device=self.device) if dq else None
        gp = torch.empty((n, 3), dtype=torch.float32, device=self.device) if dpos else None
        L.check(self.lib.msm_force_vjp(self.handle, _ptr(self.workspace), _ptr(u), _ptr(gq), _ptr(gp),
                                       _stream(self.device)))
        return gq, gp

    def potential_vjp(self, g, dq=True, dpos=True):
        """(dL/dq, dL/dpos) for L = sum_k g_k phi_k of the last forward (g: (n,) float32 device):
        dL/dq = A g, dL/dr = -g E(q) - q E(g), computed by the library (msm_potential_vjp).
        Consumes the workspace: a later backward needs a new forward."""
        n = self._n
        g = g.detach().to(device=self.device, dtype=torch.float32).contiguous()
        gq = torch.empty(n, dtype=torch.float32, device=self.device) if dq else None
        gp = torch.empty((n, 3), dtype=torch.float32, device=self.device) if dpos else None
        L.check(self.lib.msm_potential_vjp(self.handle, _ptr(self.workspace), _ptr(g), _ptr(gq), _ptr(gp),
                                           _stream(self.device)))
        return gq, gp

    def autotune(self, pos, q):
        """Time the tunable launch shapes on these inputs and keep the fastest; returns them.
        A new forward is needed before the next backward."""
        n = int(pos.shape[0])
        assert pos.dtype == torch.float32 and q.dtype == torch.float32 and pos.is_contiguous() and q.is_contiguous()
        L.check(self.lib.msm_autotune(self.handle, _ptr(self.workspace), self.workspace.numel(), n, _ptr(pos), _ptr(q),
                                      _stream(self.device)))
        info = self.info()
        return {"anterp_tz": info["anterp_tz"], "short_block": info["short_block"], "level_method": info["level_method"]}

    def set_tuning(self, anterp_tz=32, short_block=256):
        """anterp_tz in (16, 32, 64); short_block 128 or 256 (per-atom kernel) or SHORT_CLUSTER."""
        L.check(self.lib.msm_set_tuning(self.handle, int(anterp_tz), int(short_block)))

    def set_level_method(self, method):
        """LEVELS_BALL or LEVELS_SPECTRAL (plans with info()["spectral_ok"]); a new forward is
        needed before the next backward."""
        L.check(self.lib.msm_set_level_method(self.handle, int(method)))

    def status(self):
        st = C.c_int()
        L.check(self.lib.msm_status(self.handle, _ptr(self.workspace), _stream(self.device), C.byref(st)))
        return st.value

    def evaluate_host(self, pos, q, virial=True, pinned_out=None):
        """End-to-end call on host tensors (msm_evaluate_host): the library copies the
        inputs in, runs forward + backward and copies E, dE/dpos, dE/dq and the virial
        out, then returns. pos (n, 3) and q (n,) are float32 CPU tensors (pinned for
        asynchronous copies); pinned_out optionally gives the four host outputs."""
        n = int(pos.shape[0])
        assert pos.dtype == torch.float32 and q.dtype == torch.float32 and pos.is_contiguous() and q.is_contiguous()
        if pinned_out is None:
            pinned_out = (torch.empty(1, dtype=torch.float64, pin_memory=True),
                          torch.empty((n, 3), dtype=torch.float32, pin_memory=True),
                          torch.empty(n, dtype=torch.float32, pin_memory=True),
                          torch.empty((3, 3), dtype=torch.float64, pin_memory=True))
        oE, op, oq, oW = pinned_out
        L.check(self.lib.msm_evaluate_host(self.handle, _ptr(self.workspace), self.workspace.numel(), n, _ptr(pos),
                                           _ptr(q), _ptr(oE), _ptr(op), _ptr(oq), _ptr(oW) if virial else None,
                                           _stream(self.device)))
        self._n = n
        return oE, op, oq, oW

    def profile(self, enable=True, serial=False):
        """Record CUDA-event times per phase of every forward/backward; serial=True runs
        every phase on the caller's stream (no overlap), so each phase time is its own."""
        L.check(self.lib.msm_profile(self.handle, (2 if serial else 1) if enable else 0))

    def profile_read(self):
        """(dict phase -> ms of the last forward + backward, kernels launched by them)."""
        ms = (C.c_double * len(L.PHASES))()
        nl = C.c_int()
        L.check(self.lib.msm_profile_read(self.handle, ms, C.byref(nl)))
        return {p: ms[i] for i, p in enumerate(L.PHASES)}, nl.value


class MSMFunction(torch.autograd.Function):
    """(E, phi, F) of (pos, q) through the library.

    Backward takes upstream gradients on E, phi and F, each through a library call:
      E:   msm_backward (the adjoint kernels): dE/dpos = -F, dE/dq = phi; plan.last_virial
           holds W * dL/dE.
      phi: msm_potential_vjp: phi = A q with A symmetric, so for L = sum_i g_i phi_i
           dL/dq = A g and dL/dr_k = -g_k E_k(q) - q_k E_k(g), one more evaluation with
           charges g on the same sorted positions.
      F:   msm_force_vjp (dipole potential and Hessian-vector products).
    The plan's workspace is reused: backward must follow its own forward. The two VJPs
    consume the workspace, so when both upstreams are given the forward is run again
    between them."""

    @staticmethod
    def forward(ctx, pos, q, plan):
        ctx.set_materialize_grads(False)
        pos_d, q_d = pos.detach().contiguous(), q.detach().contiguous()
        E, phi, F = plan.forward(pos_d, q_d, forces=True, virial=True, phi=True)
        ctx.plan = plan
        ctx.need = (pos.requires_grad, q.requires_grad)
        ctx.save_for_backward(pos_d, q_d)
        return E.reshape(()), phi, F

    @staticmethod
    def backward(ctx, gE, gphi, gF):
        use_phi = gphi is not None and bool((gphi != 0).any())
        use_F = gF is not None and bool((gF != 0).any())
        if gE is None and not use_phi and not use_F:
            return None, None, None
        plan = ctx.plan
        gp = gq = None

        def acc(a, b):
            return b if a is None else (a if b is None else a + b)

        if gE is not None:
            gp, gq, _ = plan.backward(gE, dpos=ctx.need[0], dq=ctx.need[1], virial=True)
        if use_phi:
            pq, pp = plan.potential_vjp(gphi, dq=ctx.need[1], dpos=ctx.need[0])
            gq, gp = acc(gq, pq), acc(gp, pp)
        if use_F:
            if use_phi:  # the potential VJP consumed the workspace
                pos, q = ctx.saved_tensors
                plan.forward(pos, q, forces=True, virial=False, phi=False)
            fq, fp = plan.force_vjp(gF, dq=ctx.need[1], dpos=ctx.need[0])
            gq, gp = acc(gq, fq), acc(gp, fp)
        return gp, gq, None


def msm_energy(pos, q, plan):
    """Differentiable MSM energy (autograd through the library's adjoint kernels)."""
    return MSMFunction.apply(pos, q, plan)[0]


def msm_outputs(pos, q, plan):
    """(E, phi, F); E and phi are differentiable, F is not (its upstream must be zero)."""
    return MSMFunction.apply(pos, q, plan)


class Batch:
    """Many independent systems in one set of launches (one launch per MSM phase).

    systems: list of dicts/objects with cell, pbc, h, a (cutoff), p (order), levels, n.
    Atoms are packed back to back in system order.
    """

    def __init__(self, systems, device=None):
        self.lib = L.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        ns = len(systems)
        arr = (L.Params * ns)()
        counts = (C.c_int * ns)()
        self.counts = []
        for i, s in enumerate(systems):
            arr[i] = L.make_params(s.cell, s.pbc, s.h, s.a, s.p, getattr(s, "levels", 0),
                                   getattr(s, "grid_override", (0, 0, 0)), 0, getattr(s, "qi_mode", 0))
            counts[i] = int(s.n)
            self.counts.append(int(s.n))
        with torch.cuda.device(self.device):
            h_ = C.c_void_p()
            L.check(self.lib.msm_batch_create(arr, counts, ns, C.byref(h_)))
            self.handle = h_
            nb = C.c_size_t()
            L.check(self.lib.msm_batch_workspace_bytes(self.handle, C.byref(nb)))
            self.workspace = torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=self.device)
        self.nsys = ns
        self.ntot = sum(self.counts)

    def __del__(self):
        try:
            if getattr(self, "handle", None) is not None and self.lib is not None:
                self.lib.msm_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    def forward(self, pos, q, forces=True, virial=False, phi=True, out=None):
        n = self.ntot
        if out is None:
            E = torch.empty(self.nsys, dtype=torch.float64, device=self.device)
            ph = torch.empty(n, dtype=torch.float32, device=self.device) if phi else None
            F = torch.empty((n, 3), dtype=torch.float32, device=self.device) if forces else None
        else:
            E, ph, F = out
        flags = (L.MSM_WANT_FORCES if forces else 0) | (L.MSM_WANT_VIRIAL if virial else 0)
        L.check(self.lib.msm_batch_forward(self.handle, _ptr(self.workspace), self.workspace.numel(), _ptr(pos),
                                           _ptr(q), _ptr(E), _ptr(ph), _ptr(F), flags, _stream(self.device)))
        return E, ph, F

    def backward(self, grad_E, dpos=True, dq=True, virial=True, out=None):
        n = self.ntot
        g = grad_E.to(device=self.device, dtype=torch.float64).reshape(self.nsys).contiguous()
        if out is None:
            gp = torch.empty((n, 3), dtype=torch.float32, device=self.device) if dpos else None
            gq = torch.empty(n, dtype=torch.float32, device=self.device) if dq else None
            W = torch.empty(9 * self.nsys, dtype=torch.float64, device=self.device) if virial else None
        else:
            gp, gq, W = out
        L.check(self.lib.msm_batch_backward(self.handle, _ptr(self.workspace), _ptr(g), _ptr(gp), _ptr(gq), _ptr(W),
                                            _stream(self.device)))
        return gp, gq, (None if W is None else W.view(self.nsys, 3, 3))

    def potential_vjp(self, g, dq=True, dpos=True):
        """Plan.potential_vjp for the packed atoms of all systems."""
        g = g.detach().to(device=self.device, dtype=torch.float32).contiguous()
        gq = torch.empty(self.ntot, dtype=torch.float32, device=self.device) if dq else None
        gp = torch.empty((self.ntot, 3), dtype=torch.float32, device=self.device) if dpos else None
        L.check(self.lib.msm_batch_potential_vjp(self.handle, _ptr(self.workspace), _ptr(g), _ptr(gq), _ptr(gp),
                                                 _stream(self.device)))
        return gq, gp

    def force_vjp(self, u, dq=True, dpos=True):
        """Plan.force_vjp for the packed atoms of all systems."""
        u = u.detach().to(device=self.device, dtype=torch.float32).contiguous()
        gq = torch.empty(self.ntot, dtype=torch.float32, device=self.device) if dq else None
        gp = torch.empty((self.ntot, 3), dtype=torch.float32, device=self.device) if dpos else None
        L.check(self.lib.msm_batch_force_vjp(self.handle, _ptr(self.workspace), _ptr(u), _ptr(gq), _ptr(gp),
                                             _stream(self.device)))
        return gq, gp

    def field(self, out=None):
        """Field -grad phi ((sum n), 3) float32 at every atom of every system from the last forward."""
        fld = out if out is not None else torch.empty((self.ntot, 3), dtype=torch.float32, device=self.device)
        L.check(self.lib.msm_batch_field(self.handle, _ptr(self.workspace), _ptr(fld), _stream(self.device)))
        return fld

    def set_tuning(self, anterp_tz=32, short_block=256):
        """anterp_tz in (16, 32, 64); short_block 128 or 256 (per-atom kernel) or SHORT_CLUSTER."""
        L.check(self.lib.msm_batch_set_tuning(self.handle, int(anterp_tz), int(short_block)))

    def autotune(self, pos, q):
        """Time the tunable launch shapes on this batch's inputs and keep the fastest; returns them.
        A new forward is needed before the next backward; call it before capturing a graph."""
        L.check(self.lib.msm_batch_autotune(self.handle, _ptr(self.workspace), self.workspace.numel(), _ptr(pos), _ptr(q),
                                            _stream(self.device)))
        tz, nb = C.c_int(), C.c_int()
        L.check(self.lib.msm_batch_get_tuning(self.handle, C.byref(tz), C.byref(nb)))
        return {"anterp_tz": tz.value, "short_block": nb.value}

    def status(self):
        st = C.c_int()
        L.check(self.lib.msm_batch_status(self.handle, _ptr(self.workspace), _stream(self.device), C.byref(st)))
        return st.value
