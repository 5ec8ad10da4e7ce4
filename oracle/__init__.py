"""ctypes front end of the FP64 MSM oracle (``msm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package; the product library never
imports it. It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
MAXLEV = 20
ST_OUTSIDE = 1
ST_NONFINITE = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Plan(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3), ("pbc", C.c_int * 3), ("h", C.c_double), ("grid_override", C.c_int * 3),
        ("a", C.c_double), ("p", C.c_int), ("levels", C.c_int), ("qi_mode", C.c_int),
        ("nlev", C.c_int), ("ncomp", C.c_int), ("top_kept", C.c_int),
        ("M", C.c_int * 3), ("h1", C.c_double * 3),
        ("lo", (C.c_int * 3) * MAXLEV), ("n", (C.c_int * 3) * MAXLEV),
        ("S", C.c_int * 3), ("R", C.c_int * 3), ("hw", C.c_int),
        ("C", C.c_int * 3), ("edge", C.c_double * 3), ("nnbr", C.c_int * 3),
        ("invLf", C.c_float * 3),
        ("A", C.c_double * 9), ("tri", C.c_int), ("Ainv", C.c_double * 9), ("Tinv", C.c_double * 9),
        ("Tf", C.c_float * 9), ("wplane", C.c_double * 3),
    ]

    def level_shape(self, l):
        return tuple(self.n[l - 1][d] for d in range(3))

    def level_lo(self, l):
        return tuple(self.lo[l - 1][d] for d in range(3))


_lib = None
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.or_gamma.restype = C.c_double
        L.or_gamma.argtypes = [C.c_int, C.c_double]
        L.or_dgamma.restype = C.c_double
        L.or_dgamma.argtypes = [C.c_int, C.c_double]
        L.or_kl.restype = C.c_double
        L.or_kl.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, C.c_double]
        L.or_dkl.restype = C.c_double
        L.or_dkl.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, C.c_double]
        L.or_bspline.restype = C.c_double
        L.or_bspline.argtypes = [C.c_int, C.c_double]
        L.or_dbspline.restype = C.c_double
        L.or_dbspline.argtypes = [C.c_int, C.c_double]
        L.or_J.argtypes = [C.c_int, _dp]
        L.or_omega.restype = C.c_int
        L.or_omega.argtypes = [C.c_int, _dp]
        L.or_omega_exact.restype = C.c_int
        L.or_omega_exact.argtypes = [C.c_int, _dp, C.c_int]
        L.or_plan_init.restype = C.c_int
        L.or_plan_init.argtypes = [C.POINTER(Plan)]
        L.or_bin.restype = C.c_int
        L.or_bin.argtypes = [C.POINTER(Plan), C.c_int, _fp, _fp, _ip, _ip, _ip]
        L.or_anterp.argtypes = [C.POINTER(Plan), C.c_int, _dp, _dp, _dp]
        L.or_interp.argtypes = [C.POINTER(Plan), C.c_int, _dp, _dp, _dp, _dp, _dp]
        L.or_restrict.argtypes = [C.POINTER(Plan), C.c_int, _dp, _dp]
        L.or_prolong_add.argtypes = [C.POINTER(Plan), C.c_int, _dp, _dp]
        L.or_stencil_box.argtypes = [C.POINTER(Plan), C.c_int, _ip, _ip]
        L.or_stencil_build.argtypes = [C.POINTER(Plan), C.c_int, C.c_int, _dp, _dp]
        L.or_stencil_apply.argtypes = [C.POINTER(Plan), C.c_int, _dp, _dp, _dp]
        L.or_grid_virial_level.argtypes = [C.POINTER(Plan), C.c_int, _dp, _dp]
        L.or_short_range.argtypes = [C.POINTER(Plan), C.c_int, _dp, _dp, _dp, _dp, _dp]
        L.or_energy.restype = C.c_double
        L.or_energy.argtypes = [C.c_int, _dp, _dp]
        L.or_grid_pass.argtypes = [C.POINTER(Plan), _dp, _dp]
        L.or_grid_total.restype = C.c_size_t
        L.or_grid_total.argtypes = [C.POINTER(Plan)]
        L.or_msm.argtypes = [C.POINTER(Plan), C.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_direct_open.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp]
        L.or_direct_level.argtypes = [C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp]
        L.or_ewald.argtypes = [_dp, C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_double, _dp, _dp, _dp]
        _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


# --------------------------------------------------------------------------- scalars
def gamma(p, rho):
    return lib().or_gamma(p, float(rho))


def dgamma(p, rho):
    return lib().or_dgamma(p, float(rho))


def kl(p, a, nlev, l, r):
    return lib().or_kl(p, float(a), nlev, l, float(r))


def dkl(p, a, nlev, l, r):
    return lib().or_dkl(p, float(a), nlev, l, float(r))


def bspline(q, t):
    return lib().or_bspline(q, float(t))


def dbspline(q, t):
    return lib().or_dbspline(q, float(t))


def J(p):
    out = np.zeros(p + 1)
    lib().or_J(p, _ptr(out))
    return out


def omega(p):
    out = np.zeros(p - 1)
    rc = lib().or_omega(p, _ptr(out))
    assert rc == 0
    return out


def omega_exact(p, maxhw=96):
    """omega' of exact interpolation (qi_mode 1), indices -hw .. hw."""
    buf = np.zeros(2 * maxhw + 1)
    hw = lib().or_omega_exact(p, _ptr(buf), maxhw)
    assert hw >= 0
    return buf[:2 * hw + 1].copy()


# --------------------------------------------------------------------------- plan
def make_plan(cell, pbc, h, a, p, levels=0, grid_override=(0, 0, 0), qi_mode=0):
    """cell: 3 edge lengths, or a 3x3 / 9-entry matrix whose rows are the cell vectors."""
    P = Plan()
    cm = np.asarray(cell, np.float64)
    if cm.size == 9:
        for k in range(9):
            P.A[k] = float(cm.reshape(9)[k])
        cell = [float(np.linalg.norm(cm.reshape(3, 3)[d])) for d in range(3)]
    for d in range(3):
        P.L[d] = float(cell[d])
        P.pbc[d] = int(pbc[d])
        P.grid_override[d] = int(grid_override[d])
    P.h = float(h)
    P.a = float(a)
    P.p = int(p)
    P.levels = int(levels)
    P.qi_mode = int(qi_mode)
    rc = lib().or_plan_init(C.byref(P))
    if rc != 0:
        raise ValueError("oracle plan rejected the parameters (code %d)" % rc)
    return P


def plan_for(w):
    return make_plan(w.cell, w.pbc, w.h, w.a, w.p, w.levels, w.grid_override, getattr(w, "qi_mode", 0))


def plan_summary(P):
    """Plain dict of the derived plan fields (for comparisons)."""
    return {
        "nlev": P.nlev, "ncomp": P.ncomp, "top_kept": P.top_kept,
        "M": [P.M[d] for d in range(3)], "h1": [P.h1[d] for d in range(3)],
        "lo": [[P.lo[l][d] for d in range(3)] for l in range(P.ncomp)],
        "n": [[P.n[l][d] for d in range(3)] for l in range(P.ncomp)],
        "S": [P.S[d] for d in range(3)], "R": [P.R[d] for d in range(3)], "hw": P.hw,
        "C": [P.C[d] for d in range(3)], "edge": [P.edge[d] for d in range(3)],
        "nnbr": [P.nnbr[d] for d in range(3)],
    }


# --------------------------------------------------------------------------- steps
def bin_atoms(P, pos32, q32):
    pos32 = np.ascontiguousarray(pos32, dtype=np.float32)
    q32 = np.ascontiguousarray(q32, dtype=np.float32)
    n = pos32.shape[0]
    ncell = P.C[0] * P.C[1] * P.C[2]
    cid = np.zeros(n, np.int32)
    start = np.zeros(ncell + 1, np.int32)
    perm = np.zeros(n, np.int32)
    st = lib().or_bin(C.byref(P), n, _ptr(pos32, _fp), _ptr(q32, _fp), _ptr(cid, _ip), _ptr(start, _ip),
                      _ptr(perm, _ip))
    return cid, start, perm, st


def anterp(P, pos, q):
    pos, q = _d(pos), _d(q)
    g = np.zeros(P.level_shape(1))
    lib().or_anterp(C.byref(P), pos.shape[0], _ptr(pos), _ptr(q), _ptr(g))
    return g


def interp(P, pos, q, e1, forces=True):
    pos, q, e1 = _d(pos), _d(q), _d(e1)
    n = pos.shape[0]
    phi = np.zeros(n)
    F = np.zeros((n, 3)) if forces else None
    lib().or_interp(C.byref(P), n, _ptr(pos), _ptr(q), _ptr(e1), _ptr(phi), _ptr(F))
    return phi, F


def restrict(P, l, fine):
    out = np.zeros(P.level_shape(l + 1))
    lib().or_restrict(C.byref(P), l, _ptr(_d(fine)), _ptr(out))
    return out


def prolong_add(P, l, coarse, fine):
    fine = _d(fine).copy()
    lib().or_prolong_add(C.byref(P), l, _ptr(_d(coarse)), _ptr(fine))
    return fine


def stencil_box(P, l):
    lo = (C.c_int * 3)()
    sz = (C.c_int * 3)()
    lib().or_stencil_box(C.byref(P), l, lo, sz)
    return tuple(lo), tuple(sz)


def stencil(P, l, which=0, G=None):
    lo, sz = stencil_box(P, l)
    out = np.zeros(sz)
    Gp = None if G is None else _d(np.asarray(G).reshape(9))
    lib().or_stencil_build(C.byref(P), l, which, _ptr(Gp), _ptr(out))
    return out, lo


def stencil_apply(P, l, K, qg):
    out = np.zeros(P.level_shape(l))
    lib().or_stencil_apply(C.byref(P), l, _ptr(_d(K)), _ptr(_d(qg)), _ptr(out))
    return out


def grid_virial_level(P, l, qg):
    W6 = np.zeros(6)
    lib().or_grid_virial_level(C.byref(P), l, _ptr(_d(qg)), _ptr(W6))
    return W6


def short_range(P, pos, q, forces=True, virial=True):
    pos, q = _d(pos), _d(q)
    n = pos.shape[0]
    phi0 = np.zeros(n)
    F0 = np.zeros((n, 3)) if forces else None
    W0 = np.zeros(9) if virial else None
    lib().or_short_range(C.byref(P), n, _ptr(pos), _ptr(q), _ptr(phi0), _ptr(F0), _ptr(W0))
    return phi0, F0, (None if W0 is None else W0.reshape(3, 3))


def split_levels(P, flat):
    out, off = [], 0
    for l in range(1, P.ncomp + 1):
        sh = P.level_shape(l)
        sz = sh[0] * sh[1] * sh[2]
        out.append(flat[off:off + sz].reshape(sh))
        off += sz
    return out


def grid_pass(P, q1):
    tot = lib().or_grid_total(C.byref(P))
    ql = np.zeros(max(tot, 1))
    el = np.zeros(max(tot, 1))
    s = P.level_shape(1)
    ql[: s[0] * s[1] * s[2]] = _d(q1).reshape(-1)
    lib().or_grid_pass(C.byref(P), _ptr(ql), _ptr(el))
    return split_levels(P, ql), split_levels(P, el)


def msm(P, pos, q, forces=True, virial=True, grids=False):
    """Full MSM evaluation: returns dict(E, phi, F, W[, qlev, elev])."""
    pos, q = _d(pos), _d(q)
    n = pos.shape[0]
    E = np.zeros(1)
    phi = np.zeros(n)
    F = np.zeros((n, 3)) if forces else None
    W = np.zeros(9) if virial else None
    tot = lib().or_grid_total(C.byref(P))
    ql = np.zeros(max(tot, 1)) if grids else None
    el = np.zeros(max(tot, 1)) if grids else None
    lib().or_msm(C.byref(P), n, _ptr(pos), _ptr(q), _ptr(E), _ptr(phi), _ptr(F), _ptr(W), _ptr(ql), _ptr(el))
    out = {"E": float(E[0]), "phi": phi, "F": F, "W": None if W is None else W.reshape(3, 3)}
    if grids:
        out["qlev"] = split_levels(P, ql)
        out["elev"] = split_levels(P, el)
    return out


def direct_open(pos, q, forces=True):
    pos, q = _d(pos), _d(q)
    n = pos.shape[0]
    E = np.zeros(1)
    phi = np.zeros(n)
    F = np.zeros((n, 3)) if forces else None
    lib().or_direct_open(n, _ptr(pos), _ptr(q), _ptr(E), _ptr(phi), _ptr(F))
    return float(E[0]), phi, F


def direct_level(p, a, nlev, l, pos, q):
    pos, q = _d(pos), _d(q)
    n = pos.shape[0]
    E = np.zeros(1)
    phi = np.zeros(n)
    lib().or_direct_level(p, float(a), nlev, l, n, _ptr(pos), _ptr(q), _ptr(E), _ptr(phi))
    return float(E[0]), phi


def ewald(cell, pos, q, alpha, rcut, kmax, forces=True):
    pos, q = _d(pos), _d(q)
    L = _d(cell)
    n = pos.shape[0]
    E = np.zeros(1)
    phi = np.zeros(n)
    F = np.zeros((n, 3)) if forces else None
    lib().or_ewald(_ptr(L), n, _ptr(pos), _ptr(q), float(alpha), float(rcut), float(kmax), _ptr(E), _ptr(phi),
                   _ptr(F))
    return float(E[0]), phi, F


def ewald_tri(A, pos, q, alpha, rcut, kmax):
    """Ewald sum for a general periodic cell (rows of A are the cell vectors): (E, phi)."""
    pos, q = _d(pos), _d(q)
    A = _d(np.asarray(A, np.float64).reshape(9))
    n = pos.shape[0]
    E = np.zeros(1)
    phi = np.zeros(n)
    lib().or_ewald_tri(_ptr(A), n, _ptr(pos), _ptr(q), C.c_double(alpha), C.c_double(rcut), C.c_double(kmax),
                       _ptr(E), _ptr(phi))
    return float(E[0]), phi


def ewald_tri_auto(A, pos, q, tol=1e-13):
    """ewald_tri with alpha / kmax from the shortest face distance (truncation errors below tol)."""
    import math
    Am = np.asarray(A, np.float64).reshape(3, 3)
    V = abs(np.linalg.det(Am))
    w = [V / np.linalg.norm(np.cross(Am[(d + 1) % 3], Am[(d + 2) % 3])) for d in range(3)]
    rcut = min(0.5 * min(w), 12.0)
    x = math.sqrt(-math.log(tol))
    alpha = x / rcut
    return ewald_tri(Am, pos, q, alpha, rcut, 2 * alpha * x)


def ewald2d(Lx, Ly, pos, q, alpha=0.0):
    """2-D Ewald sum of a neutral slab (x, y periodic, z open): (E, phi)."""
    pos, q = _d(pos), _d(q)
    n = pos.shape[0]
    E = np.zeros(1)
    phi = np.zeros(n)
    lib().or_ewald2d(C.c_double(Lx), C.c_double(Ly), n, _ptr(pos), _ptr(q), C.c_double(alpha), _ptr(E), _ptr(phi))
    return float(E[0]), phi


def ewald1d(L, pos, q, alpha=0.0, axis=2):
    """1-D Ewald sum of a neutral wire periodic along `axis` with period L (the
    other two axes open): (E, phi)."""
    pos, q = _d(pos), _d(q)
    if axis != 2:
        order = [d for d in range(3) if d != axis] + [axis]
        pos = np.ascontiguousarray(pos[:, order])
    n = pos.shape[0]
    E = np.zeros(1)
    phi = np.zeros(n)
    lib().or_ewald1d(C.c_double(L), n, _ptr(pos), _ptr(q), C.c_double(alpha), _ptr(E), _ptr(phi))
    return float(E[0]), phi


def wire_top(p, a, nlev, L, rho):
    """Top-level kernel of a wire at the transverse distance rho (k_L summed over the 1-D lattice)."""
    f = lib().or_wire_top
    f.restype = C.c_double
    return float(f(int(p), C.c_double(a), int(nlev), C.c_double(L), C.c_double(rho)))


def slab_top(p, a, nlev, Lx, Ly, z):
    """Top-level kernel of a slab at the z offset z (k_L summed over the 2-D lattice)."""
    f = lib().or_slab_top
    f.restype = C.c_double
    return float(f(int(p), C.c_double(a), int(nlev), C.c_double(Lx), C.c_double(Ly), C.c_double(z)))


def ewald_auto(cell, pos, q, tol=1e-13, rcut=None, forces=True):
    """Ewald sum with alpha / kmax chosen so both truncation errors are below tol."""
    import math
    Lmin = min(cell)
    if rcut is None:
        rcut = min(0.5 * Lmin, 12.0) if Lmin > 8 else 0.5 * Lmin
    x = math.sqrt(-math.log(tol))
    alpha = x / rcut
    kmax = 2.0 * alpha * x
    return ewald(cell, pos, q, alpha, rcut, kmax, forces)
