"""CPU checks of the C-ABI library: it loads, exports every declared symbol,
and its host planner (grids, levels, stencils) agrees with the oracle's.

No compute call runs here (there is no GPU); the planner queries are
host-only entry points of the library.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2510_05961_gb300 import _lib, build
from paper_2510_05961_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "msm_gb300.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(msm_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    decl = _declared()
    assert len(decl) >= 15
    assert sorted(_lib.EXPORTS) == decl
    for name in decl:
        assert hasattr(lib, name), name
        # every call has its C signature declared to ctypes (an undeclared size_t argument
        # would be passed as a 32-bit int and wrap for workspaces above 2 GiB)
        assert getattr(lib, name).argtypes is not None, name


def _describe(lib, w=None, **kw):
    if w is not None:
        kw = dict(cell=w.cell, pbc=w.pbc, h=w.h, cutoff=w.a, order=w.p, levels=w.levels,
                  grid_override=w.grid_override)
    P = _lib.make_params(kw["cell"], kw["pbc"], kw["h"], kw["cutoff"], kw["order"], kw.get("levels", 0),
                         kw.get("grid_override", (0, 0, 0)), 1, kw.get("qi_mode", 0))
    I = _lib.PlanInfo()
    rc = lib.msm_plan_describe(C.byref(P), C.byref(I))
    return rc, I, P


CASES = [
    dict(cell=(30, 30, 30), pbc=(0, 0, 0), h=2.5, cutoff=10.0, order=4, levels=3),
    dict(cell=(49.6,) * 3, pbc=(1, 1, 1), h=1.5, cutoff=9.0, order=6),
    dict(cell=((1024000 / 0.1) ** (1 / 3),) * 3, pbc=(1, 1, 1), h=2.0, cutoff=8.0, order=4),
    dict(cell=((16384000 / 0.1) ** (1 / 3),) * 3, pbc=(1, 1, 1), h=2.0, cutoff=8.0, order=4),
    dict(cell=(180.48,) * 3, pbc=(1, 1, 1), h=2.0, cutoff=8.0, order=4),
    dict(cell=(6.3, 6.3, 6.3), pbc=(1, 1, 1), h=2.0, cutoff=8.0, order=4),
    dict(cell=(6.3, 6.3, 6.3), pbc=(0, 0, 0), h=2.0, cutoff=8.0, order=4),
    dict(cell=(20.0, 20.0, 20.0), pbc=(1, 1, 0), h=2.0, cutoff=8.0, order=4),
    dict(cell=(36.8, 36.8, 36.8), pbc=(1, 1, 0), h=2.0, cutoff=8.0, order=4),
    dict(cell=(17.0, 23.0, 29.0), pbc=(0, 0, 0), h=1.3, cutoff=4.5, order=8),
    dict(cell=(1.0, 1.0, 1.0), pbc=(1, 1, 1), h=0.0, cutoff=2.0, order=6, grid_override=(16, 16, 16)),
    dict(cell=(12.0, 12.0, 12.0), pbc=(0, 0, 0), h=1.0, cutoff=3.0, order=4, levels=1),
    # exact interpolation (qi_mode 1): wide omega', dense boxes on every level
    dict(cell=(30, 30, 30), pbc=(0, 0, 0), h=2.5, cutoff=10.0, order=4, levels=3, qi_mode=1),
    dict(cell=(8.0, 8.0, 8.0), pbc=(1, 1, 1), h=2.0, cutoff=2.0, order=6, qi_mode=1),
    # tilted periodic cells (rows a, b, c): a sheared cube, primitive fcc, monoclinic
    dict(cell=(12.0, 0, 0, 12.0, 12.0, 0, 0, 0, 12.0), pbc=(1, 1, 1), h=0.0, cutoff=6.0, order=4,
         grid_override=(16, 16, 16)),
    dict(cell=(0, 2.82, 2.82, 2.82, 0, 2.82, 2.82, 2.82, 0), pbc=(1, 1, 1), h=0.5, cutoff=2.0, order=6),
    dict(cell=(10.0, 0, 0, 0, 10.0, 0, 3.0, 0, 9.539392014169456), pbc=(1, 1, 1), h=1.2, cutoff=5.0, order=4),
    # slabs open along x or y and wires (one periodic axis): lattice-summed top levels
    dict(cell=(24.0, 20.0, 20.0), pbc=(0, 1, 1), h=2.0, cutoff=8.0, order=4),
    dict(cell=(20.0, 18.0, 20.0), pbc=(1, 0, 1), h=1.5, cutoff=6.0, order=6),
    dict(cell=(20.0, 20.0, 16.0), pbc=(0, 0, 1), h=2.0, cutoff=6.0, order=4),
    dict(cell=(32.0, 22.0, 26.0), pbc=(1, 0, 0), h=2.0, cutoff=8.0, order=8),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s_%s_p%d_qi%d%s" % (c["pbc"], c["cell"][0], c["order"],
                                                                            c.get("qi_mode", 0),
                                                                            "_tri" if len(c["cell"]) == 9 else ""))
def test_planner_matches_oracle(lib, oracle, case):
    rc, I, _ = _describe(lib, **case)
    assert rc == 0, lib.msm_last_error()
    P = oracle.make_plan(case["cell"], case["pbc"], case["h"], case["cutoff"], case["order"], case.get("levels", 0),
                         case.get("grid_override", (0, 0, 0)), case.get("qi_mode", 0))
    s = oracle.plan_summary(P)
    assert I.nlev == s["nlev"] and I.ncomp == s["ncomp"]
    assert list(I.M) == s["M"]
    assert np.allclose(list(I.h1), s["h1"], rtol=1e-15)
    for l in range(I.ncomp):
        assert list(I.lo[l]) == s["lo"][l] and list(I.n[l]) == s["n"][l]
    assert list(I.R) == s["R"] and list(I.C) == s["C"] and list(I.nnbr) == s["nnbr"]


def _lib_stencil(lib, P, level, which):
    lo = (C.c_int * 3)()
    sz = (C.c_int * 3)()
    assert lib.msm_plan_stencil(C.byref(P), level, which, None, 0, lo, sz) == 0
    out = np.zeros(sz[0] * sz[1] * sz[2], np.float32)
    rc = lib.msm_plan_stencil(C.byref(P), level, which, out.ctypes.data_as(C.c_void_p), out.size, lo, sz)
    assert rc == 0
    return out.reshape(tuple(sz)).astype(np.float64), tuple(lo)


def _fold(K, lo, n, pbc):
    """fold an offset box onto [0, n) along periodic axes (open axes unchanged)."""
    out_sz = [n[d] if pbc[d] else K.shape[d] for d in range(3)]
    out = np.zeros(out_sz)
    idx = [np.arange(K.shape[d]) + lo[d] for d in range(3)]
    idx = [(idx[d] % n[d]) if pbc[d] else np.arange(K.shape[d]) for d in range(3)]
    np.add.at(out, np.ix_(*idx), K)
    return out


@pytest.mark.parametrize("case", CASES[:2] + CASES[4:9] + CASES[10:],
                         ids=lambda c: "%s_%s_qi%d%s" % (c["pbc"], c["cell"][0], c.get("qi_mode", 0),
                                                        "_tri" if len(c["cell"]) == 9 else ""))
def test_stencils_match_oracle(lib, oracle, case):
    rc, I, Pl = _describe(lib, **case)
    P = oracle.make_plan(case["cell"], case["pbc"], case["h"], case["cutoff"], case["order"], case.get("levels", 0),
                         case.get("grid_override", (0, 0, 0)), case.get("qi_mode", 0))
    # every library query rebuilds the plan; the wide exact-interpolation stencils
    # are checked on K and two derivative components to keep the CPU suite short
    whiches = range(7) if case.get("qi_mode", 0) == 0 else (0, 1, 4)
    for l in range(1, I.ncomp + 1):
        ref = {which: oracle.stencil(P, l, which)[0] for which in range(7)}
        # tolerance: float32 rounding of the stored values, relative to the
        # largest entry of the stencil (which 0) or of the six derivatives
        scale_k = np.abs(ref[0]).max()
        scale_d = max(np.abs(ref[w]).max() for w in range(1, 7))
        for which in whiches:
            K, lo = _lib_stencil(lib, Pl, l, which)
            Kf = _fold(K, lo, P.level_shape(l), case["pbc"])
            assert Kf.shape == ref[which].shape, (l, which)
            scale = scale_k if which == 0 else scale_d
            err = np.abs(Kf - ref[which]).max()
            assert err <= 2e-6 * scale + 1e-30, (l, which, err, scale)


def test_planner_rejects_bad_settings(lib):
    bad = [
        (dict(cell=(10, 10, 10), pbc=(0, 0, 0), h=1.0, cutoff=3.0, order=5), _lib.MSM_ERR_INVALID_ARG),
        (dict(cell=(10, 10, 10), pbc=(0, 0, 0), h=1.0, cutoff=0.0, order=4), _lib.MSM_ERR_INVALID_ARG),
        (dict(cell=(10, 20, 10), pbc=(1, 1, 1), h=1.0, cutoff=3.0, order=4), _lib.MSM_ERR_UNSUPPORTED),
        (dict(cell=(10, 10, 10), pbc=(1, 1, 1), h=1.0, cutoff=3.0, order=4, levels=2), _lib.MSM_ERR_UNSUPPORTED),
        (dict(cell=(10, 10, 10), pbc=(1, 1, 1), h=0.0, cutoff=3.0, order=4, grid_override=(12, 12, 12)),
         _lib.MSM_ERR_UNSUPPORTED),
        (dict(cell=(10, 10, -1), pbc=(0, 0, 0), h=1.0, cutoff=3.0, order=4), _lib.MSM_ERR_INVALID_ARG),
    ]
    for kw, code in bad:
        rc, _, _ = _describe(lib, **kw)
        assert rc == code, (kw, rc)
        assert lib.msm_last_error()
    # a tilted cell needs all three axes periodic, and a right-handed basis
    P = _lib.make_params([10, 1, 0, 0, 10, 0, 0, 0, 10], (1, 1, 0), 1.0, 3.0, 4)
    I = _lib.PlanInfo()
    assert lib.msm_plan_describe(C.byref(P), C.byref(I)) == _lib.MSM_ERR_UNSUPPORTED
    P = _lib.make_params([10, 1, 0, 0, 0, 10, 0, 10, 0], (1, 1, 1), 1.0, 3.0, 4)
    assert lib.msm_plan_describe(C.byref(P), C.byref(I)) == _lib.MSM_ERR_INVALID_ARG


def test_batch_systems_plan(lib, oracle):
    for w in W.batch_systems(nsys=30, seed=77):
        rc, I, _ = _describe(lib, w)
        assert rc == 0, lib.msm_last_error()
        s = oracle.plan_summary(oracle.plan_for(w))
        assert I.nlev == s["nlev"] and list(I.M) == s["M"] and list(I.C) == s["C"]


SPECTRAL_CASES = [
    dict(cell=(49.6,) * 3, pbc=(1, 1, 1), h=1.5, cutoff=9.0, order=6),
    dict(cell=(60.0, 48.0, 54.0), pbc=(1, 1, 1), h=0.0, cutoff=8.0, order=4, grid_override=(32, 32, 32)),
    dict(cell=(39.15,) * 3, pbc=(1, 1, 1), h=1.6, cutoff=7.0, order=8),
    dict(cell=(6.3, 6.3, 6.3), pbc=(1, 1, 1), h=2.0, cutoff=8.0, order=4),
]


@pytest.mark.parametrize("case", SPECTRAL_CASES)
def test_spectra_match_fft_of_oracle_stencils(lib, oracle, case):
    """The spectral level method's stored spectra (msm_plan_stencil which 7..13: the
    octant k_d <= n_d/2 of the DFT of the folded K^l and dK^l, times 1/N and -1/2 (1/N))
    against numpy's FFT of the oracle's folded stencils on each level grid. The DFT of
    the folded stencil is real (K, dK_aa even in every axis; dK_ab odd in a and b), and
    its imaginary part vanishes to rounding."""
    rc, I, Pl = _describe(lib, **case)
    assert rc == 0
    P = oracle.make_plan(case["cell"], case["pbc"], case["h"], case["cutoff"], case["order"], case.get("levels", 0),
                         case.get("grid_override", (0, 0, 0)), case.get("qi_mode", 0))
    for l in range(1, I.ncomp + 1):
        n = P.level_shape(l)
        N = float(np.prod(n))
        h = tuple(d // 2 + 1 for d in n)
        refs = []
        for which in range(7):
            F = np.fft.fftn(oracle.stencil(P, l, which)[0])
            refs.append(F.real[:h[0], :h[1], :h[2]] * ((1.0 if which == 0 else -0.5) / N))
            assert np.abs(F.imag).max() <= 1e-9 * np.abs(F).max(), (l, which)
        # tolerance: float32 rounding of the stored values, relative to the largest
        # entry of the level's K^ (which 7) or of its six dK^ (which 8 .. 13)
        scale_k = np.abs(refs[0]).max()
        scale_d = max(np.abs(r).max() for r in refs[1:])
        for which in range(7):
            got, lo = _lib_stencil(lib, Pl, l, 7 + which)
            assert lo == (0, 0, 0) and got.shape == h
            scale = scale_k if which == 0 else scale_d
            err = np.abs(got - refs[which]).max()
            assert err <= 2e-6 * scale, (l, which, err, scale)


def test_spectra_refused_without_spectral_method(lib):
    for case in (CASES[0], dict(cell=(20.0, 20.0, 20.0), pbc=(1, 1, 0), h=2.0, cutoff=8.0, order=4)):
        rc, I, Pl = _describe(lib, **case)
        lo = (C.c_int * 3)()
        sz = (C.c_int * 3)()
        assert lib.msm_plan_stencil(C.byref(Pl), 1, 7, None, 0, lo, sz) == _lib.MSM_ERR_UNSUPPORTED
