"""Pins of the FP64 oracle against values that do not come from the oracle.

Each test checks one part of the oracle against a closed form, a textbook
value, a mathematical identity of the method, an exact direct sum, an Ewald
sum, the rock-salt Madelung constant or finite differences. A plausible slip
(a dropped term, a wrong sign or index, a transposed operand) in any oracle
function fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2510_05961_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ----------------------------------------------------------------- softening / splitting
def test_gamma_closed_forms(oracle):
    # gamma(0) = sum_k binom(2k,k)/4^k, k < p: 35/16, 693/256, 6435/2048
    assert oracle.gamma(4, 0.0) == pytest.approx(35 / 16, rel=1e-15)
    assert oracle.gamma(6, 0.0) == pytest.approx(693 / 256, rel=1e-15)
    assert oracle.gamma(8, 0.0) == pytest.approx(6435 / 2048, rel=1e-15)
    # order 3 is the classic C^2 softening 15/8 - 5/4 rho^2 + 3/8 rho^4
    for rho in np.linspace(0, 0.999, 17):
        assert oracle.gamma(3, rho) == pytest.approx(15 / 8 - 5 / 4 * rho ** 2 + 3 / 8 * rho ** 4, rel=1e-14)
    for p in (4, 6, 8):
        for rho in (1.0, 1.3, 7.0):
            assert oracle.gamma(p, rho) == pytest.approx(1 / rho, rel=1e-15)
            assert oracle.dgamma(p, rho) == pytest.approx(-1 / rho ** 2, rel=1e-15)


@pytest.mark.parametrize("p", [4, 6, 8])
def test_gamma_smooth_join(oracle, p):
    # gamma is C^(p-1) at rho = 1: on [0,1) it is a polynomial of degree 2p-2;
    # recover it from samples and compare its derivatives at 1 with those of
    # 1/rho, (-1)^k k!. Orders 0..p-1 agree, order p does not.
    deg = 2 * p - 2
    xs = 0.5 - 0.5 * np.cos(np.pi * (np.arange(deg + 1) + 0.5) / (deg + 1))
    ys = np.array([oracle.gamma(p, x) for x in xs])
    poly = np.polynomial.Polynomial.fit(xs, ys, deg).convert()
    for k in range(p + 1):
        dk = poly.deriv(k)(1.0) if k else poly(1.0)
        ref = (-1) ** k * math.factorial(k)
        if k < p:
            assert dk == pytest.approx(ref, rel=1e-7, abs=1e-7), (k, dk, ref)
        else:
            assert abs(dk - ref) > 1e-3 * abs(ref)
    # derivative function against a central difference
    for rho in (0.1, 0.5, 0.9):
        fd = (oracle.gamma(p, rho + 1e-6) - oracle.gamma(p, rho - 1e-6)) / 2e-6
        assert oracle.dgamma(p, rho) == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("p", [4, 6, 8])
@pytest.mark.parametrize("nlev", [1, 3, 6])
def test_splitting_telescopes_to_coulomb(oracle, p, nlev):
    # Eq. kernel_splitting: sum_l k_l(r) = 1/r, and sum_(l>=1) k_l(0) = gamma(0)/a
    a = 3.7
    for r in np.geomspace(0.05, 400.0, 37):
        s = sum(oracle.kl(p, a, nlev, l, r) for l in range(nlev + 1))
        assert s == pytest.approx(1.0 / r, rel=1e-13)
        ds = sum(oracle.dkl(p, a, nlev, l, r) for l in range(nlev + 1))
        assert ds == pytest.approx(-1.0 / r ** 2, rel=1e-11)
    self_sum = sum(oracle.kl(p, a, nlev, l, 0.0) for l in range(1, nlev + 1))
    assert self_sum == pytest.approx(oracle.gamma(p, 0.0) / a, rel=1e-14)
    # finite ranges: k_0 vanishes from a, k_l from 2^l a (l < L)
    assert oracle.kl(p, a, nlev, 0, a) == 0.0
    for l in range(1, nlev):
        assert oracle.kl(p, a, nlev, l, 2 ** l * a * 1.0000001) == 0.0
        assert oracle.kl(p, a, nlev, l, 2 ** l * a * 0.99) != 0.0


# ----------------------------------------------------------------- B-splines, J
@pytest.mark.parametrize("row", _golden_lines("bspline_integer_values.txt"))
def test_bspline_integer_values(oracle, row):
    p = int(row[0])
    for t, v in enumerate(row[1:]):
        assert oracle.bspline(p, t) == pytest.approx(float(Fraction(v)), rel=1e-14, abs=1e-16)
        assert oracle.bspline(p, -t) == pytest.approx(float(Fraction(v)), rel=1e-14, abs=1e-16)


@pytest.mark.parametrize("p", [4, 6, 8])
def test_bspline_partition_of_unity_and_derivative(oracle, p):
    rng = np.random.default_rng(p)
    for u in rng.uniform(-5, 5, 25):
        s = sum(oracle.bspline(p, u - m) for m in range(-12, 13))
        assert s == pytest.approx(1.0, abs=1e-14)
        ds = sum(oracle.dbspline(p, u - m) for m in range(-12, 13))
        assert abs(ds) < 1e-13
        fd = (oracle.bspline(p, u + 1e-6) - oracle.bspline(p, u - 1e-6)) / 2e-6
        assert oracle.dbspline(p, u) == pytest.approx(fd, abs=1e-8)
    # unit integral and support (-p/2, p/2)
    xs = np.linspace(-p / 2, p / 2, 4001)
    vals = np.array([oracle.bspline(p, x) for x in xs])
    assert np.trapezoid(vals, xs) == pytest.approx(1.0, abs=1e-6)
    assert oracle.bspline(p, p / 2) == 0.0 and oracle.bspline(p, p / 2 + 0.3) == 0.0


@pytest.mark.parametrize("p", [4, 6, 8])
def test_two_scale_relation(oracle, p):
    # Phi_p(x/2) = sum_k J_k Phi_p(x - k): the relation restriction rests on
    J = oracle.J(p)
    assert J[0::2].sum() == pytest.approx(1.0, abs=1e-15)
    assert J[1::2].sum() == pytest.approx(1.0, abs=1e-15)
    for x in np.linspace(-p, p, 41):
        rhs = sum(J[k + p // 2] * oracle.bspline(p, x - k) for k in range(-p // 2, p // 2 + 1))
        assert oracle.bspline(p, x / 2) == pytest.approx(rhs, abs=1e-14)


@pytest.mark.parametrize("p", [4, 6, 8])
def test_omega_polynomial_reproduction(oracle, p):
    """1-D kernel interpolation of a polynomial f(x - y) of degree < p is exact.

    S(x,y) = sum_m sum_n Phi(x-m) K_(m-n) Phi(y-n) with K_k = sum_t omega'_t f(k-t)
    (Eq. kernel_stencil_by_conv_with_universal_coeff in one dimension). Exactness
    for degree < p is the approximation order the quasi-interpolation must keep;
    degree p is not reproduced, so the sequence is no longer than it needs to be.
    """
    om = oracle.omega(p)
    r = p // 2 - 1
    rng = np.random.default_rng(10 + p)
    pts = rng.uniform(-3, 3, size=(12, 2))

    def S(f, x, y):
        mx = np.arange(math.floor(x) - p // 2 + 1, math.floor(x) + p // 2 + 1)
        ny = np.arange(math.floor(y) - p // 2 + 1, math.floor(y) + p // 2 + 1)
        tot = 0.0
        for m in mx:
            for n in ny:
                K = sum(om[t + r] * f(m - n - t) for t in range(-r, r + 1))
                tot += oracle.bspline(p, x - m) * K * oracle.bspline(p, y - n)
        return tot

    for j in range(p):
        f = lambda t, j=j: float(t) ** j
        for x, y in pts:
            assert S(f, x, y) == pytest.approx((x - y) ** j, abs=1e-10 * (1 + abs(x - y) ** j))
    f = lambda t: float(t) ** p
    errs = [abs(S(f, x, y) - (x - y) ** p) for x, y in pts]
    assert max(errs) > 1e-6


# ----------------------------------------------------------------- grids
def _random_atoms(n, side, seed, neutral=True):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, side, size=(n, 3))
    q = rng.normal(size=n)
    if neutral:
        q -= q.mean()
    return pos, q


@pytest.mark.parametrize("pbc", [(1, 1, 1), (0, 0, 0), (1, 1, 0)])
@pytest.mark.parametrize("p", [4, 6])
def test_restriction_is_exact_anterpolation(oracle, pbc, p):
    # anterpolating with the level-2 basis (spacing 2h) equals restricting the
    # level-1 grid charge: the translation operator of Sec. 2 is exact for B-splines
    side = 17.0
    pos, q = _random_atoms(60, side, 3)
    P1 = oracle.make_plan((side,) * 3, pbc, 0, 4.0, p, grid_override=(16, 16, 16))
    P2 = oracle.make_plan((side,) * 3, pbc, 0, 4.0, p, grid_override=(8, 8, 8))
    assert P1.level_shape(2) == P2.level_shape(1) and P1.level_lo(2) == P2.level_lo(1)
    g1 = oracle.anterp(P1, pos, q)
    g2 = oracle.restrict(P1, 1, g1)
    d = oracle.anterp(P2, pos, q)
    assert np.abs(g2 - d).max() <= 1e-13 * np.abs(d).max()


@pytest.mark.parametrize("pbc", [(1, 1, 1), (0, 0, 0), (0, 1, 1)])
def test_charge_conservation_and_adjoint(oracle, pbc):
    side = 23.0
    pos, q = _random_atoms(80, side, 4, neutral=False)
    P = oracle.make_plan((side,) * 3, pbc, 2.0, 5.0, 4)
    g = oracle.anterp(P, pos, q)
    levels = [g]
    for l in range(1, P.ncomp):
        levels.append(oracle.restrict(P, l, levels[-1]))
    for g in levels:
        assert g.sum() == pytest.approx(q.sum(), rel=1e-12, abs=1e-12)
    rng = np.random.default_rng(5)
    for l in range(1, P.ncomp):
        f = rng.normal(size=P.level_shape(l))
        c = rng.normal(size=P.level_shape(l + 1))
        lhs = (oracle.restrict(P, l, f) * c).sum()
        rhs = (f * oracle.prolong_add(P, l, c, np.zeros_like(f))).sum()
        assert lhs == pytest.approx(rhs, rel=1e-12)


def test_plan_rules(oracle):
    P = oracle.plan_for(W.open_cluster())
    s = oracle.plan_summary(P)
    assert s["nlev"] == 3 and s["M"] == [12, 12, 12]
    assert s["lo"] == [[-2] * 3, [-2] * 3, [-2] * 3] and s["n"] == [[17] * 3, [11] * 3, [8] * 3]
    assert s["R"] == [8] * 3
    # 1M-atom sweep point: M = 128, 8 levels, top dropped
    L = (1024000 / 0.1) ** (1 / 3)
    P = oracle.make_plan((L,) * 3, (1, 1, 1), 2.0, 8.0, 4)
    assert (P.M[0], P.nlev, P.ncomp, P.R[0]) == (128, 8, 7, 10)
    with pytest.raises(ValueError):
        oracle.make_plan((10, 20, 10), (1, 1, 1), 1.0, 3.0, 4)  # unequal periodic grids
    with pytest.raises(ValueError):
        oracle.make_plan((10, 10, 10), (0, 0, 0), 1.0, 3.0, 5)  # odd order


def test_stencil_symmetry_and_level_scaling_open(oracle):
    # K_m = K_-m, the cube's axis symmetry, and K^l = K^1 / 2^(l-1) below the top level (Sec. 3.4)
    side = 19.0
    P = oracle.make_plan((side,) * 3, (0, 0, 0), 1.2, 3.0, 4)
    K1, lo1 = oracle.stencil(P, 1)
    assert np.allclose(K1, K1[::-1, ::-1, ::-1], rtol=1e-14, atol=0)
    assert np.allclose(K1, np.transpose(K1, (1, 0, 2)), rtol=1e-14, atol=0)
    assert P.ncomp >= 3
    for l in range(2, P.ncomp):
        Kl, _ = oracle.stencil(P, l)
        assert np.abs(Kl - K1 / 2 ** (l - 1)).max() <= 1e-14 * np.abs(K1).max()


def _fold(K, n):
    """Sum of a periodic stencil over its images on a grid of n points per axis (n divides K's size)."""
    m = K.shape[0] // n
    return K.reshape(m, n, m, n, m, n).sum(axis=(0, 2, 4))


def test_stencil_symmetry_and_level_scaling_periodic(oracle):
    """Periodic levels store the folded stencil on the level's own grid (index m mod n_l).
    It is even (K_m = K_(-m mod n)) and symmetric under exchanging the axes of the
    cube; and since k_l(|h_l n|) = k_1(|h_1 n|) / 2^(l-1), each coarser level is the
    level-1 stencil folded onto its grid and scaled: K^l = fold_(n_l)(K^1) / 2^(l-1).
    Level 1 here has 2R + 1 = 13 < 16 points per axis (no self-overlap), level 2
    folds onto 8 points, so images that overlap must be summed."""
    side = 19.0
    P = oracle.make_plan((side,) * 3, (1, 1, 1), 1.2, 3.0, 4)
    assert P.M[0] == 16 and 2 * P.R[0] + 1 < 16 and P.ncomp == 4
    K1, lo1 = oracle.stencil(P, 1)
    assert K1.shape == (16, 16, 16) and tuple(lo1) == (0, 0, 0)
    # the unfolded support [-R, R] maps one to one onto the 16-point grid
    R = P.R[0]
    idx = np.r_[np.arange(0, R + 1), np.arange(16 - R, 16)]
    assert np.abs(np.delete(K1, idx, axis=0)).max() == 0.0
    scale = np.abs(K1).max()
    for l in range(1, P.ncomp + 1):
        Kl, lo = oracle.stencil(P, l)
        n = Kl.shape[0]
        neg = np.roll(Kl[::-1, ::-1, ::-1], 1, axis=(0, 1, 2))  # K[(-m) mod n]
        assert np.abs(Kl - neg).max() <= 1e-14 * scale
        for perm in [(1, 0, 2), (0, 2, 1), (2, 1, 0)]:
            assert np.abs(Kl - np.transpose(Kl, perm)).max() <= 1e-14 * scale
        assert np.abs(Kl - _fold(K1, n) / 2 ** (l - 1)).max() <= 1e-13 * scale, l


@pytest.mark.parametrize("p", [4, 6])
def test_level_interpolation_converges_at_order_p(oracle, p):
    # level-1 grid energy 1/2 q~^T K^1 q~ against the direct sum of k_1 over all
    # pairs (i == j included, Eq. U_oneplus): the error falls by ~2^p per halving of h
    side, a = 12.0, 5.0
    pos, q = _random_atoms(70, side, 6)
    Ue, _ = oracle.direct_level(p, a, 3, 1, pos, q)
    errs = []
    for h in (1.25, 0.625):
        P = oracle.make_plan((side,) * 3, (0, 0, 0), h, a, p, 3)
        g = oracle.anterp(P, pos, q)
        K, _ = oracle.stencil(P, 1)
        e = oracle.stencil_apply(P, 1, K, g)
        errs.append(abs(0.5 * (g * e).sum() - Ue) / abs(Ue))
    assert errs[0] / errs[1] > 0.6 * 2 ** p, errs


# ----------------------------------------------------------------- short range
def test_short_range_against_brute_force_images(oracle):
    # cell > a and cell < a (self images, a > L/2): brute force over images
    for side, a in ((9.0, 4.0), (5.0, 6.5)):
        pos, q = _random_atoms(40, side, 8)
        P = oracle.make_plan((side,) * 3, (1, 1, 1), 1.0, a, 4)
        phi0, F0, W0 = oracle.short_range(P, pos, q)
        nimg = int(math.ceil(a / side)) + 1
        phi = np.zeros(40)
        F = np.zeros((40, 3))
        Wb = np.zeros((3, 3))
        for i in range(40):
            for j in range(40):
                for n in np.ndindex(*(2 * nimg + 1,) * 3):
                    sh = (np.array(n) - nimg) * side
                    if i == j and not sh.any():
                        continue
                    d = pos[j] + sh - pos[i]
                    r = np.linalg.norm(d)
                    if r >= a:
                        continue
                    phi[i] += q[j] * oracle.kl(4, a, P.nlev, 0, r)
                    dk = oracle.dkl(4, a, P.nlev, 0, r)
                    F[i] += q[i] * q[j] * dk * d / r
                    Wb += -0.5 * q[i] * q[j] * dk * np.outer(d, d) / r
            phi[i] -= q[i] * oracle.gamma(4, 0.0) / a
        assert np.allclose(phi0, phi, rtol=1e-12, atol=1e-12)
        assert np.allclose(F0, F, rtol=1e-11, atol=1e-11)
        assert np.allclose(W0, Wb, rtol=1e-11, atol=1e-11)
        assert np.abs(F0.sum(0)).max() < 1e-10 * np.abs(F0).max()  # Newton's third law


def test_binning_contract(oracle):
    # the FP32 cell-index contract written out independently in numpy float32
    for w in (W.random_box(3000, seed=11), W.open_cluster(n=500, seed=12)):
        P = oracle.plan_for(w)
        cid, start, perm, st = oracle.bin_atoms(P, w.pos, w.q)
        assert st == 0
        C = np.array([P.C[d] for d in range(3)])
        c = np.zeros((w.n, 3), np.int64)
        for d in range(3):
            inv = np.float32(1.0 / w.cell[d])
            s = w.pos[:, d].astype(np.float32) * inv
            if w.pbc[d]:
                s = (s - np.floor(s)).astype(np.float32)
                s[s >= np.float32(1.0)] = np.float32(0.0)
            t = (s * np.float32(C[d])).astype(np.float32)
            c[:, d] = np.minimum(t.astype(np.int64), C[d] - 1)
        ref = (c[:, 0] * C[1] + c[:, 1]) * C[2] + c[:, 2]
        assert np.array_equal(cid, ref)
        assert np.array_equal(perm, np.lexsort((np.arange(w.n), ref)))
        assert np.array_equal(start, np.concatenate([[0], np.cumsum(np.bincount(ref, minlength=C.prod()))]))
    # out-of-cell and non-finite inputs are flagged
    w = W.open_cluster(n=50)
    pos = w.pos.copy()
    pos[3, 1] = -1.0
    P = oracle.plan_for(w)
    assert oracle.bin_atoms(P, pos, w.q)[3] & oracle.ST_OUTSIDE
    pos[3, 1] = np.nan
    assert oracle.bin_atoms(P, pos, w.q)[3] & oracle.ST_NONFINITE


# ----------------------------------------------------------------- whole method
def test_omega_exact_closed_form_p4(oracle):
    """Exact interpolation, p = 4: the sampled cubic B-spline is (1/6, 2/3, 1/6),
    whose inverse is omega_n = sqrt(3) z^|n| with z = sqrt(3) - 2 (the root of
    z^2 + 4 z + 1 inside the unit circle); omega' = omega * omega is then
    3 z^|n| (|n| + (1 + z^2) / (1 - z^2))."""
    w = oracle.omega_exact(4)
    hw = (len(w) - 1) // 2
    z = math.sqrt(3.0) - 2.0
    for n in range(-hw, hw + 1):
        ref = 3.0 * z ** abs(n) * (abs(n) + (1 + z * z) / (1 - z * z))
        assert w[n + hw] == pytest.approx(ref, rel=1e-12, abs=1e-15)
    # truncation: the first dropped coefficient is below 1e-12 of omega'_0
    ref_next = 3.0 * abs(z) ** (hw + 1) * (hw + 1 + (1 + z * z) / (1 - z * z))
    assert ref_next < 1e-12 * w[hw] <= 3.0 * abs(z) ** hw * (hw + (1 + z * z) / (1 - z * z))


@pytest.mark.parametrize("p", [6, 8])
def test_omega_exact_inverts_the_sampled_bspline(oracle, p):
    """omega' convolved with the sampled B-spline b twice is the unit impulse
    (b * b * omega' = delta), checked against the direct inverse of the banded
    Toeplitz matrix of b (numpy linear algebra, an independent method)."""
    w = oracle.omega_exact(p)
    hw = (len(w) - 1) // 2
    b = np.array([oracle.bspline(p, m) for m in range(-p // 2 + 1, p // 2)])
    bb = np.convolve(b, b)
    d = np.convolve(bb, w)
    c = len(d) // 2
    impulse = np.zeros_like(d)
    impulse[c] = 1.0
    assert np.abs(d[c - hw + 2 * p:c + hw - 2 * p + 1] - impulse[c - hw + 2 * p:c + hw - 2 * p + 1]).max() < 1e-11
    n = 4 * hw + 1
    T = np.zeros((n, n))
    for i in range(n):
        for k, bk in enumerate(b):
            j = i + k - (len(b) - 1) // 2
            if 0 <= j < n:
                T[i, j] = bk
    om = np.linalg.solve(T, np.eye(n)[:, n // 2])  # omega, the inverse of b
    om2 = np.convolve(om, om)[n - 1 - hw:n + hw]   # omega * omega around the centre
    assert np.abs(om2 - w).max() < 1e-10 * w[hw]


def test_exact_interpolation_msm_against_direct(oracle):
    """The open cluster (config 1 settings): exact interpolation of the grid kernels
    is closer to the direct Coulomb sum than minimal quasi-interpolation."""
    w = W.open_cluster()
    pos, q = w.pos.astype(np.float64), w.q.astype(np.float64)
    E0, phi0, F0 = oracle.direct_open(pos, q)
    errs = {}
    for qi in (0, 1):
        P = oracle.make_plan(w.cell, w.pbc, w.h, w.a, w.p, w.levels, qi_mode=qi)
        assert P.hw == (1 if qi == 0 else 23) and P.R[0] == P.S[0] + P.hw
        r = oracle.msm(P, pos, q, virial=False)
        ferr = np.sqrt(((r["F"] - F0) ** 2).sum(1).mean() / (F0 ** 2).sum(1).mean())
        errs[qi] = (abs(r["E"] - E0) / abs(E0), ferr)
    assert errs[1][1] < errs[0][1] / 2 and errs[1][0] < errs[0][0] / 2


def test_open_cluster_against_direct_coulomb(oracle):
    w = W.open_cluster()
    pos, q = w.pos.astype(np.float64), w.q.astype(np.float64)
    E0, phi0, F0 = oracle.direct_open(pos, q)
    errs = {}
    for h, p in ((2.5, 4), (1.25, 4), (1.25, 6)):
        P = oracle.make_plan(w.cell, w.pbc, h, w.a, p)
        r = oracle.msm(P, pos, q, virial=False)
        ferr = np.sqrt(((r["F"] - F0) ** 2).sum(1).mean() / (F0 ** 2).sum(1).mean())
        perr = np.sqrt(((r["phi"] - phi0) ** 2).mean() / (phi0 ** 2).mean())
        errs[(h, p)] = (abs(r["E"] - E0) / abs(E0), ferr, perr)
    assert errs[(2.5, 4)][1] < 5e-3
    assert errs[(1.25, 4)][1] < errs[(2.5, 4)][1] / 5
    assert errs[(1.25, 4)][0] < errs[(2.5, 4)][0] / 5
    assert errs[(1.25, 6)][1] < errs[(1.25, 4)][1]
    assert errs[(1.25, 4)][1] < 5e-4


def test_periodic_against_ewald(oracle):
    pos, q = _random_atoms(300, 14.0, 9)
    cell = (14.0,) * 3
    Ee, phie, Fe = oracle.ewald_auto(cell, pos, q)
    # the error falls as h halves (M = 8, 16, 32) and, once the grid resolves
    # the kernels, as p rises
    errs = {}
    for M, p in ((8, 4), (16, 4), (32, 4), (32, 6)):
        P = oracle.make_plan(cell, (1, 1, 1), 0, 6.0, p, grid_override=(M, M, M))
        r = oracle.msm(P, pos, q, virial=False)
        ferr = np.sqrt(((r["F"] - Fe) ** 2).sum(1).mean() / (Fe ** 2).sum(1).mean())
        errs[(M, p)] = (abs(r["E"] - Ee) / abs(Ee), ferr)
    for a, b in (((8, 4), (16, 4)), ((16, 4), (32, 4)), ((32, 4), (32, 6))):
        assert errs[b][0] < errs[a][0] / 3 and errs[b][1] < errs[a][1] / 3, errs
    assert errs[(32, 6)][1] < 1e-4


def test_ewald_madelung(oracle):
    ref = float(_golden_lines("madelung_nacl.txt")[0][0])
    pos, q, L = W.nacl_crystal(1)
    E, phi, F = oracle.ewald_auto((L,) * 3, pos, q, rcut=0.5)
    assert -E * 0.5 / 4 == pytest.approx(ref, abs=1e-6)


def test_msm_madelung(oracle):
    # Sec. 4.1: p = 6 in FP64 reaches 7-8 decimals of the Madelung constant
    ref = float(_golden_lines("madelung_nacl.txt")[0][0])
    pos, q, L = W.nacl_crystal(1)
    P = oracle.make_plan((L,) * 3, (1, 1, 1), 0, 4.0 * 0.5 * L, 6, grid_override=(16, 16, 16))  # a = 4 d_min, h = d_min / 8
    r = oracle.msm(P, pos, q, virial=True)
    M = -r["E"] * 0.5 / 4
    assert M == pytest.approx(ref, abs=1e-6)
    assert np.abs(r["F"]).max() < 1e-12
    # cubic symmetry and Coulomb homogeneity: W = E/3 * identity (a not scaled: approx)
    assert np.allclose(r["W"], np.eye(3) * r["E"] / 3, rtol=5e-5, atol=5e-5 * abs(r["E"]))


def _sheared(L=12.0, n=60, seed=5):
    # a cube of atoms and a tilted cell spanning the same lattice (b' = a + b)
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, L, (n, 3))
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    rng.shuffle(q)
    return pos, q, L, np.array([[L, 0, 0], [L, L, 0], [0, 0, L]])


def test_triclinic_ewald_lattice_invariance(oracle):
    """The general-cell Ewald sum depends on the lattice, not on the cell that
    spans it, and reduces to the rectangular sum for a diagonal cell."""
    pos, q, L, A = _sheared()
    E0 = oracle.ewald_auto((L, L, L), pos, q, forces=False)[0]
    Ed = oracle.ewald_tri_auto(np.diag([L, L, L]), pos, q)[0]
    Es = oracle.ewald_tri_auto(A, pos, q)[0]
    Es2 = oracle.ewald_tri_auto(np.array([[L, 0, 0], [2 * L, L, 0], [L, -L, L]]), pos, q)[0]
    assert Ed == pytest.approx(E0, rel=1e-12)
    assert Es == pytest.approx(E0, rel=1e-10) and Es2 == pytest.approx(E0, rel=1e-10)


def test_triclinic_msm_against_ewald(oracle):
    """MSM in a tilted cell (fractional grids, metric-aware stencils) converges to
    the Ewald sum of the same lattice as the grid is refined."""
    pos, q, L, A = _sheared()
    E0, phi0 = oracle.ewald_auto((L, L, L), pos, q, forces=False)[:2]
    errs = []
    for M in (16, 32):
        P = oracle.make_plan(A, (1, 1, 1), 0, 6.0, 6, grid_override=(M, M, M))
        assert P.tri == 1
        r = oracle.msm(P, pos, q, forces=False, virial=False)
        errs.append(np.sqrt(((r["phi"] - phi0) ** 2).mean() / (phi0 ** 2).mean()))
    assert errs[1] <= 1e-4 and errs[0] > 10 * errs[1]


def test_triclinic_forces_and_virial_by_differences(oracle):
    """F = -dE/dr and all six W = -dE/d eps (r -> (1+eps) r, cell rows -> (1+eps) rows)
    by central differences in a tilted cell."""
    pos, q, L, A = _sheared()
    P = oracle.make_plan(A, (1, 1, 1), 0, 6.0, 4, grid_override=(16, 16, 16))
    r = oracle.msm(P, pos, q)
    for i in (3, 7):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += 1e-5
            pm[i, d] -= 1e-5
            fd = (oracle.msm(P, pp, q, False, False)["E"] - oracle.msm(P, pm, q, False, False)["E"]) / 2e-5
            assert -fd == pytest.approx(r["F"][i, d], rel=1e-6, abs=1e-7)
    for a, b in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
        es = []
        for sg in (1, -1):
            eps = np.zeros((3, 3))
            eps[a, b] += 0.5e-6 * sg
            eps[b, a] += 0.5e-6 * sg
            Fm = np.eye(3) + eps
            P2 = oracle.make_plan(A @ Fm.T, (1, 1, 1), 0, 6.0, 4, grid_override=(16, 16, 16))
            es.append(oracle.msm(P2, pos @ Fm.T, q, False, False)["E"])
        assert -(es[0] - es[1]) / 2e-6 == pytest.approx(r["W"][a, b], rel=1e-5, abs=1e-7)


def test_primitive_nacl_madelung(oracle):
    """Rock salt in its primitive (rhombohedral) cell, two ions: the general-cell
    Ewald sum and the MSM (p = 6) reproduce the Madelung constant of the
    conventional cell (Sec. 4.1's non-orthorhombic check)."""
    ref = float(_golden_lines("madelung_nacl.txt")[0][0])
    A = 0.5 * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0]])
    pos = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    q = np.array([1.0, -1.0])
    assert -oracle.ewald_tri_auto(A, pos, q)[0] * 0.5 == pytest.approx(ref, abs=1e-6)
    P = oracle.make_plan(A, (1, 1, 1), 0, 4.0 * 0.5, 6, grid_override=(16, 16, 16))  # a = 4 d_min
    r = oracle.msm(P, pos, q, virial=False)
    assert -r["E"] * 0.5 == pytest.approx(ref, abs=1e-6)
    assert np.abs(r["F"]).max() < 1e-10


def test_triclinic_binning_contract(oracle):
    """The FP32 cell contract of a general cell, written out in numpy float32:
    s_d = ((T_d0 x + T_d1 y) + T_d2 z) with T = (float) A^-T, each step rounded."""
    pos, q, L, A = _sheared(n=500, seed=9)
    pos = (pos + np.array([0.3, -0.2, 0.1]) * L).astype(np.float32)  # some atoms outside the cell
    P = oracle.make_plan(A, (1, 1, 1), 0, 6.0, 4, grid_override=(16, 16, 16))
    cid, start, perm, st = oracle.bin_atoms(P, pos, q.astype(np.float32))
    assert st == 0
    T = np.linalg.inv(A).T.astype(np.float32)
    C = np.array([P.C[d] for d in range(3)])
    c = np.zeros((len(pos), 3), np.int64)
    for d in range(3):
        s = ((T[d, 0] * pos[:, 0]).astype(np.float32) + (T[d, 1] * pos[:, 1]).astype(np.float32)).astype(np.float32)
        s = (s + (T[d, 2] * pos[:, 2]).astype(np.float32)).astype(np.float32)
        s = (s - np.floor(s)).astype(np.float32)
        s[s >= np.float32(1.0)] = np.float32(0.0)
        t = (s * np.float32(C[d])).astype(np.float32)
        c[:, d] = np.minimum(t.astype(np.int64), C[d] - 1)
    assert np.array_equal(cid, (c[:, 0] * C[1] + c[:, 1]) * C[2] + c[:, 2])


def _small_periodic():
    pos, q = _random_atoms(40, 9.0, 13)
    return pos, q, (9.0, 9.0, 9.0)


@pytest.mark.parametrize("pbc", [(1, 1, 1), (0, 0, 0), (1, 1, 0)])
def test_exact_invariants(oracle, pbc):
    rng = np.random.default_rng(14)
    pos, q, cell = _small_periodic()
    if not any(pbc) or pbc == (1, 1, 0):
        pos = np.clip(pos, 0.5, 8.5)
    P = oracle.make_plan(cell, pbc, 1.2, 3.5, 4)
    r = oracle.msm(P, pos, q)
    assert r["E"] == pytest.approx(0.5 * (q * r["phi"]).sum(), rel=1e-14)
    # E(lambda q) = lambda^2 E
    assert oracle.msm(P, pos, 2.5 * q, forces=False, virial=False)["E"] == pytest.approx(6.25 * r["E"], rel=1e-13)
    # dE/dq = phi and F = -dE/dr (central differences of the MSM energy)
    for i in rng.choice(40, 5, replace=False):
        dq = 1e-5
        qp, qm = q.copy(), q.copy()
        qp[i] += dq
        qm[i] -= dq
        fd = (oracle.msm(P, pos, qp, False, False)["E"] - oracle.msm(P, pos, qm, False, False)["E"]) / (2 * dq)
        assert fd == pytest.approx(r["phi"][i], rel=1e-7, abs=1e-8)
        for d in range(3):
            dx = 1e-5
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += dx
            pm[i, d] -= dx
            fd = (oracle.msm(P, pp, q, False, False)["E"] - oracle.msm(P, pm, q, False, False)["E"]) / (2 * dx)
            assert -fd == pytest.approx(r["F"][i, d], rel=1e-5, abs=1e-6)
    # a permutation of atoms permutes the outputs
    perm = rng.permutation(40)
    rp = oracle.msm(P, pos[perm], q[perm])
    assert rp["E"] == pytest.approx(r["E"], rel=1e-13)
    assert np.allclose(rp["phi"], r["phi"][perm], rtol=1e-12, atol=1e-12)
    assert np.allclose(rp["F"], r["F"][perm], rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("pbc", [(1, 1, 1), (0, 0, 0)])
def test_potential_adjoint_against_differences(oracle, pbc):
    """phi = A q with A symmetric, so for L = sum_i g_i phi_i(r, q):
    dL/dq = A g = phi(g) and dL/dr_k = -g_k E_k(q) - q_k E_k(g) with the field
    E = F / q; checked by central differences of the oracle's potentials."""
    rng = np.random.default_rng(15)
    pos, q, cell = _small_periodic()
    if not any(pbc):
        pos = np.clip(pos, 0.5, 8.5)
    P = oracle.make_plan(cell, pbc, 1.2, 3.5, 4)
    g = rng.choice([-1.0, 1.0], len(q)) * rng.uniform(0.5, 1.5, len(q))
    rq = oracle.msm(P, pos, q, True, False)
    rg = oracle.msm(P, pos, g, True, False)
    # symmetry of A: g . A q = q . A g
    assert (g * rq["phi"]).sum() == pytest.approx((q * rg["phi"]).sum(), rel=1e-12)

    def loss(pp, qq):
        return float((g * oracle.msm(P, pp, qq, False, False)["phi"]).sum())

    Eq, Eg = rq["F"] / q[:, None], rg["F"] / g[:, None]
    for i in rng.choice(len(q), 4, replace=False):
        h = 1e-5
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        assert (loss(pos, qp) - loss(pos, qm)) / (2 * h) == pytest.approx(rg["phi"][i], rel=1e-7, abs=1e-8)
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = (loss(pp, q) - loss(pm, q)) / (2 * h)
            assert fd == pytest.approx(-g[i] * Eq[i, d] - q[i] * Eg[i, d], rel=1e-5, abs=1e-6)


@pytest.mark.parametrize("pbc", [(1, 1, 1), (0, 0, 0)])
def test_force_vjp_identities_against_differences(oracle, pbc):
    """For L = sum_k u_k . F_k: dL/dq = -D_u phi (the derivative of the potentials
    when every atom moves along u, by the symmetry of A) and dL/dr = -H u =
    D_u F (the symmetry of the Hessian); both sides by central differences
    of the oracle."""
    rng = np.random.default_rng(16)
    pos, q, cell = _small_periodic()
    if not any(pbc):
        pos = np.clip(pos, 0.5, 8.5)
    P = oracle.make_plan(cell, pbc, 1.2, 3.5, 4)
    u = rng.normal(size=pos.shape)

    def loss(pp, qq):
        return float((u * oracle.msm(P, pp, qq, True, False)["F"]).sum())

    eps = 1e-5
    rp = oracle.msm(P, pos + eps * u, q, True, False)
    rm = oracle.msm(P, pos - eps * u, q, True, False)
    dq_ref = -(rp["phi"] - rm["phi"]) / (2 * eps)
    dr_ref = (rp["F"] - rm["F"]) / (2 * eps)
    for i in rng.choice(len(q), 4, replace=False):
        h = 1e-5
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        assert (loss(pos, qp) - loss(pos, qm)) / (2 * h) == pytest.approx(dq_ref[i], rel=1e-5, abs=1e-6)
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, d] += h
            pm[i, d] -= h
            fd = (loss(pp, q) - loss(pm, q)) / (2 * h)
            assert fd == pytest.approx(dr_ref[i, d], rel=1e-4, abs=1e-5)


def test_ewald2d_alpha_independence_and_gap_limit(oracle):
    """The 2-D Ewald sum of a neutral slab does not depend on the splitting
    parameter, and the 3-D Ewald sum with a vacuum gap plus the slab dipole
    correction 2 pi M_z^2 / V converges to it as the gap grows."""
    rng = np.random.default_rng(17)
    Lx, Ly, n = 10.0, 12.0, 40
    pos = np.column_stack([rng.uniform(0, Lx, n), rng.uniform(0, Ly, n), rng.uniform(0, 6, n)])
    q = np.concatenate([np.ones(n // 2), -np.ones(n // 2)])
    rng.shuffle(q)
    Es = [oracle.ewald2d(Lx, Ly, pos, q, al)[0] for al in (0.4, 0.6, 0.9)]
    assert max(Es) - min(Es) <= 1e-12 * abs(Es[0])
    Mz = (q * pos[:, 2]).sum()
    errs = []
    for gap in (20.0, 40.0, 80.0):
        Lz = 6.0 + gap
        E3 = oracle.ewald_auto((Lx, Ly, Lz), pos, q, forces=False)[0]
        errs.append(abs(E3 + 2 * math.pi / (Lx * Ly * Lz) * Mz ** 2 - Es[0]))
    assert errs[0] > errs[1] > errs[2] and errs[2] <= 1e-9 * abs(Es[0])


def test_slab_top_level_against_ewald2d(oracle):
    """A slab keeps its top level with k_L summed over the 2-D lattice: the MSM
    potentials then match the 2-D Ewald sum to the method's accuracy (as the
    periodic MSM matches the 3-D Ewald sum); dropping the top level, as for
    periodic cells, would leave a 100x larger error."""
    from paper_2510_05961_gb300 import workloads as W
    w = W.random_box(800, seed=41, pbc=(1, 1, 0), p=8, h=1.2, a=10.0)
    pos, q = w.pos.astype(np.float64), w.q.astype(np.float64)
    P = oracle.plan_for(w)
    assert P.top_kept == 1 and P.ncomp == P.nlev
    r = oracle.msm(P, pos, q, forces=False, virial=False)
    E2, phi2 = oracle.ewald2d(w.cell[0], w.cell[1], pos, q)
    rel = np.sqrt(((r["phi"] - phi2) ** 2).mean() / (phi2 ** 2).mean())
    assert rel <= 1e-3 and abs(r["E"] - E2) <= 5e-3 * abs(E2)
    P.ncomp = P.nlev - 1  # the top level left out
    rd = oracle.msm(P, pos, q, forces=False, virial=False)
    assert np.sqrt(((rd["phi"] - phi2) ** 2).mean() / (phi2 ** 2).mean()) >= 20 * rel
    # the lattice-summed top kernel is even in z and smooth through z = 0
    k = [oracle.slab_top(8, 10.0, P.nlev, w.cell[0], w.cell[1], z) for z in (-3.0, -1e-4, 0.0, 1e-4, 3.0)]
    assert k[0] == pytest.approx(k[4], rel=1e-12) and k[1] == pytest.approx(k[3], rel=1e-12)
    assert abs(k[2] - k[1]) <= 1e-6 * abs(k[2])


def test_wire_top_level_strain_derivatives(oracle):
    """dK/d eps of a wire's top level (z periodic) against stencils of a
    strained cell: the diagonal components (the period, the open offsets) and
    the shear of the two open axes; shears with the periodic axis vanish."""
    P = oracle.make_plan((14.0, 15.0, 12.0), (0, 0, 1), 1.5, 4.0, 4)
    l = P.nlev
    for which, (a, b) in zip(range(1, 5), [(0, 0), (1, 1), (2, 2), (0, 1)]):
        dK, _ = oracle.stencil(P, l, which)
        eps = 1e-5
        Ks = []
        for sg in (1, -1):
            G = np.eye(3)
            G[a, b] += sg * eps / (2 if a != b else 1)
            G[b, a] += sg * eps / 2 if a != b else 0
            Ks.append(oracle.stencil(P, l, 0, G)[0])
        fd = (Ks[0] - Ks[1]) / (2 * eps)
        assert np.abs(dK).max() > 0
        assert np.abs(fd - dK).max() <= 1e-5 * np.abs(dK).max(), which
    for which in (5, 6):
        assert np.abs(oracle.stencil(P, l, which)[0]).max() == 0.0


def test_ewald1d_alpha_independence_and_direct_sum(oracle):
    """The 1-D Ewald sum of a neutral wire does not depend on the splitting
    parameter and equals the direct sum over replicas of the cell, whose
    truncation error falls as 1/K^2 (cell-cell terms decay as 1/n^3)."""
    rng = np.random.default_rng(19)
    L, n = 10.0, 12
    pos = np.column_stack([rng.uniform(0, 6, n), rng.uniform(0, 6, n), rng.uniform(0, L, n)])
    q = np.array([1.0, -1.0] * (n // 2))
    rng.shuffle(q)
    Es = [oracle.ewald1d(L, pos, q, al)[0] for al in (0.4, 0.6, 0.9)]
    assert max(Es) - min(Es) <= 1e-12 * abs(Es[0])
    d = pos[None, :, :] - pos[:, None, :]

    def direct(K):
        ns = np.arange(-K, K + 1)
        E = 0.0
        for i in range(n):
            for j in range(n):
                r = np.sqrt(d[i, j, 0] ** 2 + d[i, j, 1] ** 2 + (d[i, j, 2] + ns * L) ** 2)
                if i == j:
                    r = r[ns != 0]
                E += 0.5 * q[i] * q[j] * (1.0 / r).sum()
        return E
    errs = [abs(direct(K) - Es[0]) for K in (250, 1000, 4000)]
    assert errs[0] / errs[1] > 10 and errs[1] / errs[2] > 10 and errs[2] <= 1e-7 * abs(Es[0])
    # potentials: the same sum with the charge of atom 0 as probe
    E0, phi = oracle.ewald1d(L, pos, q)
    assert 0.5 * (q * phi).sum() == pytest.approx(E0, rel=1e-14)


@pytest.mark.parametrize("axis", [2, 0])
def test_wire_top_level_against_ewald1d(oracle, axis):
    """A wire (one periodic axis) keeps its top level with k_L summed over the
    1-D lattice: the MSM potentials then match the 1-D Ewald sum to the
    method's accuracy; dropping the top level leaves a 20x larger error."""
    from paper_2510_05961_gb300 import workloads as W
    pbc = tuple(1 if d == axis else 0 for d in range(3))
    w = W.random_box(500, seed=43, pbc=pbc, p=8, h=1.2, a=10.0)
    pos, q = w.pos.astype(np.float64), w.q.astype(np.float64)
    P = oracle.plan_for(w)
    assert P.top_kept == 1 and P.ncomp == P.nlev
    r = oracle.msm(P, pos, q, forces=False, virial=False)
    E1, phi1 = oracle.ewald1d(w.cell[axis], pos, q, axis=axis)
    rel = np.sqrt(((r["phi"] - phi1) ** 2).mean() / (phi1 ** 2).mean())
    assert rel <= 1e-3 and abs(r["E"] - E1) <= 5e-3 * abs(E1)
    P.ncomp = P.nlev - 1  # the top level left out
    rd = oracle.msm(P, pos, q, forces=False, virial=False)
    assert np.sqrt(((rd["phi"] - phi1) ** 2).mean() / (phi1 ** 2).mean()) >= 20 * rel
    # the lattice-summed top kernel is smooth through rho = 0 and decays like
    # -(2/L) ln rho far from the wire (the 2-D Coulomb law of a line charge)
    k = [oracle.wire_top(8, 10.0, P.nlev, 16.0, x) for x in (0.0, 1e-4, 400.0, 800.0)]
    assert abs(k[1] - k[0]) <= 1e-7 * abs(k[0])
    assert (k[3] - k[2]) == pytest.approx(-2.0 / 16.0 * math.log(2.0), rel=1e-9)


@pytest.mark.parametrize("pbc,perm", [((0, 1, 1), (2, 0, 1)), ((1, 0, 1), (1, 2, 0)), ((1, 0, 0), (2, 0, 1)),
                                      ((0, 1, 0), (1, 2, 0))])
def test_axis_relabelling_invariance(oracle, pbc, perm):
    """Relabelling the axes maps a slab open along x or y onto the slab open
    along z, and a wire along x or y onto the wire along z: the MSM's grids,
    stencils and level sums are per axis, so E, phi, F and W agree to rounding.
    perm[d] is the axis that takes axis d's coordinates."""
    rng = np.random.default_rng(23)
    cell = np.array([14.0, 16.0, 18.0])
    n = 60
    pos = rng.uniform(0.5, 1.0, (n, 3)) * cell * 0.9
    q = rng.normal(size=n)
    q -= q.mean()
    c2 = np.zeros(3)
    p2 = np.zeros_like(pos)
    pbc2 = [0, 0, 0]
    for d in range(3):
        c2[perm[d]] = cell[d]
        p2[:, perm[d]] = pos[:, d]
        pbc2[perm[d]] = pbc[d]
    assert tuple(pbc2) in ((1, 1, 0), (0, 0, 1))
    P1 = oracle.make_plan(tuple(cell), pbc, 1.6, 5.0, 4)
    P2 = oracle.make_plan(tuple(c2), tuple(pbc2), 1.6, 5.0, 4)
    assert P1.top_kept == 1 and P2.top_kept == 1
    r1 = oracle.msm(P1, pos, q)
    r2 = oracle.msm(P2, p2, q)
    assert r2["E"] == pytest.approx(r1["E"], rel=1e-12)
    assert np.allclose(r2["phi"], r1["phi"], rtol=1e-11, atol=1e-12)
    F1 = np.zeros_like(r1["F"])
    W1 = np.zeros((3, 3))
    for d in range(3):
        F1[:, perm[d]] = r1["F"][:, d]
        for e in range(3):
            W1[perm[d], perm[e]] = r1["W"][d, e]
    assert np.allclose(r2["F"], F1, rtol=1e-10, atol=1e-12 * np.abs(F1).max())
    assert np.allclose(r2["W"], W1, rtol=1e-10, atol=1e-12 * np.abs(W1).max())


def test_half_cell_translation_invariance(oracle):
    # shifting a periodic system by L/2 moves every evaluated level by whole points
    pos, q, cell = _small_periodic()
    P = oracle.make_plan(cell, (1, 1, 1), 1.2, 3.5, 4)
    r = oracle.msm(P, pos, q)
    for d in range(3):
        sh = pos.copy()
        sh[:, d] += 4.5
        rs = oracle.msm(P, sh, q)
        assert rs["E"] == pytest.approx(r["E"], rel=1e-12)
        assert np.allclose(rs["F"], r["F"], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("pbc", [(1, 1, 1), (0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 0, 1)])
def test_virial_against_strain_differences(oracle, pbc):
    """W = -dE/d eps under r -> (1+eps) r, A -> (1+eps) A (grid coordinates fixed);
    for slabs and wires this includes the strain derivatives of the lattice-summed
    top level (the period of each periodic axis, the offsets along open ones)."""
    pos, q, cell = _small_periodic()
    if not all(pbc):
        pos = np.clip(pos, 0.5, 8.5)
    P = oracle.make_plan(cell, pbc, 0, 3.5, 4, grid_override=(8, 8, 8))
    r = oracle.msm(P, pos, q)
    for d in range(3):
        es = []
        for s in (+1, -1):
            eps = 1e-6 * s
            c2 = list(cell)
            c2[d] *= 1 + eps
            p2 = pos.copy()
            p2[:, d] *= 1 + eps
            P2 = oracle.make_plan(c2, pbc, 0, 3.5, 4, grid_override=(8, 8, 8))
            es.append(oracle.msm(P2, p2, q, False, False)["E"])
        assert -(es[0] - es[1]) / 2e-6 == pytest.approx(r["W"][d, d], rel=1e-5, abs=1e-7)
    assert np.allclose(r["W"], r["W"].T, rtol=1e-12, atol=1e-12)


def test_strain_derivative_stencils(oracle):
    # off-diagonal dK/d eps against sheared stencils: dK_xy = d K(G) / d eps at G = 1 + eps (xy + yx)/2
    P = oracle.make_plan((11.0,) * 3, (0, 0, 0), 1.1, 2.5, 4, levels=3)
    for which, (a, b) in zip(range(1, 7), [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        dK, _ = oracle.stencil(P, 1, which)
        eps = 1e-6
        G = np.eye(3)
        G[a, b] += eps / (2 if a != b else 1)
        G[b, a] += eps / 2 if a != b else 0
        Kp, _ = oracle.stencil(P, 1, 0, G)
        G = np.eye(3)
        G[a, b] -= eps / (2 if a != b else 1)
        G[b, a] -= eps / 2 if a != b else 0
        Km, _ = oracle.stencil(P, 1, 0, G)
        fd = (Kp - Km) / (2 * eps)
        assert np.abs(fd - dK).max() <= 1e-6 * np.abs(dK).max()


def _read_fd_golden():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fd_rocksalt32.txt")
    rows, vir = [], None
    for ln in open(path):
        if ln.startswith("virial"):
            vir = np.array([float(v) for v in ln.split()[1:]])
        elif ln[:1].isdigit():
            rows.append([float(v) for v in ln.split()])
    rows = np.array(rows)
    return rows[:, 0].astype(int), rows[:, 1:4], rows[:, 4], vir


def test_rocksalt32_gradients_against_stored_differences(oracle):
    """The oracle's analytic gradients on the full 32^3 rock-salt supercell (262,144
    atoms) against central differences of its own energy (tests/golden/fd_rocksalt32.txt,
    written by make_fd_rocksalt32.py beside it): dE/dr = -F and dE/dq = phi at 64
    seeded atoms (Sec. 3.2.2 derivatives) and the six virial components W = -dE/d eps
    from strained cells (sheared ones through the general-cell path)."""
    from paper_2510_05961_gb300 import workloads as W
    idx, dEdr, dEdq, vir = _read_fd_golden()
    w = W.rocksalt(ncell=32)
    P = oracle.make_plan(w.cell, w.pbc, w.h, w.a, w.p, grid_override=(64, 64, 64))
    r = oracle.msm(P, w.pos.astype(np.float64), w.q.astype(np.float64))
    assert np.abs(dEdr + r["F"][idx]).max() <= 5e-6 * np.abs(r["F"][idx]).max()
    assert np.abs(dEdq - r["phi"][idx]).max() <= 1e-6 * np.abs(r["phi"][idx]).max()
    Wr = r["W"]
    ref = np.array([Wr[0, 0], Wr[1, 1], Wr[2, 2], Wr[0, 1], Wr[0, 2], Wr[1, 2]])
    assert np.abs(vir - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("periodic", [True, False], ids=["slab", "open"])
def test_sheet_against_exact_sums(oracle, periodic):
    """A two-dimensional arrangement (charges in the plane z = 0 of a cell 2 A
    thick): the MSM against the 2-D Ewald sum (periodic in x, y) or the direct
    Coulomb sum (open), potentials to the method's accuracy and improving from
    p = 4 to p = 8."""
    from paper_2510_05961_gb300 import workloads as W
    errs = []
    for p, h in [(4, 1.0), (8, 0.8)]:
        w = W.sheet(periodic=periodic, p=p, h=h)
        pos, q = w.pos.astype(np.float64), w.q.astype(np.float64)
        r = oracle.msm(oracle.plan_for(w), pos, q, forces=False, virial=False)
        if periodic:
            _, phi_ref = oracle.ewald2d(w.cell[0], w.cell[1], pos, q)
        else:
            _, phi_ref, _ = oracle.direct_open(pos, q)
        errs.append(np.sqrt(((r["phi"] - phi_ref) ** 2).mean() / (phi_ref ** 2).mean()))
    assert errs[1] < errs[0] and errs[1] < 3e-5 and errs[0] < 2e-4, errs


@pytest.mark.parametrize("periodic", [True, False], ids=["wire", "open"])
def test_chain_against_exact_sums(oracle, periodic):
    """A one-dimensional arrangement (charges on the line x = y = 0): the MSM
    against the 1-D Ewald sum (periodic along z) or the direct Coulomb sum
    (open), improving from p = 4 to p = 8."""
    from paper_2510_05961_gb300 import workloads as W
    errs = []
    for p, h in [(4, 1.0), (8, 0.8)]:
        w = W.chain(periodic=periodic, p=p, h=h)
        pos, q = w.pos.astype(np.float64), w.q.astype(np.float64)
        r = oracle.msm(oracle.plan_for(w), pos, q, forces=False, virial=False)
        if periodic:
            _, phi_ref = oracle.ewald1d(w.cell[2], pos, q, axis=2)
        else:
            _, phi_ref, _ = oracle.direct_open(pos, q)
        errs.append(np.sqrt(((r["phi"] - phi_ref) ** 2).mean() / (phi_ref ** 2).mean()))
    assert errs[1] < errs[0] and errs[1] < 5e-6 and errs[0] < 5e-5, errs
