"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, an independent algorithm (de Casteljau,
angle-sum winding, dense sampling, brute-force tile overlap), a symmetry of the problem, central
finite differences, or a library routine (torch.optim.Adam), chosen so that a dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_2406_04008_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KAPPA = 9.0 / 35.0         # integral over [-1,1] of S(1-S) for S(x) = 1/2 + 3x/4 - x^3/4
S2_NEG = 33.0 / 560.0      # integral over [-1,0] of S^2


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                out[k.strip()] = float(v)
    return out


def _poly_area_perim(v):
    x, y = v[:, 0], v[:, 1]
    xn, yn = np.roll(x, -1), np.roll(y, -1)
    area = 0.5 * abs(np.sum(x * yn - xn * y))
    perim = np.sum(np.hypot(xn - x, yn - y))
    return area, perim


def _square_ring(lo, hi):
    return [np.array([(lo, lo), (hi, lo), (hi, hi), (lo, hi)])]


def _params(rows):
    return np.asarray(rows, np.float64).reshape(-1)


# ------------------------------------------------------------------------------------------------
def test_constants_match_paper(oracle_mod):
    g = _golden("paper_constants.txt")
    o = oracle_mod.options()
    assert (o.alpha, o.beta, o.gamma) == (g["alpha"], g["beta"], g["gamma"])
    assert (o.w_in, o.w_out) == (g["w_in"], g["w_out"])


def _de_casteljau(P, t):
    pts = [np.asarray(p, float) for p in P]
    while len(pts) > 1:
        pts = [(1 - t) * pts[i] + t * pts[i + 1] for i in range(len(pts) - 1)]
    return pts[0]


def test_flatten_matches_de_casteljau(oracle_mod):
    rng = W.PCG32(7)
    ctrl = W.blob_controls(rng, 0.05)
    prob = W.make_problem([(0, ctrl, 0.0)], _square_ring(0.1, 0.9), [(0.5, 0.5, 0.0, 1.0)], 64)
    sc = oracle_mod.Scene(prob, segs_per_cubic=16)
    v = sc.local_vertices(0)
    c32 = ctrl.astype(np.float32).astype(np.float64)
    ref = []
    for k in range(8):
        P = [c32[(3 * k + i) % 24] for i in range(4)]
        for j in range(16):
            ref.append(_de_casteljau(P, j / 16.0))
    np.testing.assert_allclose(v, np.array(ref), atol=1e-15, rtol=0)


def _angle_winding(p, v):
    a = v - p
    b = np.roll(a, -1, axis=0)
    ang = np.arctan2(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0], np.sum(a * b, 1))
    return int(round(ang.sum() / (2 * np.pi)))


def _dense_distance(p, v, closed, n=4000):
    segs = len(v) if closed else len(v) - 1
    u = np.linspace(0.0, 1.0, n)[:, None]
    best = np.inf
    for j in range(segs):
        a, b = v[j], v[(j + 1) % len(v)]
        pts = a + u * (b - a)
        best = min(best, np.min(np.hypot(pts[:, 0] - p[0], pts[:, 1] - p[1])))
    return best


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_signed_distance_brute_force(oracle_mod, kind):
    rng = W.PCG32(11 + kind)
    if kind == 0:
        shape, hw = W.blob_controls(rng, 0.3), 0.0
    elif kind == 1:
        shape, hw = W.convex_polygon(rng, 0.3, 9), 0.0
    else:
        shape, hw = W.polyline(rng, 0.3, 7), 0.03
    q = (0.5, 0.48, 0.3, 1.1)
    prob = W.make_problem([(kind, shape, hw)], _square_ring(0.0, 1.0), [q], 8)
    hw = float(np.float32(hw))  # the problem stores the half-width in float32
    sc = oracle_mod.Scene(prob)
    wv = sc.world_vertices(_params(q), 0)
    # the 8x8 pixel centres plus random points around the outline
    pts = [((j + 0.5) / 8, (i + 0.5) / 8) for i in range(8) for j in range(8)]
    pts += [(rng.uniform(0.05, 0.95), rng.uniform(0.05, 0.95)) for _ in range(40)]
    pts = np.array(pts)
    sd, seg, u = sc.sd(_params(q), 0, pts)
    for p, s in zip(pts, sd):
        d = _dense_distance(p, wv, kind != 2)
        if kind == 2:
            ref = hw - d
        else:
            ref = d if _angle_winding(p, wv) != 0 else -d
        # dense sampling overestimates the distance by at most half a sample spacing
        assert abs(abs(s) - abs(ref)) < 2e-5 and (s > 0) == (ref > 0), (p, s, ref)
    # the reported closest segment and parameter reproduce the distance exactly
    for p, s, j, uu in zip(pts, sd, seg, u):
        a, b = wv[j], wv[(j + 1) % len(wv)]
        q_ = a + uu * (b - a)
        d = math.hypot(p[0] - q_[0], p[1] - q_[1])
        assert abs(d - (hw - s if kind == 2 else abs(s))) < 1e-14


@pytest.mark.parametrize("shape", ["square_rot", "convex9", "ngon12"])
def test_area_from_coverage(oracle_mod, shape):
    rng = W.PCG32(21)
    if shape == "square_rot":
        v, th = np.array([(-0.15, -0.15), (0.15, -0.15), (0.15, 0.15), (-0.15, 0.15)]), 0.3
    elif shape == "convex9":
        v, th = W.convex_polygon(rng, 0.2, 9), 0.0
    else:
        v, th = W.regular_polygon(0.2, 12), 0.1
    q = (0.5, 0.5, th, 1.0)
    prob = W.make_problem([(1, v, 0.0)], _square_ring(0.0, 1.0), [q], 256)
    sc = oracle_mod.Scene(prob)
    area_ref, _ = _poly_area_perim(v.astype(np.float32).astype(np.float64))
    errs = []
    for R in (256, 512):
        ihat, atau, _ = sc.render(_params(q), R, oracle_mod.options())
        errs.append(abs((1 - ihat).sum() / R ** 2 - area_ref) / area_ref)
        # one opaque item with tau: A_tau = tau * c exactly
        np.testing.assert_allclose(atau, 0.5 * (1 - ihat), atol=1e-15)
    assert errs[1] < 2e-4, errs


def test_disk_area_converges_to_pi_r2(oracle_mod):
    r = 0.2
    prob = W.make_problem([(1, W.regular_polygon(r, 1024), 0.0)], _square_ring(0.0, 1.0),
                          [(0.5, 0.5, 0.0, 1.0)], 512)
    sc = oracle_mod.Scene(prob)
    ihat, _, _ = sc.render(_params((0.5, 0.5, 0.0, 1.0)), 512, oracle_mod.options())
    assert abs((1 - ihat).sum() / 512 ** 2 - np.pi * r * r) / (np.pi * r * r) < 1e-4


def test_stroke_area_is_capsule(oracle_mod):
    # one-segment open polyline of half-width hw: area 2 hw L + pi hw^2
    L, hw = 0.5, 0.04
    prob = W.make_problem([(2, np.array([(-L / 2, 0.0), (L / 2, 0.0)]), hw)],
                          _square_ring(0.0, 1.0), [(0.5, 0.5, 0.4, 1.0)], 512)
    sc = oracle_mod.Scene(prob)
    ihat, _, _ = sc.render(_params((0.5, 0.5, 0.4, 1.0)), 512, oracle_mod.options())
    hw32 = float(np.float32(hw))
    ref = 2 * hw32 * L + np.pi * hw32 ** 2
    assert abs((1 - ihat).sum() / 512 ** 2 - ref) / ref < 2e-4


def test_padding_is_outward_offset(oracle_mod):
    # padded overlap render of one convex polygon covers A + P pad + pi pad^2 (Steiner formula)
    v = W.regular_polygon(0.2, 12)
    R, pad_px = 512, 6.0
    q = (0.5, 0.5, 0.1, 1.0)
    prob = W.make_problem([(1, v, 0.0)], _square_ring(0.0, 1.0), [q], R)
    sc = oracle_mod.Scene(prob)
    _, atau, _ = sc.render(_params(q), R, oracle_mod.options(pad_px=pad_px))
    A, P = _poly_area_perim(v.astype(np.float32).astype(np.float64))
    pad = pad_px / R
    ref = A + P * pad + np.pi * pad * pad
    got = (atau / 0.5).sum() / R ** 2
    assert abs(got - ref) / ref < 2e-4
    assert abs(got - A) / A > 0.05  # the padding is visible at this size


def test_containment_closed_forms(oracle_mod):
    R = 512
    ring = W.regular_polygon(0.3, 256) + (0.5, 0.5)
    disk = W.regular_polygon(0.1, 64)
    A_C, P_C = _poly_area_perim(ring.astype(np.float32).astype(np.float64))
    A_e, P_e = _poly_area_perim(disk.astype(np.float32).astype(np.float64))
    o = oracle_mod.options(gamma=0.0)
    o1 = oracle_mod.options(gamma=0.0, w_out=1.0)
    dlt = 1.0 / R

    def lc(params, els, opts=o):
        prob = W.make_problem(els, [ring], params, R)
        return oracle_mod.Scene(prob).eval(_params(params), R, opts, grad=False)["terms"][0]

    far = [(5.0, 5.0, 0.0, 1e-3)]  # a speck far outside the image: Ihat = 1 everywhere
    speck = [(1, W.regular_polygon(1e-4, 8), 0.0)]
    # empty container with W = 1: sum cov^2 = sum cov - sum cov(1-cov) = A_C - kappa P_C dlt
    empty1 = lc(far, speck, o1)
    ref1 = A_C - KAPPA * P_C * dlt
    assert abs(empty1 - ref1) / ref1 < 1e-4, (empty1, ref1)  # the kappa term is 3.4e-3
    # with w_out = 100 the band where cov < 1/2 gains 99 cov^2; W jumps there, so the pixel sum
    # carries lattice-count noise and is checked against the image and loosely against the integral
    empty = lc(far, speck)
    _, _, cov = oracle_mod.Scene(W.make_problem(speck, [ring], far, R)).render(
        _params(far[0]), R, o)
    band = (cov[cov < 0.5] ** 2).sum() * dlt * dlt
    assert abs((empty - empty1) - 99.0 * band) < 1e-12
    assert abs(band / (S2_NEG * P_C * dlt) - 1.0) < 0.15
    inside = lc([(0.5, 0.5, 0.0, 1.0)], [(1, disk, 0.0)])
    outside = lc([(0.09, 0.09, 0.0, 0.5)], [(1, disk, 0.0)])
    # a disk inside removes sum (2c - c^2) = A_e + kappa P_e dlt
    ref_in = A_e + KAPPA * P_e * dlt
    assert abs((empty - inside) - ref_in) / ref_in < 1e-3
    # a half-size disk outside adds w_out * sum c^2 = 100 (A_e' - kappa P_e' dlt)
    ref_out = 100.0 * (A_e / 4 - KAPPA * P_e / 2 * dlt)
    assert abs((outside - empty) - ref_out) / ref_out < 1e-3


def _lens(r1, r2, d):
    a1 = r1 * r1 * math.acos((d * d + r1 * r1 - r2 * r2) / (2 * d * r1))
    a2 = r2 * r2 * math.acos((d * d + r2 * r2 - r1 * r1) / (2 * d * r2))
    k = math.sqrt((-d + r1 + r2) * (d + r1 - r2) * (d - r1 + r2) * (d + r1 + r2))
    return a1 + a2 - 0.5 * k, k / d  # area, chord length = -d(area)/dd


def _shift_average(fn, R, K=32, L=13):
    """Mean of fn(dx, dy) over K sub-pixel shifts on a rank-1 lattice (k, L k mod K) / (K R).

    Sampling the 2-px-wide filter on the pixel grid adds terms periodic in the sub-pixel offset,
    one per 2-D harmonic m = (mx, my) with phase exp(2 pi i m . shift R).  The lattice average
    cancels every harmonic with mx + L my != 0 (mod K), which leaves only high orders; values then
    match the continuum to the order of those harmonics, derivatives (one factor |m| more) less well.
    """
    return np.mean([fn(k / (K * R), ((k * L) % K) / (K * R)) for k in range(K)], axis=0)


def test_overlap_lens_area_and_derivative(oracle_mod):
    R, r1, r2, d, tau = 512, 0.15, 0.12, 0.2, 0.5
    o = oracle_mod.options(alpha=0.0, beta=1.0, gamma=0.0, tau=tau)

    def run(dx, dy):
        params = [(0.5 - d / 2 + dx, 0.5 + dy, 0.0, 1.0), (0.5 + d / 2 + dx, 0.5 + dy, 0.0, 1.0)]
        prob = W.make_problem([(1, W.regular_polygon(r1, 1024), 0.0),
                               (1, W.regular_polygon(r2, 1024), 0.0)],
                              _square_ring(-1.0, 2.0), params, R)
        out = oracle_mod.Scene(prob).eval(_params(params), R, o)
        return np.concatenate([[out["terms"][1]], out["grad_a"]])

    res = _shift_average(run, R)
    area, chord = _lens(float(np.float32(r1)), float(np.float32(r2)), d)
    k = tau * (1 - tau)
    # inside the lens A_tau - tau = tau(1 - tau); wh * dlt^2 = 1 on the unit square
    assert abs(res[0] / k - area) / area < 1e-3
    g = res[1:].reshape(2, 4)
    # moving disk 1 right shrinks the separation: dL/dt1x = tau(1-tau) * chord
    assert abs(g[0, 0] / k - chord) / chord < 2e-3
    assert abs(g[1, 0] / k + chord) / chord < 2e-3
    assert abs(g[0, 1]) < 2e-3 * chord * k and abs(g[1, 1]) < 2e-3 * chord * k


def test_distribution_term_integer_case(oracle_mod):
    # rho = 0.25 px and a pixel-aligned 4x4 block: every coverage is exactly 0 or 1, so
    # min(1, box sum) = 1 exactly where the window meets the block (Chebyshev distance <= r_k)
    g = _golden("paper_constants.txt")
    R = 16
    blk = np.array([(0.0, 0.0), (4.0, 0.0), (4.0, 4.0), (0.0, 4.0)]) / R
    q = (4.0 / R, 5.0 / R, 0.0, 1.0)  # block covers pixel columns 4..7 and rows 5..8
    prob = W.make_problem([(1, blk, 0.0)], _square_ring(-0.5, 1.5), [q], R)
    sc = oracle_mod.Scene(prob)
    wts = (1.0, 2.0, 3.0, 4.0)
    o = oracle_mod.options(alpha=0.0, beta=0.0, gamma=1.0, rho_px=0.25, dil_weight=wts)
    ihat, _, _ = sc.render(_params(q), R, o)
    occ = 1 - ihat
    assert set(np.unique(occ)) == {0.0, 1.0} and occ.sum() == 16
    ref = 0.0
    for k in range(4):
        width = g["dil_first_width"] + g["dil_width_step"] * k
        r = int((width - 1) // 2)
        for i in range(R):
            for j in range(R):
                di = max(5 - i, 0, i - 8)
                dj = max(4 - j, 0, j - 7)
                if occ[i, j] == 0 and max(di, dj) > r:
                    ref += wts[k]
    out = sc.eval(_params(q), R, o, grad=False)
    assert out["terms"][2] == ref and ref > 0


def test_distribution_gradient_central_differences(oracle_mod):
    # dL_u/dO of Eq. 7 (the adjoint the allocation-free call and the raster adjoint consume)
    # against central differences of L_u in every pixel of a 14 x 14 image.  L_u is a polynomial
    # of degree 2 in each O(q) away from the kinks of min(1, B_k), so the differences are exact up
    # to rounding; pixels whose windows hold a box sum within 4h of 1 are skipped.  Occupancies are
    # small (mostly B_k < 1) with a dense patch (B_k > 1 there), so both branches of the min occur.
    rng = np.random.default_rng(11)
    R, h = 14, 1e-6
    occ = rng.uniform(0.0, 0.03, (R, R))
    occ[2:6, 8:12] = rng.uniform(0.3, 1.0, (4, 4))
    cov = np.clip(rng.uniform(-0.3, 1.3, (R, R)), 0.0, 1.0)
    wts = (1.0, 2.5, 4.0)
    lu, gou = oracle_mod.uniform_term(occ, cov, wts)

    def box(img, r):
        p = np.pad(img, r)
        return np.array([[p[i:i + 2 * r + 1, j:j + 2 * r + 1].sum() for j in range(R)] for i in range(R)])

    B = [box(occ, 2 + 3 * k) for k in range(len(wts))]
    assert any((b > 1).any() for b in B) and any((b < 1).any() for b in B)
    checked = 0
    for i in range(R):
        for j in range(R):
            near_kink = any(np.abs(B[k][max(i - r, 0):i + r + 1, max(j - r, 0):j + r + 1] - 1).min() < 4 * h
                            for k, r in enumerate(2 + 3 * k for k in range(len(wts))))
            if near_kink:
                continue
            a, b = occ.copy(), occ.copy()
            a[i, j] += h
            b[i, j] -= h
            fd = (oracle_mod.uniform_term(a, cov, wts, grad=False)[0] -
                  oracle_mod.uniform_term(b, cov, wts, grad=False)[0]) / (2 * h)
            assert abs(fd - gou[i, j]) <= 1e-6 * max(1.0, abs(gou[i, j])), (i, j, fd, gou[i, j])
            checked += 1
    assert checked > R * R // 2


def test_distribution_term_alone_equals_full_evaluation(oracle_mod):
    # the standalone Eq. 7 entry gives the L_u of the full loss evaluation on the same render
    prob = W.config_problem(1, n_elems=10, grid=64)
    sc = oracle_mod.Scene(prob)
    o = oracle_mod.options(n_dil=3, dil_weight=(1.0, 2.0, 3.0))
    q = prob["params0"].astype(np.float64)
    ihat, _, cov = sc.render(q, 64, o)
    lu, _ = oracle_mod.uniform_term(1.0 - ihat, cov, (1.0, 2.0, 3.0), grad=False)
    assert lu == sc.eval(q, 64, o, grad=False)["terms"][2] and lu > 0


def _rot_problem(prob, params):
    """The same scene rotated by 90 degrees about (1/2, 1/2): (x, y) -> (1 - y, x)."""
    q = params.reshape(-1, 4).copy()
    q2 = np.stack([1.0 - q[:, 1], q[:, 0], q[:, 2] + np.pi / 2, q[:, 3]], 1)
    rp = prob["ring_pts"].reshape(-1, 2).astype(np.float64)
    rp2 = np.stack([1.0 - rp[:, 1], rp[:, 0]], 1)
    p2 = dict(prob)
    p2["ring_pts"] = rp2.astype(np.float32).reshape(-1)
    assert np.array_equal(p2["ring_pts"].astype(np.float64), rp2.reshape(-1))
    return p2, q2.reshape(-1)


def test_invariance_pixel_shift_and_quarter_turn(oracle_mod):
    R = 128
    # dyadic container so that shifted / rotated copies are exact in float32
    ring = np.array([(24, 20), (100, 28), (108, 96), (60, 110), (18, 80)], float) / 128
    els, params = [], []
    rng = W.PCG32(31)
    for k in range(5):
        els.append((k % 3, [W.blob_controls(rng, 0.08), W.convex_polygon(rng, 0.07, 7),
                            W.polyline(rng, 0.07, 5)][k % 3], 0.01 if k % 3 == 2 else 0.0))
        params.append((0.3 + 0.1 * k, 0.35 + 0.07 * k, 0.4 * k, 0.9 + 0.05 * k))
    prob = W.make_problem(els, [ring], params, R)
    q = _params(params)
    o = oracle_mod.options(pad_px=1.5)
    base = oracle_mod.Scene(prob).eval(q, R, o)
    # shift by 3 whole pixels in x
    shifted = dict(prob)
    shifted["ring_pts"] = (prob["ring_pts"].reshape(-1, 2) + (3.0 / R, 0.0)).astype(
        np.float32).reshape(-1)
    qs = q.reshape(-1, 4).copy()
    qs[:, 0] += 3.0 / R
    sh = oracle_mod.Scene(shifted).eval(qs.reshape(-1), R, o)
    np.testing.assert_allclose(sh["terms"], base["terms"], rtol=1e-11)
    np.testing.assert_allclose(sh["grad_a"], base["grad_a"], rtol=1e-8,
                               atol=1e-9 * np.abs(base["grad_a"]).max())
    # quarter turn: losses equal (no force term), translation gradients rotate
    p2, q2 = _rot_problem(prob, q)
    rot = oracle_mod.Scene(p2).eval(q2, R, o)
    keep = [0, 1, 2, 4]  # the force term (index 3) depends on y and has weight 0 here
    np.testing.assert_allclose(rot["terms"][keep], base["terms"][keep], rtol=1e-11)
    g0, g1 = base["grad_a"].reshape(-1, 4), rot["grad_a"].reshape(-1, 4)
    sc = 1e-8 * np.abs(g0).max()
    np.testing.assert_allclose(g1[:, 0], -g0[:, 1], atol=sc)
    np.testing.assert_allclose(g1[:, 1], g0[:, 0], atol=sc)
    np.testing.assert_allclose(g1[:, 2:], g0[:, 2:], atol=sc)


def test_force_term_closed_form(oracle_mod):
    R, r, yc = 256, 0.15, 0.3
    o = oracle_mod.options(alpha=0, beta=0, gamma=0, delta=1.0)

    def run(dx, dy):
        q = (0.5 + dx, yc + dy, 0.0, 1.0)
        prob = W.make_problem([(1, W.regular_polygon(r, 512), 0.0)], _square_ring(-1, 2), [q], R)
        out = oracle_mod.Scene(prob).eval(_params(q), R, o)
        return np.concatenate([[out["terms"][3], yc + dy], out["grad_a"]])

    res = _shift_average(run, R)
    A = np.pi * float(np.float32(r)) ** 2
    y = res[1]
    assert abs(res[0] - A * (1 - y)) / (A * (1 - y)) < 1e-3
    # dL/dty = -area (moving down lowers the potential), dL/dtx = 0, dL/ds = 2 A (1 - yc)
    g = res[2:]
    assert abs(g[1] + A) / A < 2e-3 and abs(g[0]) < 1e-3 * A
    assert abs(g[3] - 2 * A * (1 - y)) / (2 * A * (1 - y)) < 2e-3


def _point_potential(D, rr):
    """Integral of |p - c| over a disk of radius rr whose centre lies at distance D from c, and
    its derivatives in D and rr, by Gauss-Legendre quadrature in polar coordinates about the
    disk's centre (independent of the oracle)."""
    from numpy.polynomial.legendre import leggauss
    xr, wr = leggauss(64)
    xt, wt = leggauss(128)
    rho = 0.5 * rr * (xr + 1.0)
    th = np.pi * (xt + 1.0)
    P, TH = np.meshgrid(rho, th, indexing="ij")
    Wt = np.outer(wr * 0.5 * rr, wt * np.pi)
    dist = np.sqrt(D * D + P * P + 2 * D * P * np.cos(TH))
    phi = np.sum(Wt * dist * P)
    dphi_dD = np.sum(Wt * (D + P * np.cos(TH)) / np.maximum(dist, 1e-300) * P)
    # d/drr: the boundary integral of |p - c| over the circle of radius rr
    ring = np.sqrt(D * D + rr * rr + 2 * D * rr * np.cos(th))
    dphi_dr = np.sum(wt * np.pi * ring) * rr
    return phi, dphi_dD, dphi_dr


def test_point_force_closed_form(oracle_mod):
    """Force towards a point (Sec. 5, force attraction): for a disk the term is the integral of
    |p - c| over the disk, whose value and derivatives come from quadrature; at D = 0 the value is
    2 pi r^3 / 3 and the translation gradient vanishes by symmetry."""
    R, r = 512, 0.12
    c = (0.5, 0.5)
    rr = float(np.float32(r))
    for D in (0.0, 0.2):
        def run(dx, dy):  # the element and the force point move together
            o = oracle_mod.options(alpha=0, beta=0, gamma=0, delta=1.0, force_kind=1,
                                   force_x=c[0] + dx, force_y=c[1] + dy)
            q = (c[0] + D + dx, c[1] + dy, 0.0, 1.0)
            prob = W.make_problem([(1, W.regular_polygon(r, 1024), 0.0)], _square_ring(-1, 2), [q], R)
            out = oracle_mod.Scene(prob).eval(_params(q), R, o)
            return np.concatenate([[out["terms"][3]], out["grad_a"]])

        res = _shift_average(run, R)
        phi, dD, dr = _point_potential(D, rr)
        # the smoothstep filter adds 0.6 (rho / r)^2 relative at a circle centred on c (its first
        # moment across the edge); the bound leaves room for it
        assert abs(res[0] - phi) / phi < 2.5e-4, (D, res[0], phi)
        g = res[1:]
        scale = abs(dr)
        assert abs(g[0] - dD) < 3e-3 * scale, (D, g[0], dD)
        assert abs(g[1]) < 3e-3 * scale
        assert abs(g[3] - dr * rr) / (dr * rr) < 3e-3, (D, g[3], dr * rr)  # radius = s r
        if D == 0.0:
            assert abs(phi - 2 * np.pi * rr ** 3 / 3) / phi < 1e-9
            g0 = run(0.0, 0.0)[1:]  # centred on a pixel corner: mirror-symmetric sampling
            assert abs(g0[0]) < 1e-9 * scale and abs(g0[1]) < 1e-9 * scale


def _small_scene(oracle_mod, seed=41, n=6, R=96):
    rng = W.PCG32(seed)
    els, params = [], []
    for k in range(n):
        kind = k % 3
        shape = [W.blob_controls(rng, 0.09), W.convex_polygon(rng, 0.08, 6),
                 W.polyline(rng, 0.09, 6)][kind]
        els.append((kind, shape, 0.012 if kind == 2 else 0.0))
        params.append((0.3 + 0.4 * rng.uniform(), 0.3 + 0.4 * rng.uniform(),
                       rng.uniform(0, 6.28), 0.8 + 0.4 * rng.uniform()))
    prob = W.make_problem(els, W.star_container(rng, r_in=0.3, r_out=0.45), params, R)
    return oracle_mod.Scene(prob), _params(params)


def test_gradient_routes_agree(oracle_mod):
    sc, q = _small_scene(oracle_mod)
    out = sc.eval(q, 96, oracle_mod.options(pad_px=1.0, delta=50.0))
    np.testing.assert_allclose(out["grad_a"], out["grad_b"], rtol=0,
                               atol=1e-10 * np.abs(out["grad_a"]).max())


def test_gradient_routes_agree_with_point_force(oracle_mod):
    sc, q = _small_scene(oracle_mod, seed=43)
    out = sc.eval(q, 96, oracle_mod.options(pad_px=1.0, delta=50.0, force_kind=1, force_x=0.4,
                                            force_y=0.55))
    np.testing.assert_allclose(out["grad_a"], out["grad_b"], rtol=0,
                               atol=1e-10 * np.abs(out["grad_a"]).max())


def test_gradient_central_differences(oracle_mod):
    R = 96
    sc, q = _small_scene(oracle_mod, R=R)
    o = oracle_mod.options(pad_px=1.0, delta=50.0)
    g = sc.eval(q, R, o)["grad_a"]
    h = 1e-6
    fd = np.zeros_like(q)
    for k in range(len(q)):
        qp, qm = q.copy(), q.copy()
        qp[k] += h
        qm[k] -= h
        fd[k] = (sc.eval(qp, R, o, grad=False)["terms"][4] -
                 sc.eval(qm, R, o, grad=False)["terms"][4]) / (2 * h)
    g4, f4 = g.reshape(-1, 4), fd.reshape(-1, 4)
    for t in range(4):
        floor = 1e-2 * np.abs(g4[:, t]).max()
        err = np.abs(g4[:, t] - f4[:, t]) / np.maximum(np.abs(g4[:, t]), floor)
        assert err.max() < 1e-3, (t, err, g4[:, t], f4[:, t])


def test_cull_is_exact(oracle_mod):
    sc, q = _small_scene(oracle_mod, seed=43)
    a = sc.eval(q, 96, oracle_mod.options(pad_px=2.0, cull=1))
    b = sc.eval(q, 96, oracle_mod.options(pad_px=2.0, cull=0))
    assert np.array_equal(a["terms"], b["terms"])
    assert np.array_equal(a["grad_a"], b["grad_a"])


def test_adam_matches_torch(oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    p0 = rng.normal(size=12)
    p0[3::4] = 1.0
    grads = [rng.normal(size=12) for _ in range(3)]
    tp = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(12), np.zeros(12)
    for k, g in enumerate(grads):
        opt.zero_grad()
        tp.grad = torch.tensor(g)
        opt.step()
        p, m, v = oracle_mod.adam(p, m, v, g, k + 1, s_min=-1e9, s_max=1e9)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=0, atol=1e-15)
    # frozen entries stay put and s is clamped
    tr = np.ones(12, np.uint8)
    tr[0] = 0
    p2, _, _ = oracle_mod.adam(p0, np.zeros(12), np.zeros(12), np.ones(12), 1, lr=10.0,
                               trainable=tr, s_min=0.5, s_max=2.0)
    assert p2[0] == p0[0] and np.all(p2[3::4] == 0.5)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_bins_rule_equals_brute_force_and_is_conservative(oracle_mod, tile):
    rng = W.PCG32(51)
    R = 200  # ragged: not a multiple of the tile
    els, params = [], []
    for k in range(12):
        kind = k % 3
        shape = [W.blob_controls(rng, 0.06), W.convex_polygon(rng, 0.05, 8),
                 W.polyline(rng, 0.06, 5)][kind]
        els.append((kind, shape, 0.01 if kind == 2 else 0.0))
        params.append((rng.uniform(-0.05, 1.05), rng.uniform(-0.05, 1.05), rng.uniform(0, 6.3),
                       rng.uniform(0.5, 1.5)))
    prob = W.make_problem(els, _square_ring(0.0, 1.0), params, R)
    sc = oracle_mod.Scene(prob)
    p32 = np.asarray(params, np.float32).reshape(-1)
    t1, e1 = sc.bins(p32, R, tile, 1.0, 2.0)
    t2, e2 = sc.bins(p32, R, tile, 1.0, 2.0, brute=True)
    assert np.array_equal(t1, t2) and np.array_equal(e1, e2) and len(t1) > 0
    # every pixel where an element has nonzero (padded) coverage lies in one of its tiles
    nt = (R + tile - 1) // tile
    xy = np.array([((j + 0.5) / R, (i + 0.5) / R) for i in range(R) for j in range(R)])
    q64 = p32.astype(np.float64)
    for e in range(len(els)):
        sd, _, _ = sc.sd(q64, e, xy)
        live = np.nonzero(sd + 3.0 / R > -1e-12)[0]  # rho + pad = 3 px
        tiles = set(t1[e1 == e].tolist())
        need = {(i // R // tile) * nt + (i % R) // tile for i in live}
        assert need <= tiles, (e, sorted(need - tiles))


# ------------------------------------------------------------------------------------------------
# Quality metrics (Sec. 6 "Metrics of Collage Quality"; L-nU of the Sec. 6.1 ablation)
def _disk_scene_masks(disks, box, R):
    """Object, overlap and shape masks of disks in a square container, from the circles' own
    signed distances (numpy), with the renderer's composite O = 1 - prod(1 - S(sd/rho))."""
    yy, xx = np.mgrid[0:R, 0:R]
    px, py = (xx + 0.5) / R, (yy + 0.5) / R
    rho = 1.0 / R

    def S(x):
        x = np.clip(x, -1, 1)
        return 0.5 + 0.75 * x - 0.25 * x ** 3

    keep = np.ones((R, R))
    n_in = np.zeros((R, R), int)
    for cx, cy, r in disks:
        sd = r - np.hypot(px - cx, py - cy)
        keep *= 1 - S(sd / rho)
        n_in += sd >= 0
    lo, hi = box
    shape = (px >= lo) & (px <= hi) & (py >= lo) & (py <= hi)
    return 1 - keep >= 0.5, n_in >= 2, shape


def test_metrics_counts_match_masks(oracle_mod):
    R = 200
    disks = [(0.4, 0.5, 0.15), (0.62, 0.47, 0.12), (0.3, 0.28, 0.05)]
    box = (0.2, 0.7)
    prob = W.make_problem([(1, W.regular_polygon(r, 2048), 0.0) for _, _, r in disks],
                          _square_ring(*box), [(cx, cy, 0.0, 1.0) for cx, cy, _ in disks], R)
    out = oracle_mod.Scene(prob).metrics(_params([(cx, cy, 0.0, 1.0) for cx, cy, _ in disks]), R,
                                         oracle_mod.options())
    obj, over, shape = _disk_scene_masks(disks, box, R)
    assert out[0] == (obj & shape).sum() and out[1] == shape.sum()
    assert out[2] == over.sum() and out[3] == (obj & ~shape).sum()
    assert out[3] > 0 and out[2] > 0  # the case exercises both
    assert abs(out[4] - out[0] / out[1]) < 1e-15 and abs(out[5] - out[2] / out[1]) < 1e-15
    assert abs(out[6] - out[3] / out[1]) < 1e-15


def test_layout_nonuniformity_matches_brute_force(oracle_mod):
    R = 48
    rng = W.PCG32(91)
    disks = [(0.25 + 0.5 * rng.uniform(), 0.25 + 0.5 * rng.uniform(), 0.03 + 0.04 * rng.uniform())
             for _ in range(5)]
    box = (0.1, 0.9)
    prob = W.make_problem([(1, W.regular_polygon(r, 2048), 0.0) for _, _, r in disks],
                          _square_ring(*box), [(cx, cy, 0.0, 1.0) for cx, cy, _ in disks], R)
    out = oracle_mod.Scene(prob).metrics(_params([(cx, cy, 0.0, 1.0) for cx, cy, _ in disks]), R,
                                         oracle_mod.options())
    obj, _, shape = _disk_scene_masks(disks, box, R)
    assert out[0] == (obj & shape).sum() and out[3] == (obj & ~shape).sum()
    oy, ox = np.nonzero(obj)
    fy, fx = np.nonzero(shape & ~obj)
    d2 = ((fy[:, None] - oy[None, :]) ** 2 + (fx[:, None] - ox[None, :]) ** 2).min(1)
    assert abs(out[7] - d2.mean() / R ** 2) <= 1e-12 * out[7]


# ---- outline fitting (Sec. 3, Vector Representation): gradients of the points ------------------
def _fit_loss(oracle_mod, **extra):
    return oracle_mod.options(**dict(W.FIT_LOSS, **extra))


def test_bernstein_weights_reproduce_oracle_flattening(oracle_mod):
    # the weights control_grad takes transposed are the ones the oracle flattens with
    prob = W.fit_problem(1, n_cubics=7, grid=64)
    sc = oracle_mod.Scene(prob, segs_per_cubic=12)
    P = np.asarray(prob["pts"], np.float64).reshape(-1, 2)
    w = oracle_mod.bernstein_weights(12)
    v = np.concatenate([w @ P[[3 * c, 3 * c + 1, 3 * c + 2, (3 * c + 3) % len(P)]]
                        for c in range(len(P) // 3)])
    np.testing.assert_allclose(sc.local_vertices(0), v, rtol=0, atol=1e-15)


def test_control_grad_central_differences(oracle_mod):
    R = 64
    prob = W.fit_problem(0, n_cubics=20, grid=R)
    o = _fit_loss(oracle_mod)
    g, _ = oracle_mod.control_grad(prob, prob["params0"], R, o)
    P = np.asarray(prob["pts"], np.float64).reshape(-1, 2)

    def loss(pp):
        pr = dict(prob)
        pr["pts"] = pp.reshape(-1).astype(np.float32)
        return oracle_mod.Scene(pr).eval(prob["params0"], R, o, grad=False)["terms"][4]

    floor = 1e-2 * np.abs(g).max()
    for k in (0, 1, 2, 5, 17, 30, 44, 59):
        for c in range(2):
            # the points are float32: step between float32 neighbours of the point
            a, b = P.copy(), P.copy()
            a[k, c] += 1e-4
            b[k, c] -= 1e-4
            a, b = (x.astype(np.float32).astype(np.float64) for x in (a, b))
            fd = (loss(a) - loss(b)) / (a[k, c] - b[k, c])
            assert abs(g[k, c] - fd) <= 1e-4 * max(abs(fd), floor), (k, c, g[k, c], fd)


@pytest.mark.parametrize("force_kind", [0, 1])
def test_control_grad_rigid_motions(oracle_mod, force_kind):
    # moving every point of an element by a rigid motion or a scaling about its origin moves the
    # element as its transform would: sum_k dP_k = s R^T dL/dt, sum_k (J P_k) . dP_k = dL/dtheta,
    # sum_k P_k . dP_k = s dL/ds, against the spatial-gradient route of the transform gradient
    R = 96
    rng = W.PCG32(47)
    els, params = [], []
    for k in range(6):
        kind = k % 3
        r = 0.05 + 0.05 * rng.uniform()
        shape = (W.blob_controls(rng, r) if kind == 0 else
                 W.convex_polygon(rng, r, 7) if kind == 1 else W.polyline(rng, r, 5))
        els.append((kind, shape, 0.012 if kind == 2 else 0.0))
        params.append((0.3 + 0.4 * rng.uniform(), 0.3 + 0.4 * rng.uniform(),
                       rng.uniform(0, 6.28), 0.8 + 0.4 * rng.uniform()))
    prob = W.make_problem(els, W.star_container(rng, r_in=0.3, r_out=0.45), params, R)
    q = np.asarray(params, np.float64).reshape(-1)
    o = oracle_mod.options(pad_px=1.0, delta=50.0, force_kind=force_kind, force_x=0.4, force_y=0.55)
    g, _ = oracle_mod.control_grad(prob, q, R, o)
    gb = oracle_mod.Scene(prob).eval(q, R, o)["grad_b"].reshape(-1, 4)
    P = np.asarray(prob["pts"], np.float32).astype(np.float64).reshape(-1, 2)
    off = prob["pt_off"]
    scale = np.abs(gb).max()
    for e in range(len(els)):
        th, s = q[4 * e + 2], q[4 * e + 3]
        c, sn = np.cos(th), np.sin(th)
        ge, Pe = g[off[e]:off[e + 1]], P[off[e]:off[e + 1]]
        t_loc = s * np.array([c * gb[e, 0] + sn * gb[e, 1], -sn * gb[e, 0] + c * gb[e, 1]])
        np.testing.assert_allclose(ge.sum(0), t_loc, rtol=0, atol=1e-9 * scale)
        rot = np.sum(Pe[:, 0] * ge[:, 1] - Pe[:, 1] * ge[:, 0])
        assert abs(rot - gb[e, 2]) <= 1e-9 * scale, (e, rot, gb[e, 2])
        dil = np.sum(Pe * ge)
        assert abs(dil - s * gb[e, 3]) <= 1e-9 * scale, (e, dil, s * gb[e, 3])


def test_adam_points_matches_torch(oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    p0 = rng.normal(size=(10, 2))
    grads = [rng.normal(size=(10, 2)) for _ in range(3)]
    tp = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for k, gk in enumerate(grads):
        opt.zero_grad()
        tp.grad = torch.tensor(gk)
        opt.step()
        p, m, v = oracle_mod.adam_points(p, m, v, gk, k + 1)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=0, atol=1e-15)


# ---- skeleton-based initialisation (Sec. 4.1) -----------------------------------------------------
def test_medial_width_matches_scipy_edt(oracle_mod):
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(11)
    for R in (17, 40):
        cov = (rng.uniform(size=(R, R)) < 0.8).astype(np.float64)
        D2, _ = oracle_mod.medial_axis(cov)
        # scipy measures to the nearest zero of its input: pad the image with one outside ring
        padded = np.zeros((R + 2, R + 2))
        padded[1:-1, 1:-1] = cov >= 0.5
        ref = nd.distance_transform_edt(padded)[1:-1, 1:-1]
        np.testing.assert_array_equal(D2, np.rint(ref ** 2).astype(np.int64))


def test_medial_axis_closed_forms(oracle_mod):
    # a horizontal strip of odd height: the centre row is the ridge away from the ends, and only it
    R = 64
    cov = np.zeros((R, R))
    cov[20:31, 4:60] = 1.0  # 11 rows: centre row 25
    D2, axis = oracle_mod.medial_axis(cov)
    assert axis[25, 12:52].all()
    assert not axis[20:25, 12:52].any() and not axis[26:31, 12:52].any()
    assert (D2[25, 12:52] == 36).all()  # 6 rows to the outside rows 19 and 31
    # a square: the ridge is its two diagonals (and the centre has the largest width)
    cov = np.zeros((R, R))
    cov[10:41, 10:41] = 1.0  # 31 x 31, centre (25, 25)
    D2, axis = oracle_mod.medial_axis(cov)
    assert D2.max() == D2[25, 25] == 16 ** 2
    for k in range(-12, 13):
        assert axis[25 + k, 25 + k] and axis[25 + k, 25 - k]
    assert not axis[25, 18] and not axis[18, 25]


def _place_brute(D2, axis, r, res):
    """The placement rule with explicit loops: largest radius first (lower index on ties); among the
    axis pixels with clearance >= r the largest D2 (lower pixel index on ties), else the largest
    clearance; clearances in float32."""
    cands = [(int(i), int(D2.reshape(-1)[i])) for i in np.flatnonzero(axis.reshape(-1))]
    clear = {i: np.float32(np.finfo(np.float32).max) for i, _ in cands}
    todo = list(range(len(r)))
    out = {}
    while todo:
        e = todo[0]
        for f in todo:
            if r[f] > r[e]:
                e = f
        todo.remove(e)
        best = None
        for i, w in cands:
            if clear[i] >= r[e] and (best is None or w > best[1] or (w == best[1] and i < best[0])):
                best = (i, w)
        if best is None:
            for i, _ in cands:
                if best is None or clear[i] > clear[best[0]] or (clear[i] == clear[best[0]] and i < best[0]):
                    best = (i, 0)
        c = best[0]
        out[e] = c
        for i, _ in cands:
            d = np.float32(np.sqrt(np.float32((i % res - c % res) ** 2 + (i // res - c // res) ** 2)))
            clear[i] = min(clear[i], np.float32(d - r[e]))
    return out


def test_mat_placement_brute_force(oracle_mod):
    R = 48
    rng = W.PCG32(5)
    els = [(1, W.regular_polygon(0.03 + 0.05 * rng.uniform(), 8), 0.0) for _ in range(7)]
    params = [(0.5, 0.5, 0.0, 1.0)] * 7
    prob = W.make_problem(els, W.star_container(rng, r_in=0.2, r_out=0.45), params, R)
    o = oracle_mod.options()
    q, D2, axis = oracle_mod.mat_init(prob, prob["params0"], R, o)
    sc = oracle_mod.Scene(prob)
    r = (np.array([sc.bin_radius(e) for e in range(7)], np.float32) * np.float32(1.0)) * np.float32(R)
    ref = _place_brute(D2, axis, r, R)
    for e, c in ref.items():
        assert q[e, 0] == np.float32((np.float32(c % R) + np.float32(0.5)) / np.float32(R))
        assert q[e, 1] == np.float32((np.float32(c // R) + np.float32(0.5)) / np.float32(R))
    # the largest element sits at the widest pixel of the container
    e0 = int(np.argmax(r))
    c0 = ref[e0]
    assert D2.reshape(-1)[c0] == D2.max()
    # rotation and scale are untouched
    assert np.array_equal(q[:, 2:], np.asarray(prob["params0"], np.float32).reshape(-1, 4)[:, 2:])
