"""Pins for the oracle's per-triangle update step (Sec. 3.2, the planar
Kimmel-Sethian update with the monotonicity condition Q X^T n < 0 and the
edge fallback).  Every expected value here comes from geometry, not from the
oracle's own formula: a linear distance field is reproduced exactly when its
upwind ray enters the triangle, hand-computed special cases, and invariances.
"""
import math

import numpy as np
import pytest

import oracle


def _plane_basis(e1, e2):
    u = e1 / np.linalg.norm(e1)
    w = e2 - np.dot(e2, u) * u
    w /= np.linalg.norm(w)
    return u, w


def _upwind_ray_hits_segment(x0, x1, x2, n):
    """Does the ray x0 - s*n (s > 0) cross the open segment (x1, x2)?
    Returns the segment parameter t of the crossing, or None."""
    u, w = _plane_basis(x1 - x0, x2 - x0)
    to2 = lambda p: np.array([np.dot(p - x0, u), np.dot(p - x0, w)])
    a, b = to2(x1), to2(x2)
    r = -np.array([np.dot(n, u), np.dot(n, w)])
    # solve s*r = a + t*(b - a)
    M = np.array([[r[0], -(b - a)[0]], [r[1], -(b - a)[1]]])
    if abs(np.linalg.det(M)) < 1e-14:
        return None
    s, t = np.linalg.solve(M, a)
    if s <= 0:
        return None
    return t


def _random_triangle(rng):
    while True:
        P = rng.normal(size=(3, 3))
        e1, e2, e3 = P[1] - P[0], P[2] - P[0], P[2] - P[1]
        ang = []
        for p, q in [(e1, e2), (-e1, e3), (-e2, -e3)]:
            c = np.dot(p, q) / (np.linalg.norm(p) * np.linalg.norm(q))
            ang.append(math.acos(max(-1.0, min(1.0, c))))
        if min(ang) > 0.1:
            return P


def _expected_by_edge_construction(x0, x1, x2, d1, d2, margin=0.01):
    """The update from the edge's point of view: a unit in-plane gradient g
    with g.(x1 - x2) = d1 - d2 has two solutions, mirror images across the
    edge; each gives an arrival time p = d1 - g.(x1 - x0).  The larger one
    is kept when its upwind ray from x0 crosses the open edge (x1, x2), else
    the shortest edge path.  Returns None near the crossing's ends."""
    fb = min(d1 + np.linalg.norm(x1 - x0), d2 + np.linalg.norm(x2 - x0))
    L = np.linalg.norm(x1 - x2)
    u = (x1 - x2) / L
    w = (x0 - x2) - np.dot(x0 - x2, u) * u
    w /= np.linalg.norm(w)
    alpha = (d1 - d2) / L
    if abs(alpha) >= 1.0:
        return fb if abs(alpha) > 1.0 + 1e-9 else None
    cands = []
    for sgn in (1.0, -1.0):
        g = alpha * u + sgn * math.sqrt(1.0 - alpha * alpha) * w
        cands.append((d1 - np.dot(g, x1 - x0), g))
    p, g = max(cands, key=lambda c: c[0])
    t = _upwind_ray_hits_segment(x0, x1, x2, g)
    if t is not None and margin < t < 1.0 - margin:
        return p
    if t is None or t < -margin or t > 1.0 + margin:
        return fb
    return None


def test_linear_field_reproduced():
    """d_i = n.x_i + c for a unit in-plane n: when the upwind ray from x0
    enters the triangle the update must return n.x0 + c exactly (a linear
    field has |grad d| = 1 and is the planar model's own solution)."""
    rng = np.random.default_rng(1)
    hits = 0
    for _ in range(3000):
        x0, x1, x2 = _random_triangle(rng)
        e1, e2 = x1 - x0, x2 - x0
        n = rng.normal() * e1 + rng.normal() * e2
        n /= np.linalg.norm(n)
        c = rng.uniform(5.0, 10.0)
        d1, d2 = np.dot(n, x1) + c, np.dot(n, x2) + c
        t = _upwind_ray_hits_segment(x0, x1, x2, n)
        if t is not None and 0.01 < t < 0.99:
            assert oracle.update(x0, x1, x2, d1, d2) == pytest.approx(np.dot(n, x0) + c, abs=1e-10)
            hits += 1
    assert hits > 500


def test_matches_edge_construction():
    """Arbitrary neighbour distances: the update equals the edge-based
    construction of the planar solution with its causality check, or the
    edge fallback."""
    rng = np.random.default_rng(11)
    planar = fallback = 0
    for _ in range(4000):
        x0, x1, x2 = _random_triangle(rng)
        d1, d2 = rng.uniform(0.0, 3.0, size=2)
        exp = _expected_by_edge_construction(x0, x1, x2, d1, d2)
        if exp is None:
            continue
        got = oracle.update(x0, x1, x2, d1, d2)
        assert got == pytest.approx(exp, abs=1e-10)
        fb = min(d1 + np.linalg.norm(x1 - x0), d2 + np.linalg.norm(x2 - x0))
        if exp < fb - 1e-9:
            planar += 1
        else:
            fallback += 1
    assert planar > 300 and fallback > 300


def test_equilateral_from_opposite_edge():
    """Front along the opposite edge (d1 = d2 = 0) of an equilateral triangle
    of side h: the arrival time is the height h*sqrt(3)/2."""
    h = 0.37
    x1 = np.array([0.0, 0.0, 0.0])
    x2 = np.array([h, 0.0, 0.0])
    x0 = np.array([h / 2, h * math.sqrt(3) / 2, 0.0])
    assert oracle.update(x0, x1, x2, 0.0, 0.0) == pytest.approx(h * math.sqrt(3) / 2, abs=1e-15)


def test_right_and_obtuse_vertex_from_opposite_edge():
    # right angle at x0: distance from x0 to the line through x1, x2
    assert oracle.update([0, 0, 0], [1, 0, 0], [0, 1, 0], 0.0, 0.0) == pytest.approx(1 / math.sqrt(2), abs=1e-15)
    # obtuse angle at x0, foot of the perpendicular inside the edge
    assert oracle.update([0, 0, 0], [1, 0.1, 0], [-1, 0.1, 0], 0.0, 0.0) == pytest.approx(0.1, abs=1e-15)


def test_non_causal_planar_wave_falls_back_to_edge():
    """x1=(0,0,0), x2=(1,0,0), x0=(0,1,0), d1=0, d2=1: the planar wave d = x
    fits the data and would give p = 0, but its characteristic reaches x0
    from outside the triangle, so the update is the edge value min(0+1, 1+sqrt2) = 1."""
    assert oracle.update([0, 1, 0], [0, 0, 0], [1, 0, 0], 0.0, 1.0) == pytest.approx(1.0, abs=1e-15)


def test_infinite_and_degenerate_inputs():
    x0, x1, x2 = [0, 0, 0], [1, 0, 0], [0, 2, 0]
    assert oracle.update(x0, x1, x2, math.inf, math.inf) == math.inf
    assert oracle.update(x0, x1, x2, 0.5, math.inf) == pytest.approx(1.5)
    assert oracle.update(x0, x1, x2, math.inf, 0.25) == pytest.approx(2.25)
    # collinear: x0 on the segment x1 x2 -> edge fallback only
    assert oracle.update([0.5, 0, 0], [0, 0, 0], [1, 0, 0], 0.3, 0.1) == pytest.approx(0.6)


def test_invariances():
    """Swapping the two neighbours, shifting both distances, scaling the
    whole triangle with the distances, and rigid motions leave the update
    unchanged (up to the same shift / scale)."""
    rng = np.random.default_rng(2)
    for _ in range(500):
        x0, x1, x2 = _random_triangle(rng)
        d1, d2 = rng.uniform(1.0, 3.0, size=2)
        u = oracle.update(x0, x1, x2, d1, d2)
        assert oracle.update(x0, x2, x1, d2, d1) == pytest.approx(u, abs=1e-12)
        s = rng.uniform(-0.5, 5.0)
        assert oracle.update(x0, x1, x2, d1 + s, d2 + s) == pytest.approx(u + s, abs=1e-11)
        lam = rng.uniform(0.1, 10.0)
        assert oracle.update(lam * x0, lam * x1, lam * x2, lam * d1, lam * d2) == pytest.approx(lam * u, rel=1e-11)
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        t = rng.normal(size=3)
        assert oracle.update(Q @ x0 + t, Q @ x1 + t, Q @ x2 + t, d1, d2) == pytest.approx(u, abs=1e-11)


def test_bounds():
    """The update never exceeds the edge paths; a planar solution in a
    triangle that is not obtuse at x0 arrives after both neighbours (the
    monotonicity property of Sec. 3.2, which needs non-obtuse triangles)."""
    rng = np.random.default_rng(3)
    later = 0
    for _ in range(2000):
        x0, x1, x2 = _random_triangle(rng)
        d1, d2 = rng.uniform(0.0, 2.0, size=2)
        u = oracle.update(x0, x1, x2, d1, d2)
        fb = min(d1 + np.linalg.norm(x1 - x0), d2 + np.linalg.norm(x2 - x0))
        assert u <= fb + 1e-12
        assert u >= min(d1, d2)
        if u < fb - 1e-12 and np.dot(x1 - x0, x2 - x0) >= 0.0:
            assert u > max(d1, d2) - 1e-12
            later += 1
    assert later > 100


def _sliver(rng, sin2, where):
    """A triangle (x0, x1, x2) in a random plane whose smallest angle has
    squared sine sin2, at x0 (a needle pointing at the updated vertex), at
    x1 (x0 at the blunt end of a needle) or an obtuse cap with the angle
    pi - asin(sqrt(sin2)) at x0."""
    th = math.asin(math.sqrt(sin2))
    L1, L2 = rng.uniform(0.5, 2.0, size=2)
    if where == "x0":
        P = [(0.0, 0.0), (L1, 0.0), (L2 * math.cos(th), L2 * math.sin(th))]
    elif where == "x1":
        P = [(L2 * math.cos(th), L2 * math.sin(th)), (0.0, 0.0), (L1, 0.0)]
    else:  # cap: x0 nearly on the segment x1 x2
        P = [(0.0, 0.0), (-L1 * math.cos(th / 2), L1 * math.sin(th / 2)),
             (L2 * math.cos(th / 2), L2 * math.sin(th / 2))]
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    t = rng.normal(size=3)
    return [Q @ np.array([x, y, 0.0]) + t for x, y in P]


def _textbook_update_hp(x0, x1, x2, d1, d2, mp):
    """The update of Sec. 3.2 exactly as written -- Q = (X^T X)^{-1}, the
    larger root of (1^T Q 1) p^2 - 2 (1^T Q t) p + (t^T Q t - 1) = 0 and the
    test Q (t - p 1) < 0 -- evaluated in `mp` (60-digit) arithmetic from the
    given doubles.  Returns (value, margin): margin is how far, relative to
    the size of its terms, each decision lies from its boundary (the
    degenerate threshold; |d2 - d1| against |x2 - x1|, where the two roots
    meet; the two causality signs, scaled by det so their terms are edge-
    sized), so that cases an FP64 evaluation cannot decide are skipped."""
    X0, X1, X2 = ([mp.mpf(float(v)) for v in x] for x in (x0, x1, x2))
    D1, D2 = mp.mpf(float(d1)), mp.mpf(float(d2))
    e1 = [X1[i] - X0[i] for i in range(3)]
    e2 = [X2[i] - X0[i] for i in range(3)]
    a = sum(v * v for v in e1)
    b = sum(e1[i] * e2[i] for i in range(3))
    c = sum(v * v for v in e2)
    fb = min(D1 + mp.sqrt(a), D2 + mp.sqrt(c))
    det = a * c - b * b
    margins = [abs(det / (a * c) / mp.mpf("1e-12") - 1)]
    if det <= mp.mpf("1e-12") * a * c:
        return fb, min(margins)
    q11, q12, q22 = c / det, -b / det, a / det
    qa = q11 + 2 * q12 + q22
    qb = q11 * D1 + q12 * (D1 + D2) + q22 * D2
    qc = q11 * D1 * D1 + 2 * q12 * D1 * D2 + q22 * D2 * D2 - 1
    disc = qb * qb - qa * qc
    A, delta = a + c - 2 * b, D2 - D1
    margins.append(abs(A - delta * delta) / A)
    if disc < 0:
        return fb, min(margins)
    p = (qb + mp.sqrt(disc)) / qa
    l1 = q11 * (D1 - p) + q12 * (D2 - p)
    l2 = q12 * (D1 - p) + q22 * (D2 - p)
    r = p - D1
    margins += [abs(l1 * det) / (abs((b - c) * r) + abs(b * delta)),
                abs(l2 * det) / (abs((b - a) * r) + abs(a * delta))]
    return (p if (l1 < 0 and l2 < 0) else fb), min(margins)


def test_slivers_match_the_definition_in_high_precision():
    """Near-degenerate triangles (smallest squared sine 1e-12 .. 1e-6, the
    range the GPU solves in FP64; needles at x0 or at x1 and obtuse caps)
    with linear-field and arbitrary data: the oracle's FP64 update equals
    the textbook quadratic evaluated in 60-digit arithmetic to within
    1e-10 of the triangle's size, away from decision boundaries.  Evaluating
    the coefficients as written in FP64 misses this by up to 1e-3."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp.clone() if hasattr(mpmath.mp, "clone") else mpmath.mp
    mp.dps = 60
    rng = np.random.default_rng(21)
    planar = checked = 0
    worst = 0.0
    for k in range(1500):
        sin2 = 10.0 ** rng.uniform(-11.8, -6.0)
        x0, x1, x2 = _sliver(rng, sin2, ("x0", "x1", "cap")[k % 3])
        L = np.linalg.norm(x2 - x1)
        scale = max(np.linalg.norm(x1 - x0), np.linalg.norm(x2 - x0))
        base = rng.uniform(0.5, 10.0)
        if k % 2 == 0:  # a unit in-plane linear field
            u, w = _plane_basis(x1 - x0, x2 - x0)
            phi = rng.uniform(0.0, 2.0 * math.pi)
            n = math.cos(phi) * u + math.sin(phi) * w
            d1, d2 = np.dot(n, x1) + base, np.dot(n, x2) + base
        else:  # any difference the edge allows
            d1 = base
            d2 = base + rng.uniform(-0.999, 0.999) * L
        exp, margin = _textbook_update_hp(x0, x1, x2, d1, d2, mp)
        if margin < 1e-6:
            continue
        got = oracle.update(x0, x1, x2, d1, d2)
        err = abs(got - float(exp))
        worst = max(worst, err / scale)
        assert err <= 1e-10 * scale, (k, sin2, got, float(exp))
        checked += 1
        fb = min(d1 + np.linalg.norm(x1 - x0), d2 + np.linalg.norm(x2 - x0))
        planar += got < fb
    assert checked > 1200 and planar > 150, (checked, planar)


def test_needle_at_the_updated_vertex_below_the_threshold_takes_the_edge():
    """Below the degeneracy threshold (the squared sine of the angle at x0
    at most 1e-12) the update is the edge fallback, even for data that a
    planar wave through the needle would fit."""
    rng = np.random.default_rng(22)
    for _ in range(200):
        x0, x1, x2 = _sliver(rng, 10.0 ** rng.uniform(-16.0, -12.5), "x0")
        target = x1 + 0.5 * (x2 - x1)
        n = (x0 - target) / np.linalg.norm(x0 - target)
        d1, d2 = np.dot(n, x1) + 3.0, np.dot(n, x2) + 3.0
        fb = min(d1 + np.linalg.norm(x1 - x0), d2 + np.linalg.norm(x2 - x0))
        assert oracle.update(x0, x1, x2, d1, d2) == pytest.approx(fb, rel=1e-14)
