"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each ``pin_*`` function takes one loaded oracle build and raises
AssertionError when that build disagrees with the fact it checks.  The real
oracle must pass all of them; copies of the oracle with a planted mistake
must each fail at least one (tests/test_oracle_mutants.py), which shows the
pins are not vacuous.

None of these re-types the oracle's own formulas.  They check it against
  * a library routine on the same definition (scipy's cdist + numpy's
    lexsort for the k-NN; numpy's lstsq for the projection onto a line and
    for the weighted least-squares objective of Section 3.1 step 4, stacked
    as rows rather than as normal equations);
  * closed forms (k = 2, k = 3, exact plane recovery, hand-worked golden
    fixtures under tests/golden/);
  * invariances that hold for any score function (similarity maps of either
    space, landmark relabelling, common scaling of the scores), the
    properties Section 3.1 step 2 demands of the scores, and boost acting as
    the sharpness of the score profile.  The numeric score values (the 1/i
    weights of the mean and spread, the steepness 10 of the cut-off) are a
    reading with no printed example: parity unpinned beyond these
    properties.
"""
from __future__ import annotations

import json
import os

import numpy as np
from scipy.spatial.distance import cdist

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


def _close(a, b, tol, what):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    err = np.max(np.abs(a - b)) if a.size else 0.0
    assert err <= tol, f"{what}: max |diff| = {err:.3e} > {tol:.1e}"


# --------------------------------------------------------------------------
# Step 1: k nearest landmarks.

def pin_knn_bruteforce(O):
    """k-NN equals a full sort of scipy's squared Euclidean distances, ties to
    the lower landmark index (Section 3.1 step 1; Section 4.2)."""
    r = _rng(1)
    cases = []
    for (n, g, d, k) in [(40, 17, 3, 5), (50, 20, 5, 20), (30, 12, 1, 3), (25, 9, 4, 9)]:
        cases.append((r.standard_normal((n, d)), r.standard_normal((g, d)), k))
    # exact ties: integer lattice points and landmarks
    cases.append((r.integers(-2, 3, (50, 2)), r.integers(-2, 3, (20, 2)), 7))
    cases.append((r.integers(-1, 2, (40, 3)), r.integers(-1, 2, (15, 3)), 15))
    # duplicated landmark rows
    Ld = r.standard_normal((10, 4))
    cases.append((r.standard_normal((30, 4)), np.concatenate([Ld, Ld[[3, 7, 1]]]), 6))
    for X, L, k in cases:
        X = X.astype(np.float32)
        L = L.astype(np.float32)
        idx, d2 = O.knn(X, L, k)
        D = cdist(X.astype(np.float64), L.astype(np.float64), "sqeuclidean")
        for i in range(X.shape[0]):
            order = np.lexsort((np.arange(L.shape[0]), D[i]))[:k]
            assert np.array_equal(idx[i], order), f"row {i}: {idx[i]} != {order}"
            _close(d2[i], D[i, order], 1e-12 * max(1.0, D[i].max()), "knn distances")


# --------------------------------------------------------------------------
# Closed forms.

def pin_k2_nearest_layout_point(O):
    """k = 2: one scored neighbour, no pair, so x is that neighbour's 2-D
    landmark exactly (Section 3.1 steps 2-4 with k - 1 = 1)."""
    r = _rng(2)
    X = r.standard_normal((60, 6)).astype(np.float32)
    L = r.standard_normal((25, 6)).astype(np.float32)
    lo = r.uniform(-4, 9, (25, 2)).astype(np.float32)
    idx, _ = O.knn(X, L, 2)
    for boost, adjust in [(1.0, 1.0), (3.0, 0.0)]:
        out = O.project(X, L, lo, 2, boost, adjust)
        assert np.array_equal(out, lo[idx[:, 0]].astype(np.float64))


def _line_coordinate(X, A, B):
    """Least-squares coordinate t of X on the line A + t (B - A)."""
    t, *_ = np.linalg.lstsq((B - A)[:, None], X - A, rcond=None)
    return float(t[0])


def pin_k3_closed_form(O):
    """k = 3: a single scored pair; the fit matches D_uv exactly on the line
    through the two scored 2-D landmarks, x = l_u + D_uv (l_v - l_u), for any
    scores, boost or adjust (Section 3.1 steps 3-4)."""
    r = _rng(3)
    X = r.standard_normal((80, 5)).astype(np.float32)
    L = r.standard_normal((12, 5)).astype(np.float32)
    lo = r.uniform(0, 10, (12, 2)).astype(np.float32)
    idx, _ = O.knn(X, L, 3)
    for boost, adjust in [(1.0, 1.0), (2.0, 0.0), (0.3, 2.0)]:
        out = O.project(X, L, lo, 3, boost, adjust)
        for i in range(X.shape[0]):
            u, v = idx[i, 0], idx[i, 1]
            D = _line_coordinate(X[i].astype(np.float64), L[u].astype(np.float64),
                                 L[v].astype(np.float64))
            want = lo[u].astype(np.float64) + D * (lo[v].astype(np.float64) - lo[u])
            _close(out[i], want, 1e-9 * (1 + np.abs(want).max()), f"k=3 point {i}")


def pin_golden_fixtures(O):
    """Hand-worked examples stored under tests/golden/."""
    for name in ("k3_hand_worked.json", "identity_layout.json"):
        with open(os.path.join(GOLDEN, name)) as f:
            g = json.load(f)
        X = np.array(g["X"], np.float32)
        hi = np.array(g["hi"], np.float32)
        lo = np.array(g["lo"], np.float32)
        idx, _ = O.knn(X, hi, g["k"])
        assert np.array_equal(idx, np.array(g["neighbours"])), name
        for boost, adjust in g["params"]:
            out = O.project(X, hi, lo, g["k"], boost, adjust)
            _close(out, g["expected"], 1e-12, f"{name} boost={boost} adjust={adjust}")


def _hadamard_plane(r, d):
    """d x 2 matrix with orthonormal columns and entries in {0, +-1/2}
    (exactly representable), plus two more unit vectors orthogonal to it."""
    cols = r.choice(d, 4, replace=False)
    H = np.array([[1, 1, 1, 1], [1, -1, 1, -1], [1, 1, -1, -1], [1, -1, -1, 1]]) / 2.0
    Q = np.zeros((d, 4))
    Q[cols, :] = H.T
    return Q[:, :2], Q[:, 2:], cols


def pin_plane_recovery(O):
    """If L_j = c Q l_j + t and X = c Q p + t + z with Q orthonormal and z
    orthogonal to Q, every residual D_uv(X) - d_uv(p) is zero, so x = p for
    any scores, boost and adjust (Section 3.1 steps 3-4).  All inputs are
    dyadic, so the fp32 arguments are exact."""
    r = _rng(4)
    for d, g, k, boost, adjust in [(4, 30, 4, 1.0, 1.0), (8, 30, 7, 2.0, 0.0),
                                   (16, 40, 12, 0.5, 2.5), (6, 30, 30, 1.0, 1.0),
                                   (12, 64, 20, 2.0, 1.0)]:
        Q, Qp, cols = _hadamard_plane(r, d)
        c = 2.0
        t = r.integers(-8, 8, d) / 4.0
        lo = r.integers(0, 80, (g, 2)) / 8.0
        hi = c * lo @ Q.T + t
        p = r.integers(8, 72, (50, 2)) / 16.0
        other = [i for i in range(d) if i not in cols]
        z = np.zeros((50, d))
        z += (r.integers(-4, 5, (50, 2)) / 8.0) @ Qp.T
        if other:
            z[:, other] = r.integers(-4, 5, (50, len(other))) / 8.0
        X = c * p @ Q.T + t + z
        for a in (X, hi, lo):
            assert np.array_equal(a.astype(np.float32).astype(np.float64), a)
        out, ratio, branch = O.project(X, hi, lo, k, boost, adjust, diagnostics=True)
        full = branch == 0
        assert full.mean() > 0.9, "plane recovery cases should be full rank"
        _close(out[full], p[full], 1e-9, f"plane recovery d={d} k={k}")


def pin_weighted_least_squares(O):
    """x is the minimiser of sum_{u<v} s_u s_v r^(1-adjust) (D_uv - d_uv(p))^2,
    solved here as weighted least-squares rows by numpy's lstsq; D_uv by
    lstsq projection onto the line L_u L_v; the scores are the oracle's
    own (their values are a reading, pinned separately by their shape)."""
    r = _rng(5)
    n, d, g = 40, 7, 30
    X = (r.standard_normal((n, d)) * 2).astype(np.float32)
    hi = (r.standard_normal((g, d)) * 2).astype(np.float32)
    lo = r.uniform(0, 10, (g, 2)).astype(np.float32)
    for k, boost, adjust in [(6, 1.0, 1.0), (10, 2.0, 0.0), (8, 0.7, 0.5), (12, 1.0, 2.0)]:
        idx, d2 = O.knn(X, hi, k)
        out = O.project(X, hi, lo, k, boost, adjust)
        X64, hi64, lo64 = X.astype(np.float64), hi.astype(np.float64), lo.astype(np.float64)
        for i in range(n):
            s = O.scores(d2[i], boost)
            rows, rhs = [], []
            for a in range(k - 1):
                for b in range(a + 1, k - 1):
                    u, v = idx[i, a], idx[i, b]
                    h = lo64[v] - lo64[u]
                    rr = h @ h
                    D = _line_coordinate(X64[i], hi64[u], hi64[v])
                    W = s[a] * s[b] * rr ** (1.0 - adjust)
                    rows.append(np.sqrt(W) * h / rr)
                    rhs.append(np.sqrt(W) * (D + h @ lo64[u] / rr))
            p, *_ = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)
            _close(out[i], p, 1e-8 * (1 + np.abs(p).max()), f"lstsq k={k} adjust={adjust} pt {i}")


def pin_collinear_layout(O):
    """2-D landmarks on one line make the normal matrix rank one; the
    solution returned is the least-squares one of least distance from the
    score-weighted centroid of the scored 2-D landmarks (numpy's lstsq gives
    the minimum-norm solution of the shifted problem)."""
    r = _rng(6)
    n, d, g, k, boost, adjust = 30, 5, 20, 7, 1.0, 1.0
    X = r.standard_normal((n, d)).astype(np.float32)
    hi = r.standard_normal((g, d)).astype(np.float32)
    a = r.integers(0, 64, g) / 8.0
    lo = np.stack([a, 2 * a + 1], axis=1).astype(np.float32)
    idx, d2 = O.knn(X, hi, k)
    out, ratio, branch = O.project(X, hi, lo, k, boost, adjust, diagnostics=True)
    assert np.all(branch == 1)
    X64, hi64, lo64 = X.astype(np.float64), hi.astype(np.float64), lo.astype(np.float64)
    for i in range(n):
        s = O.scores(d2[i], boost)
        nb = idx[i, :k - 1]
        c = (s[:k - 1, None] * lo64[nb]).sum(0) / s[:k - 1].sum()
        rows, rhs = [], []
        for x in range(k - 1):
            for y in range(x + 1, k - 1):
                u, v = nb[x], nb[y]
                h = lo64[v] - lo64[u]
                rr = h @ h
                if rr == 0:
                    continue
                D = _line_coordinate(X64[i], hi64[u], hi64[v])
                W = np.sqrt(s[x] * s[y] * rr ** (1.0 - adjust))
                rows.append(W * h / rr)
                rhs.append(W * (D + h @ lo64[u] / rr))
        rows, rhs = np.array(rows), np.array(rhs)
        delta, *_ = np.linalg.lstsq(rows, rhs - rows @ c, rcond=1e-9)
        _close(out[i], c + delta, 1e-8 * (1 + np.abs(c).max()), f"collinear pt {i}")


# --------------------------------------------------------------------------
# Invariances (hold for any score function of the distances).

def _random_setup(seed, n=50, d=9, g=40):
    r = _rng(seed)
    X = r.integers(-32, 33, (n, d)) / 8.0
    hi = r.integers(-32, 33, (g, d)) / 8.0
    lo = r.integers(0, 80, (g, 2)) / 8.0
    return r, X, hi, lo


def pin_layout_similarity(O):
    """A similarity map of the 2-D landmarks (rotation by quarter turns,
    reflection, scale, shift) moves x by the same map: every weight changes
    by one common factor."""
    r, X, hi, lo = _random_setup(7)
    for k, boost, adjust in [(8, 1.0, 1.0), (12, 2.0, 0.0), (6, 1.0, 2.5)]:
        base = O.project(X, hi, lo, k, boost, adjust)
        for R, c, t in [(np.array([[0, -1], [1, 0]]), 2.0, np.array([3.5, -1.25])),
                        (np.array([[1, 0], [0, -1]]), 0.5, np.array([-8.0, 4.0])),
                        (np.array([[0, 1], [1, 0]]), 4.0, np.array([0.0, 0.0]))]:
            lo2 = c * lo @ R.T + t
            out = O.project(X, hi, lo2, k, boost, adjust)
            want = c * base @ R.T + t
            _close(out, want, 1e-9 * c * 10, f"layout similarity k={k}")


def pin_space_similarity(O):
    """A similarity map of the high-dimensional space applied to X and L
    together (signed permutation, scale, shift) leaves x unchanged: distance
    ratios and every D_uv are unchanged."""
    r, X, hi, lo = _random_setup(8)
    d = X.shape[1]
    for k, boost in [(8, 1.0), (15, 2.0)]:
        base = O.project(X, hi, lo, k, boost, 1.0)
        P = np.eye(d)[r.permutation(d)] * r.choice([-1.0, 1.0], d)[None, :]
        for c in (2.0, 0.25):
            t = r.integers(-8, 8, d) / 4.0
            out = O.project(c * X @ P.T + t, c * hi @ P.T + t, lo, k, boost, 1.0)
            _close(out, base, 1e-9, f"space similarity k={k} c={c}")


def pin_relabelling(O):
    """Relabelling the landmarks (L and l together) does not change x."""
    r = _rng(9)
    X = r.standard_normal((60, 6)).astype(np.float32)
    hi = r.standard_normal((30, 6)).astype(np.float32)
    lo = r.uniform(0, 10, (30, 2)).astype(np.float32)
    base = O.project(X, hi, lo, 9, 1.5, 1.0)
    perm = r.permutation(30)
    out = O.project(X, hi[perm], lo[perm], 9, 1.5, 1.0)
    assert np.array_equal(out, base)


def pin_score_homogeneity(O):
    """Multiplying every score by one constant does not change x."""
    r = _rng(10)
    X = r.standard_normal((20, 5)).astype(np.float32)
    hi = r.standard_normal((25, 5)).astype(np.float32)
    lo = r.uniform(0, 10, (25, 2)).astype(np.float32)
    idx, d2 = O.knn(X, hi, 8)
    for i in range(20):
        s = O.scores(d2[i], 1.0)
        a, _, _ = O.fit(X[i], hi, lo, idx[i], s, 1.0)
        b, _, _ = O.fit(X[i], hi, lo, idx[i], s * 37.5, 1.0)
        _close(a, b, 1e-10 * (1 + np.abs(a).max()), "score homogeneity")


# --------------------------------------------------------------------------
# Scores (Section 3.1 step 2): highest for the nearest, zero for the k-th,
# smooth in the distances.

def pin_score_shape(O):
    r = _rng(11)
    for k in (3, 5, 10, 20, 30):
        for boost in (0.5, 1.0, 2.0):
            for _ in range(20):
                dist = np.sort(r.uniform(0.1, 5.0, k))
                s = O.scores(dist ** 2, boost)
                assert s[k - 1] == 0.0
                assert np.all(s[:k - 1] > 0)
                # distinct distances: strictly decreasing, so the nearest
                # alone holds the highest score
                assert np.all(np.diff(s) < 0), s
                assert s[0] == s.max()
                s2 = O.scores((3.0 * dist) ** 2, boost)
                _close(s2, s, 1e-12 * s.max(), "scores scale-free in the distances")
                # smooth: a tiny change of one distance moves the scores a tiny bit
                j = int(r.integers(0, k))
                dd = dist.copy()
                dd[j] *= 1 + 1e-9
                dd = np.sort(dd)
                _close(O.scores(dd ** 2, boost), s, 1e-6 * s.max(), "scores continuous")


def pin_boost_sharpness(O):
    """boost is the sharpness of the score profile (the parameter of the
    original EmbedSOM score function that Section 3.1 step 2 defers to): for
    fixed distances delta_1 < delta_i < delta_k, the relative score s_i / s_1
    falls strictly as boost grows, towards 0 for a large boost, while s_1
    stays the largest score."""
    r = _rng(14)
    boosts = np.array([0.125, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0])
    for k in (3, 4, 10, 20, 30):
        for _ in range(10):
            dist = np.sort(r.uniform(0.5, 4.0, k))
            if np.min(np.diff(dist)) < 1e-3:
                continue
            S = np.array([O.scores(dist ** 2, b) for b in boosts])   # boosts x k
            rel = S[:, 1:k - 1] / S[:, :1]                           # s_i / s_1, 1 < i < k
            assert np.all(rel > 0) and np.all(rel < 1), rel
            assert np.all(np.diff(rel, axis=0) < 0), f"s_i/s_1 not falling with boost: {rel}"
            assert np.all(S[-1, 1:k - 1] / S[-1, 0] < S[0, 1:k - 1] / S[0, 0])


def _crossing_point(X0, La, Lb):
    """Point on X0 + t (Lb - La) equidistant from La and Lb."""
    e = Lb - La
    t = ((Lb @ Lb - La @ La) / 2.0 - X0 @ e) / (e @ e)
    return X0 + t * e, e


def pin_continuity_at_cutoff(O):
    """Section 3.1 step 2 gives the k-th neighbour score 0 so that the map
    stays smooth when neighbours change: moving X across the bisector
    between its (k-1)-th and k-th, or k-th and (k+1)-th, neighbours moves x
    only by O(step).  This needs the system left without the vanishing
    neighbour to be well conditioned (with k = 4 the two remaining scored
    landmarks give a rank-one system whose weak direction is then set by
    the vanishing pairs), so k >= 6 and det/trace^2 > 1e-3 are required."""
    r = _rng(12)
    g, d = 40, 6
    hi = r.standard_normal((g, d)) * 2.0
    lo = r.uniform(0, 10, (g, 2))
    checked = 0
    for trial in range(40):
        k = int(r.choice([6, 9, 12]))
        X0 = r.standard_normal(d)
        idx, _ = O.knn(X0[None], hi, k + 1)
        for ra, rb in ((k - 2, k - 1), (k - 1, k)):
            Xc, e = _crossing_point(X0, hi[idx[0, ra]], hi[idx[0, rb]])
            eps = 1e-4 / np.sqrt(e @ e)
            ts = np.array([-3, -1, 1, 3]) * eps
            Xs = (Xc[None] + ts[:, None] * e[None]).astype(np.float32)
            i2, _ = O.knn(Xs, hi, k + 1)
            if not (np.array_equal(np.sort(i2[0, :k + 1]), np.sort(i2[1, :k + 1]))
                    and np.array_equal(np.sort(i2[2, :k + 1]), np.sort(i2[3, :k + 1]))):
                continue
            out, ratio, _ = O.project(Xs, hi, lo, k, 1.0, 1.0, diagnostics=True)
            if ratio.min() < 1e-3:
                continue
            slope = max(np.abs(out[1] - out[0]).max(), np.abs(out[3] - out[2]).max())
            jump = np.abs(out[2] - out[1]).max()
            assert jump <= 10 * slope + 1e-6, f"jump {jump:.3e} vs slope {slope:.3e}"
            checked += 1
    assert checked >= 15, checked


# --------------------------------------------------------------------------
# SOM step (reading R6 of the oracle header; used by the frame server).

def pin_som_step_limits(O):
    """sigma -> 0: each landmark moves towards the mean of the minibatch
    points whose best-matching landmarks are the nearest assigned ones to it
    on the grid (itself, if any point picked it: a k-means step with rate
    alpha); sigma -> infinity: every landmark moves towards the mean of the
    whole minibatch; alpha = 0 changes nothing."""
    r = _rng(13)
    L, d, b = 16, 5, 200
    hi = r.standard_normal((L, d)).astype(np.float32)
    lo = np.stack([np.arange(L) % 4, np.arange(L) // 4], 1).astype(np.float32)
    batch = r.standard_normal((b, d)).astype(np.float32)
    bmu = r.integers(0, L - 3, b).astype(np.int32)       # the last landmarks unassigned
    hi64, batch64 = hi.astype(np.float64), batch.astype(np.float64)
    for alpha in (0.05, 0.5, 1.0):
        out = O.som_step(hi, lo, batch, bmu, alpha, 0.05)
        assigned = np.unique(bmu)
        for j in range(L):
            g2 = ((lo[assigned] - lo[j]) ** 2).sum(1)
            near = assigned[g2 == g2.min()]
            sel = np.isin(bmu, near)
            want = hi64[j] + alpha * (batch64[sel].mean(0) - hi64[j])
            _close(out[j], want, 1e-12, f"som sigma->0 landmark {j}")
        out = O.som_step(hi, lo, batch, bmu, alpha, 1e6)
        want = hi64 + alpha * (batch64.mean(0)[None] - hi64)
        _close(out, want, 1e-9, "som sigma->inf")
    _close(O.som_step(hi, lo, batch, bmu, 0.0, 1.5), hi64, 0.0, "som alpha=0")


ALL_PINS = [pin_knn_bruteforce, pin_k2_nearest_layout_point, pin_k3_closed_form,
            pin_golden_fixtures, pin_plane_recovery, pin_weighted_least_squares,
            pin_collinear_layout, pin_layout_similarity, pin_space_similarity,
            pin_relabelling, pin_score_homogeneity, pin_score_shape,
            pin_boost_sharpness, pin_continuity_at_cutoff, pin_som_step_limits]
