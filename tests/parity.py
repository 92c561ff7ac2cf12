"""Comparison of the CUDA path with the FP64 oracle.

Tolerances (stated here, used by every parity test):
  * k-NN indices: identical, except at a rank where the two landmarks'
    squared distances, recomputed in FP64, differ by at most 1e-6 relative
    (a tie at FP32 resolution); the GPU's k landmarks must still be distinct
    and their FP64 distances must equal the oracle's k smallest within 1e-6
    relative.
  * k-NN distances (FP32): within 1e-5 relative of the oracle's FP64 values
    (the FP32 sum of d squared differences carries at most ~(d/4+3) * 2^-24
    relative error with four partial sums).
  * Coordinates: |x_gpu - x_oracle| <= 1e-4 * layout extent (the largest range
    of the 2-D landmarks over both axes) for every point, the bound stated for
    the FP32 path.  The one exemption: points whose oracle normal matrix lies
    within 10x of the rank-one threshold of the solve (1e-11 <= det/trace^2 <
    1e-9) may take the other branch under rounding; they are counted
    ("exempt").  Points with 1e-9 <= det/trace^2 < 1e-3 are held to the same
    bound and counted ("ill_conditioned"); the CUDA path recomputes such
    points in FP64 because FP32 sums cannot resolve them.
"""
from __future__ import annotations

import numpy as np

COORD_TOL = 1e-4
TIE_REL = 1e-6
DIST_REL = 1e-5
DET_EXEMPT_LO = 1e-11
DET_EXEMPT_HI = 1e-9
COND_KNEE = 1e-3        # det/trace^2 below this counts as ill-conditioned


def knn_mismatches(X, hi, gidx, gd2, oidx, od2, tie_rel=TIE_REL, dist_rel=DIST_REL):
    """Checks GPU k-NN against the oracle; returns (n_rank_diffs, n_tie_ok)."""
    X64, hi64 = X.astype(np.float64), hi.astype(np.float64)
    n, k = oidx.shape
    diff_rows = np.nonzero(np.any(gidx != oidx, axis=1))[0]
    ties = 0
    for i in diff_rows:
        g = gidx[i]
        assert len(set(g.tolist())) == k, f"row {i}: repeated landmark {g}"
        assert g.min() >= 0 and g.max() < hi.shape[0], f"row {i}: index out of range"
        dg = ((X64[i][None, :] - hi64[g]) ** 2).sum(1)
        for r in np.nonzero(g != oidx[i])[0]:
            ref = od2[i, r]
            assert abs(dg[r] - ref) <= tie_rel * max(ref, 1e-30), (
                f"row {i} rank {r}: gpu landmark {g[r]} (d2 {dg[r]:.9g}) vs oracle "
                f"{oidx[i, r]} (d2 {ref:.9g})")
            ties += 1
        assert np.allclose(np.sort(dg), od2[i], rtol=tie_rel, atol=0), f"row {i}: k-set differs"
    if gd2 is not None:
        # FP32 distances of the landmarks the GPU chose, against FP64
        ref = ((X64[:, None, :] - hi64[gidx]) ** 2).sum(-1)
        rel = np.abs(gd2.astype(np.float64) - ref) / np.maximum(ref, 1e-30)
        assert rel.max() <= dist_rel, f"dist2 relative error {rel.max():.3e} > {dist_rel}"
    return len(diff_rows), ties


def coord_errors(gpu, ref, ratio, extent, tol=COORD_TOL):
    """Checks coordinates; returns a dict of error statistics."""
    gpu = np.asarray(gpu, np.float64)
    err = np.abs(gpu - ref).max(axis=1)
    exempt = (ratio >= DET_EXEMPT_LO) & (ratio < DET_EXEMPT_HI)
    ill = (ratio >= DET_EXEMPT_HI) & (ratio < COND_KNEE)
    checked = ~exempt
    bound = tol * extent
    stats = {
        "n": int(len(err)),
        "exempt": int(exempt.sum()),
        "ill_conditioned": int(ill.sum()),
        "max_err": float(err[checked].max()) if checked.any() else 0.0,
        "p99_err": float(np.percentile(err[checked], 99)) if checked.any() else 0.0,
        "max_err_ill": float(err[ill].max()) if ill.any() else 0.0,
        "bound": bound,
        "far_points": int((np.abs(ref).max(axis=1) > 2 * extent).sum()),
    }
    bad = np.nonzero(checked & ~(err <= bound))[0]
    if bad.size:
        w = bad[np.argmax(err[bad])]
        raise AssertionError(
            f"{bad.size} of {len(err)} points beyond {bound:.3e}: worst {err[w]:.3e} "
            f"at {w} (det ratio {ratio[w]:.2e}); {stats}")
    return stats


def report(stats, label=""):
    """Prints a PARITY line and records the counts in the pytest summary (a
    warning, so that -q runs keep it)."""
    import json
    import warnings
    print("PARITY", json.dumps({**stats, "label": label}))
    if stats.get("exempt") or stats.get("ill_conditioned"):
        warnings.warn(f"parity {label}: exempt={stats['exempt']} "
                      f"ill_conditioned={stats['ill_conditioned']} "
                      f"max_err_ill={stats['max_err_ill']:.2e} of bound {stats['bound']:.2e}")
