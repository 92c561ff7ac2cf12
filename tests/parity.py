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
    of the 2-D landmarks over both axes) for every point whose oracle normal
    matrix has det/trace^2 >= 1e-3 (condition number <= ~1e3; every point of
    the named workloads sits there) and for rank-one / zero systems
    (det/trace^2 < 1e-11 or A = 0).  Between those, FP32 sums of the normal
    system carry ~1e-7 relative error that the solve amplifies by the
    condition number, so the bound is scaled by 1e-3 / (det/trace^2); these
    points are counted ("ill_conditioned").  Points within 10x of the
    rank-one threshold (1e-11 <= det/trace^2 < 1e-9) may take the other
    branch under rounding and are exempt; they are counted ("exempt").
"""
from __future__ import annotations

import numpy as np

COORD_TOL = 1e-4
TIE_REL = 1e-6
DIST_REL = 1e-5
DET_EXEMPT_LO = 1e-11
DET_EXEMPT_HI = 1e-9
COND_KNEE = 1e-3


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
    strict = ~exempt & ~ill
    base = tol * extent
    bound = np.where(ill, base * COND_KNEE / np.maximum(ratio, 1e-300), base)
    stats = {
        "n": int(len(err)),
        "exempt": int(exempt.sum()),
        "ill_conditioned": int(ill.sum()),
        "max_err": float(err[strict].max()) if strict.any() else 0.0,
        "p99_err": float(np.percentile(err[strict], 99)) if strict.any() else 0.0,
        "max_err_ill": float(err[ill].max()) if ill.any() else 0.0,
        "bound": base,
        "far_points": int((np.abs(ref).max(axis=1) > 2 * extent).sum()),
    }
    bad = np.nonzero(~exempt & ~(err <= bound))[0]
    if bad.size:
        w = bad[np.argmax(err[bad] / bound[bad])]
        raise AssertionError(
            f"{bad.size} of {len(err)} points beyond their bound: worst {err[w]:.3e} > "
            f"{bound[w]:.3e} at {w} (det ratio {ratio[w]:.2e}); {stats}")
    return stats
