"""Each planted mistake in a copy of the oracle must be caught by at least
one pin: evidence that the pins constrain every part of the oracle.  The
mutants are built and run on the CPU only."""
import os
import tempfile

import pytest

import oracle
import oracle_pins

# (name, exact text in esom_oracle.c, replacement).  Not listed: weighting
# the fallback centroid differently.  When the normal matrix is exactly rank
# one, every valid pair direction is parallel, which forces the scored 2-D
# landmarks onto one line (or gives them equal scores), so the centroid's
# weights cannot be observed; only near-singular systems would show them.
# Nor pairs that include the k-th neighbour: its score is 0, so they add 0.
# Nor other weights of the mean and spread (uniform instead of 1/i) or
# another cut-off steepness: no passage fixes those values (parity
# unpinned), and any such choice keeps every property the pins check.
MUTANTS = [
    ("tie_break_reversed", "return (a->j > b->j) - (a->j < b->j);",
     "return (a->j < b->j) - (a->j > b->j);"),
    ("distance_not_squared", "acc += diff * diff;", "acc += fabs(diff);"),
    ("projection_sign", "num += ((double)x[t] - (double)Lu[t]) * e;",
     "num += ((double)Lu[t] - (double)x[t]) * e;"),
    ("projection_wrong_anchor", "num += ((double)x[t] - (double)Lu[t]) * e;",
     "num += ((double)x[t] - (double)Lv[t]) * e;"),
    ("dropped_offset_term", "double rhs = D + (h0 * lu0 + h1 * lu1) / r;",
     "double rhs = D;"),
    ("transposed_off_diagonal", "A01 += w * h0 * h1 / r;", "A01 += w * h0 * h0 / r;"),
    ("adjust_as_length_power", "double w = s[u] * s[v] / pow(r, adjust);",
     "double w = s[u] * s[v] / pow(sqrt(r), adjust);"),
    ("cramer_swapped", "out[0] = (b0 * A11 - A01 * b1) / det;",
     "out[0] = (b1 * A11 - A01 * b0) / det;"),
    ("no_cutoff_factor",
     "double f2 = (dk == 0.0) ? 1.0 : 1.0 - exp(ORACLE_SCORE_EDGE * (delta / dk - 1.0));",
     "double f2 = 1.0;"),
    ("scores_increasing", "double f1 = flat ? 1.0 : exp(boost * (mean - delta) / sigma);",
     "double f1 = flat ? 1.0 : exp(boost * (delta - mean) / sigma);"),
    ("boost_ignored", "double f1 = flat ? 1.0 : exp(boost * (mean - delta) / sigma);",
     "double f1 = flat ? 1.0 : exp((mean - delta) / sigma);"),
    ("uniform_scores", "s[i - 1] = f1 * f2;", "s[i - 1] = 1.0;"),
    ("pairs_skip_last_scored", "for (int v = u + 1; v < m; ++v) {",
     "for (int v = u + 1; v < m - 1; ++v) {"),
    ("knn_drops_nearest", "idx[i] = work[i].j;", "idx[i] = work[i + (i == 0 && k < g)].j;"),
    ("som_sigma_not_squared", "double h = exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma));",
     "double h = exp(-(dx * dx + dy * dy) / (2.0 * sigma));"),
    ("som_step_sign", "l + alpha * (hi_out[(int64_t)j * d + t] / hs - l) : l;",
     "l - alpha * (hi_out[(int64_t)j * d + t] / hs - l) : l;"),
]


@pytest.fixture(scope="module")
def source():
    with open(oracle.SRC) as f:
        return f.read()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(source, name, old, new, tmp_path):
    assert source.count(old) == 1, f"mutation site for {name} not found exactly once"
    src = tmp_path / f"mutant_{name}.c"
    src.write_text(source.replace(old, new))
    so = oracle.compile_source(str(src), str(tmp_path / f"libmutant_{name}.so"))
    M = oracle.Oracle(so)
    failures = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(M)
        except AssertionError:
            failures.append(pin.__name__)
        except (ValueError, FloatingPointError, ZeroDivisionError):
            failures.append(pin.__name__)
    assert failures, f"planted mistake {name} passed every pin"
