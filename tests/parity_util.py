"""Helpers shared by the GPU parity tests (comparison rules, not arithmetic)."""
import numpy as np

# Section 2.1 dose in FP32 with fast exponentials against the FP64 oracle:
# |D_gpu - D_oracle| <= 0.5 % of the oracle's maximum dose, per voxel.
DOSE_TOL = 5e-3


def assert_dose_close(got, want, amb=None, tol=DOSE_TOL, label=""):
    """Per-voxel bound tol * max(want); voxels where a pair's ROI or depth-range
    decision lies within rounding of its boundary may differ by that pair's
    dose as well (amb = sum of those pairs' |f_i D_i| from the oracle)."""
    got = np.asarray(got, np.float64).reshape(-1)
    want = np.asarray(want, np.float64).reshape(-1)
    assert np.all(np.isfinite(got)), f"{label}: non-finite dose"
    dmax = float(np.abs(want).max())
    bound = tol * dmax + (0.0 if amb is None else np.asarray(amb, np.float64).reshape(-1))
    err = np.abs(got - want)
    bad = np.flatnonzero(err > bound + 1e-30)
    assert bad.size == 0, (f"{label}: {bad.size} voxels beyond {tol:g} of max dose; worst "
                           f"{err[bad].max() / dmax:.3e} at voxel {bad[np.argmax(err[bad])]}")
    return float(err.max() / dmax) if dmax > 0 else 0.0


def error_stats(got, want):
    got = np.asarray(got, np.float64).reshape(-1)
    want = np.asarray(want, np.float64).reshape(-1)
    dmax = float(want.max())
    hi = want >= 0.1 * dmax
    rel = np.abs(got[hi] - want[hi]) / want[hi]
    return dict(max_over_dmax=float(np.abs(got - want).max() / dmax),
                mean_rel_hi=float(rel.mean()), p99_rel_hi=float(np.percentile(rel, 99)))
