"""Cube comparison used by the parity tests.

Criterion (FP32 path vs FP64 oracle): every voxel whose oracle value is above `thresh` x
peak agrees to `rtol` relative. Voxels below that level are held to an absolute bound of
`small_abs` x peak: in optically thin line wings the FP32 transmittance near 1 carries the
hardware exp2 error (at most about 1.2e-7 absolute, measured), which enters the intensity
as about S x 1.2e-7 <= 1.2e-7 x peak.
"""

import numpy as np


def cube_errors(gpu, ref, thresh=1e-3):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    peak = float(np.abs(ref).max())
    big = np.abs(ref) > thresh * peak
    rel = np.abs(gpu - ref)[big] / np.abs(ref)[big] if big.any() else np.zeros(1)
    small_abs = np.abs(gpu - ref)[~big] / peak if (~big).any() else np.zeros(1)
    return dict(peak=peak, n_big=int(big.sum()), max_rel=float(rel.max()),
                p99_rel=float(np.percentile(rel, 99)), max_small_abs=float(small_abs.max()))


def assert_cube_close(gpu, ref, rtol=1e-4, thresh=1e-3, small_abs=3e-7, label=""):
    e = cube_errors(gpu, ref, thresh)
    assert np.all(np.isfinite(np.asarray(gpu))), f"{label}: non-finite values"
    assert e["max_rel"] <= rtol, f"{label}: max rel err {e['max_rel']:.3e} > {rtol} ({e})"
    assert e["max_small_abs"] <= small_abs, f"{label}: sub-threshold abs err ({e})"
    return e
