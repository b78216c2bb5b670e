"""Comparison helpers shared by the tests (no rendering arithmetic)."""
import numpy as np


def rel_rmse(img, ref):
    img = np.asarray(img, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    return float(np.linalg.norm(img - ref) / max(np.linalg.norm(ref), 1e-300))


def sample_mismatch(got, want, keep, rtol):
    """Samples (rows of [n,3]) whose vector error exceeds rtol * |want| (plus a
    floor of rtol * 1e-3 * max |want|), among rows selected by ``keep``."""
    got = np.asarray(got, np.float64).reshape(-1, 3)
    want = np.asarray(want, np.float64).reshape(-1, 3)
    err = np.linalg.norm(got - want, axis=1)
    scale = np.linalg.norm(want, axis=1) + 1e-3 * np.abs(want).max()
    return (err > rtol * scale) & keep
