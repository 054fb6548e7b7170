"""Small assertion helpers shared by the tests."""
import numpy as np


def assert_within(got, ref, tol, what=""):
    """|got - ref| <= tol elementwise (tol may be an array broadcastable to got)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    err = np.abs(got - ref)
    tol = np.broadcast_to(np.asarray(tol, dtype=float), err.shape)
    bad = ~(err <= tol)
    if bad.any():
        ratio = np.max(err[bad] / np.maximum(tol[bad], 1e-300))
        idx = np.unravel_index(np.argmax(np.where(bad, err / np.maximum(tol, 1e-300), 0)),
                               err.shape)
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} entries exceed tolerance; "
                             f"worst ratio {ratio:.3g} at {idx} (got {got[idx]!r}, "
                             f"ref {ref[idx]!r}, tol {tol[idx]!r})")
