"""Image comparison used by the ray-tracer parity tests.

The ray tracer's tolerance is 1e-5 relative: every pixel brighter than 1e-3
of its image's maximum must agree with the FP64 oracle to 1e-5 of its own
value, and every dimmer pixel to 1e-5 of the maximum.
"""
import numpy as np


def assert_images_close(img, ref, rtol=1e-5, floor=1e-3):
    img = np.asarray(img, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert img.shape == ref.shape, (img.shape, ref.shape)
    lead = ref.shape[:-2]
    for idx in np.ndindex(*lead):
        a, b = img[idx], ref[idx]
        mx = float(np.abs(b).max())
        err = np.abs(a - b)
        bright = np.abs(b) > floor * mx
        bound = np.where(bright, rtol * np.abs(b), rtol * mx) + 1e-37
        bad = err > bound
        if bad.any():
            w = np.unravel_index(np.argmax(err / bound), err.shape)
            raise AssertionError(
                f"image {idx}: {int(bad.sum())} of {err.size} pixels outside {rtol:g} "
                f"(worst {w}: {a[w]!r} vs {b[w]!r}, relative {err[w] / max(abs(b[w]), 1e-300):.3e}, "
                f"of the maximum {err[w] / max(mx, 1e-300):.3e})")
