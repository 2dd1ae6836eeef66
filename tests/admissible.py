"""Distance of a float32 result to the oracle's admissible set of results.

``oracle.render_set`` (and its whole-view and window forms) returns, per
pixel, the exact result and every other result a float32 evaluation may give
where a threshold decision sits within float32 error of its threshold.  A
GPU pixel is correct when it lies within the tolerance of one of them; these
helpers measure that distance on every pixel (none is skipped).
"""
import numpy as np


def set_distance(ref, img, T=None):
    """Per pixel [H, W], the smallest max-abs distance of the GPU result
    (img [3, H, W], and T [H, W] when given) to a result of the set."""
    img = np.asarray(img, np.float64)
    H, W = img.shape[1:]
    d = np.abs(img - ref["img"]).max(0)
    if T is not None:
        d = np.maximum(d, np.abs(np.asarray(T, np.float64) - ref["T_final"]))
    d = d.reshape(-1)
    alt, off = ref["alt"], ref["alt_off"]
    if len(alt):
        pix = np.repeat(np.arange(H * W), np.diff(off))
        flat = img.reshape(3, -1)
        da = np.abs(flat[:, pix].T - alt[:, :3]).max(1)
        if T is not None:
            da = np.maximum(da, np.abs(np.asarray(T, np.float64).reshape(-1)[pix] - alt[:, 3]))
        np.minimum.at(d, pix, da)
    return d.reshape(H, W)


def n_contrib_matches(ref, img, T, nc, tol):
    """Per pixel: does some result of the set lie within ``tol`` of the GPU
    image and T_final and have the GPU's n_contrib?"""
    img = np.asarray(img, np.float64)
    H, W = img.shape[1:]
    nc = np.asarray(nc).reshape(-1).astype(np.int64)
    d0 = np.maximum(np.abs(img - ref["img"]).max(0), np.abs(np.asarray(T, np.float64) - ref["T_final"])).reshape(-1)
    ok = (d0 <= tol) & (ref["n_contrib"].reshape(-1) == nc)
    alt, off = ref["alt"], ref["alt_off"]
    if len(alt):
        pix = np.repeat(np.arange(H * W), np.diff(off))
        flat = img.reshape(3, -1)
        da = np.maximum(np.abs(flat[:, pix].T - alt[:, :3]).max(1),
                        np.abs(np.asarray(T, np.float64).reshape(-1)[pix] - alt[:, 3]))
        hit = (da <= tol) & (alt[:, 4].astype(np.int64) == nc[pix])
        np.logical_or.at(ok, pix, hit)
    return ok.reshape(H, W)


def summary(ref, dist, tol):
    """Counts for reports: pixels, pixels with other admissible results, the
    largest distance, pixels farther than tol from the set, incomplete sets."""
    return {"pixels": int(dist.size), "ambiguous_px": int((ref["flags"] & 1).sum()),
            "max_set_err": float(dist.max()) if dist.size else 0.0, "unchecked_px": 0,
            "outside_px": int((dist > tol).sum()), "incomplete_sets": int((ref["flags"] & 4).sum()),
            "max_results_per_px": int(np.diff(ref["alt_off"]).max() + 1) if dist.size else 1}
