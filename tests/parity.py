"""Helpers shared by the GPU parity tests (test code, not product code)."""
import numpy as np

from oracle import march as om

MARCH_TOL = 1e-4          # max-abs per channel, FP32 march vs FP64 oracle


def march_parity(vol, tf, cam, mp, gpu_rgbam, ids=None, tol=MARCH_TOL, max_amb_frac=0.01):
    """Compare a GPU march with the oracle at ``ids`` (all pixels if None).

    Pixels where the oracle flags an FP32/FP64 discontinuity (sample count
    at an integer, termination at the threshold, vanishing gradient) may take
    either side: they must match one of the oracle's alternative results.
    Returns (max error over unambiguous pixels, number of ambiguous pixels).
    """
    ref, amb, _ = om.march(vol, tf, cam, mp, ids=ids)
    W, H = cam.width, cam.height
    g = np.asarray(gpu_rgbam, np.float64).reshape(5, -1)
    r = ref.reshape(5, -1)
    a = amb.reshape(-1)
    sel = np.arange(W * H) if ids is None else np.asarray(ids, np.int64)
    err = np.abs(g[:, sel] - r[:, sel]).max(axis=0)
    amb_sel = a[sel] != 0
    clean_err = float(err[~amb_sel].max()) if (~amb_sel).any() else 0.0
    assert clean_err < tol, f"march error {clean_err} at unambiguous pixels"
    assert amb_sel.mean() <= max_amb_frac, f"{amb_sel.mean():.4f} of pixels ambiguous"
    bad = sel[(err >= tol) & amb_sel]
    if bad.size:
        bad32 = bad.astype(np.int32)
        alts = []
        for cs, to in ((1, 0.0), (-1, 0.0), (0, mp.term_alpha + 1e-5), (0, mp.term_alpha - 1e-5)):
            alt, _, _ = om.march(vol, tf, cam, mp, ids=bad32, count_shift=cs, term_override=to)
            alts.append(np.abs(g[:, bad] - alt.reshape(5, -1)[:, bad]).max(axis=0))
        best = np.min(np.stack(alts), axis=0)
        assert best.max() < tol, f"ambiguous pixels match no alternative (err {best.max()})"
    return clean_err, int(amb_sel.sum())
