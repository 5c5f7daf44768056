"""Helpers shared by the GPU parity tests (test code, not product code)."""
import numpy as np

from oracle import march as om

MARCH_TOL = 1e-4          # max-abs per channel, FP32 march vs FP64 oracle
GRAD_TOL = 1e-3           # pixels whose shading saw a near-zero gradient
AMB_FRAC = 0.02           # flagged rays allowed: 2 % of the compared rays ...
AMB_MIN = 6               # ... or 6 rays when fewer than 300 are compared


def march_parity(vol, tf, cam, mp, gpu_rgbam, ids=None, tol=MARCH_TOL):
    """Compare a GPU march with the oracle at ``ids`` (all pixels if None).

    Unflagged pixels must agree within ``tol``.  Pixels where the oracle
    flags a discrete FP32/FP64 ambiguity (sample count within 1e-3 of an
    integer, termination within 1e-6 of the threshold; bits 0-1) may take
    either side and must then match one of the oracle's alternative results;
    they may be at most 2 % of the compared pixels (at least 6 allowed, so
    small comparisons have a floor against counting noise).  On a foveated
    1080p frame the windows flag about 1.3 % of the rays (0.16 % by the count,
    1.1 % by termination), of which 0.06 % take the other side, with margins
    of at most 1.6e-4 and 4.0e-7 (test_march_ambiguity_margins_1080p).  Pixels flagged only for a near-zero
    gradient (bit 2: the shading normal is ill-conditioned, or exactly zero in
    flat regions) must agree within GRAD_TOL.
    Returns (max error over unflagged pixels, number of discrete-ambiguous pixels).
    """
    ref, amb, _ = om.march(vol, tf, cam, mp, ids=ids)
    W, H = cam.width, cam.height
    g = np.asarray(gpu_rgbam, np.float64).reshape(5, -1)
    r = ref.reshape(5, -1)
    a = amb.reshape(-1)
    sel = np.arange(W * H) if ids is None else np.asarray(ids, np.int64)
    err = np.abs(g[:, sel] - r[:, sel]).max(axis=0)
    disc = (a[sel] & 3) != 0
    grad = ((a[sel] & 4) != 0) & ~disc
    clean = ~disc & ~grad
    clean_err = float(err[clean].max()) if clean.any() else 0.0
    assert clean_err < tol, f"march error {clean_err} at unambiguous pixels"
    if grad.any():
        assert err[grad].max() < GRAD_TOL, f"march error {err[grad].max()} at near-zero-gradient pixels"
    assert disc.sum() <= max(AMB_FRAC * disc.size, AMB_MIN), f"{disc.mean():.4f} of pixels ambiguous"
    bad = sel[(err >= tol) & disc]
    if bad.size:
        bad32 = bad.astype(np.int32)
        alts = []
        for cs, to in ((1, 0.0), (-1, 0.0), (0, mp.term_alpha + 1e-5), (0, mp.term_alpha - 1e-5)):
            alt, _, _ = om.march(vol, tf, cam, mp, ids=bad32, count_shift=cs, term_override=to)
            alts.append(np.abs(g[:, bad] - alt.reshape(5, -1)[:, bad]).max(axis=0))
        best = np.min(np.stack(alts), axis=0)
        assert best.max() < tol, f"ambiguous pixels match no alternative (err {best.max()})"
    return clean_err, int(disc.sum())
