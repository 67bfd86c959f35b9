"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

import oracle
from paper_1101_2254_gb300 import synth

# Per-pixel tolerance of the float32 model and convolution against the FP64
# oracle: |g - o| <= REL |o| + FLOOR max|o| (the floor covers pixels far below
# the peak, where float32 round-off is absolute rather than relative).
REL, FLOOR = 1e-5, 1e-7
CHI2_REL = 1e-4
PARAM_REL = 1e-3


def assert_pix_close(g, o, rel=REL, floor=FLOOR, what=""):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    assert g.shape == o.shape, (g.shape, o.shape)
    bound = rel * np.abs(o) + floor * np.abs(o).max()
    err = np.abs(g - o)
    bad = err > bound
    if bad.any():
        k = np.argmax(err - bound)
        idx = np.unravel_index(k, o.shape)
        raise AssertionError(f"{what}: {bad.sum()} of {o.size} pixels out of tolerance; worst at "
                             f"{idx}: gpu={g[idx]!r} oracle={o[idx]!r} err={err[idx]:.3e} "
                             f"bound={bound[idx]:.3e}")


def oracle_desc(st: synth.Stamp):
    return oracle.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box)


def gpu_desc(gf, st: synth.Stamp, conv_method=0):
    return gf.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box,
                        conv_method=conv_method)


def noisy_image(st: synth.Stamp, method=0):
    """True image rendered by the oracle, plus seeded noise."""
    m = oracle.render(oracle_desc(st), st.params, st.psf, method=method)
    img, sig = synth.add_noise(m, st.noise_seed)
    return m, img, sig


SIGMA_FRAC = 0.01


def param_bound_ok(pg, po, free, sigma, rel=PARAM_REL, sfrac=SIGMA_FRAC):
    """|pg - po| <= max(rel * max(|po|, 1), sfrac * sigma) on the free slots;
    sigma = the oracle's statistical error of each free parameter (sqrt diag of
    the inverse normal matrix at its solution).  Returns (ok, |dp|/sigma, rel err)."""
    pg, po = np.asarray(pg)[free], np.asarray(po)[free]
    dp = np.abs(pg - po)
    bound = np.maximum(rel * np.maximum(np.abs(po), 1.0), sfrac * np.asarray(sigma))
    return bool(np.all(dp <= bound)), dp / np.asarray(sigma), dp / np.maximum(np.abs(po), 1.0)


def oracle_sigma(d, p, fixed, psf, img, sig, method=0):
    r = oracle.jacobian(d, p, fixed, psf, img, sig, method=method)
    return np.sqrt(np.diag(np.linalg.inv(r["A"])))


def param_rel_err(p, q, idx):
    p = np.asarray(p)[idx]
    q = np.asarray(q)[idx]
    return np.abs(p - q) / np.maximum(np.abs(q), 1.0)
