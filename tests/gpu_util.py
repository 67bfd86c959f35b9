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


def param_rel_err(p, q, idx):
    p = np.asarray(p)[idx]
    q = np.asarray(q)[idx]
    return np.abs(p - q) / np.maximum(np.abs(q), 1.0)
