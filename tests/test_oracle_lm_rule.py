"""Pins of the oracle LM's finishing rule (steps 4-5 of the loop, Sec. 2) on
hand-made one-parameter problems fed to its core through callbacks.

The rule (Marquardt's damping with MINPACK's pairing of actual and predicted
reductions): an accepted trial ends the fit only if chi^2 fell by less than
ftol relative AND the linearised model also predicted a relative fall below
ftol.  The predicted fall of the damped step is delta^T (g + lambda diag(A) delta).
A step that barely lowers chi^2 while its prediction is large must therefore
not end the fit; one whose prediction is small too must.
"""
import ctypes as C

import oracle

NORMAL = C.CFUNCTYPE(C.c_double, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                     C.POINTER(C.c_double))
EVAL = C.CFUNCTYPE(C.c_double, C.c_void_p, C.POINTER(C.c_double))
PROJECT = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(C.c_double))
XSCALE = C.CFUNCTYPE(C.c_double, C.c_void_p, C.c_int)


class Problem(C.Structure):
    _fields_ = [("nslots", C.c_int), ("nfree", C.c_int), ("free_slots", C.POINTER(C.c_int)),
                ("normal", NORMAL), ("eval", EVAL), ("project", PROJECT),
                ("xscale", XSCALE), ("ctx", C.c_void_p)]


def _run(g_first, chi2_0=100.0, small_fall=1e-10, ftol=1e-8):
    """One free parameter p.  The first normal equations are A = 1, g = g_first
    at chi^2 = chi2_0; the first trial lowers chi^2 by `small_fall` relative;
    every later normal call returns g = 0 (so the next step is zero and the
    step test ends the fit).  Returns the core's result and the number of
    normal-equation calls."""
    state = {"normal": 0, "chi2": chi2_0}

    def normal(ctx, p, A, g):
        state["normal"] += 1
        A[0] = 1.0
        g[0] = g_first if state["normal"] == 1 else 0.0
        return state["chi2"]

    def evaluate(ctx, p):
        state["chi2"] = state["chi2"] * (1.0 - small_fall)
        return state["chi2"]

    cbs = (NORMAL(normal), EVAL(evaluate), PROJECT(lambda ctx, p: None),
           XSCALE(lambda ctx, s: 1.0))
    free = (C.c_int * 1)(0)
    prob = Problem(1, 1, free, *cbs, None)
    L = oracle.lib()
    L.gfo_lm_core.restype = C.c_int
    L.gfo_lm_core.argtypes = [C.POINTER(Problem), C.POINTER(C.c_double), C.POINTER(oracle.Opts),
                              C.POINTER(oracle.Result)]
    p = (C.c_double * 1)(0.0)
    o = oracle.default_opts(ftol=ftol, xtol=1e-12)
    r = oracle.Result()
    L.gfo_lm_core(C.byref(prob), p, C.byref(o), C.byref(r))
    return r, state["normal"], p[0]


def test_small_actual_fall_with_large_prediction_does_not_stop():
    # g = 1, A = 1, lambda0 = 1e-3: delta = 1/(1.001), predicted fall ~ 1 = 1e-2 of chi^2,
    # far above ftol, while the actual fall is 1e-10 relative: the fit must go on
    # (a new Jacobian is taken), and then ends on the zero step.
    r, n_normal, p = _run(g_first=1.0)
    assert r.accepted == 1
    assert n_normal == 2, "the fit stopped on a step whose predicted fall was large"
    assert r.status == oracle.CONVERGED
    assert abs(p - 1.0 / 1.001) < 1e-15


def test_small_actual_and_predicted_fall_stops():
    # g = 1e-6: predicted fall ~ 1e-12 = 1e-14 of chi^2 (below ftol) and the actual
    # fall 1e-10 relative: the accepted step ends the fit, with no new Jacobian.
    r, n_normal, _ = _run(g_first=1e-6)
    assert r.accepted == 1
    assert n_normal == 1
    assert r.status == oracle.CONVERGED


def test_large_actual_fall_does_not_stop():
    # a real fall (1e-3 relative) goes on whatever the prediction
    r, n_normal, _ = _run(g_first=1e-6, small_fall=1e-3)
    assert r.accepted == 1 and n_normal == 2
