"""Write the stored oracle results used by the full-size parity tests and by
the benchmark's CPU-baseline leg.  Calls only the oracle (and the seeded input
generators); never the CUDA path.

    python tests/golden/make_golden.py [stamp512]

stamp512.json: the oracle's LM fit of the 512x512 bulge + disk + sky stamp
(Moffat 65x65 PSF, 10x10 oversampling in the central 20x20, 15 free slots),
started from the 20 %-perturbed guess, with the oracle's FFT convolution, plus
the statistical errors of the free parameters at the solution
(sqrt of the diagonal of the inverse normal matrix), and the per-call CPU
times of its Jacobian and of one evaluation.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1101_2254_gb300 import synth  # noqa: E402


def stamp512():
    st = synth.stamp512()
    d = oracle.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box)
    m_true = oracle.render(d, st.params, st.psf, method=1)
    img, sig = synth.add_noise(m_true, st.noise_seed)
    p0 = st.guess()
    t0 = time.perf_counter()
    oracle.jacobian(d, p0, st.fixed, st.psf, img, sig, method=1)
    t_jac = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.evaluate(d, p0, st.psf, img, sig, method=1)
    t_eval = time.perf_counter() - t0
    t0 = time.perf_counter()
    p, res = oracle.lm_fit(d, p0, st.fixed, st.psf, img, sig, method=1)
    t_fit = time.perf_counter() - t0
    x_true, _ = oracle.evaluate(d, st.params, st.psf, img, sig, method=1)
    # statistical errors of the free parameters at the solution: sqrt diag (J^T W J)^-1
    jac = oracle.jacobian(d, p, st.fixed, st.psf, img, sig, method=1)
    sigma = np.sqrt(np.diag(np.linalg.inv(jac["A"])))
    out = dict(workload="stamp512", method="fft", params=p.tolist(), guess=p0.tolist(),
               truth=st.params.tolist(), fixed=st.fixed.tolist(), chi2=res["chi2"],
               chi2_truth=x_true, iters=res["iters"], accepted=res["accepted"],
               status=res["status"], sigma_free=sigma.tolist(), cpu_s_fit=t_fit,
               cpu_s_jacobian=t_jac, cpu_s_eval=t_eval,
               threads=1, note="oracle LM, default oracle options (ftol=xtol=1e-8)")
    with open(os.path.join(HERE, "stamp512.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: v for k, v in out.items() if not isinstance(v, list)}))


if __name__ == "__main__":
    which = sys.argv[1:] or ["stamp512"]
    for w in which:
        globals()[w]()
