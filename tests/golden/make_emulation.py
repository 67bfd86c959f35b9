"""Write tests/golden/stamp512_f32.json: the oracle's LM fit of the 512x512
bulge + disk + sky stamp (the one in stamp512.json: same image, start and FFT
convolution) with the single-precision storage emulation on -- every
component pixel value and every convolved model pixel rounded to float32, the
GPU path's storage precision, all arithmetic still FP64 -- at the default
tolerances (1e-8) and at the benchmark's (1e-6).  The distances of these
endpoints from the FP64 fit, in units of the parameters' statistical errors,
show how far float32 storage alone moves the end of this fit along its flat
bulge/disk valley.  Calls only the oracle and the seeded input generators.

    python tests/golden/make_emulation.py
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


def main():
    with open(os.path.join(HERE, "stamp512.json")) as fh:
        gold = json.load(fh)
    st = synth.stamp512()
    d = oracle.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box)
    m_true = oracle.render(d, st.params, st.psf, method=1)
    img, sig = synth.add_noise(m_true, st.noise_seed)
    free = np.array(gold["fixed"]) == 0
    p64 = np.array(gold["params"])
    sigma = np.array(gold["sigma_free"])
    out = {"workload": "stamp512", "emulation": "component pixels and convolved model pixels "
           "rounded to float32; FP64 arithmetic", "fits": {}}
    for tol in (1e-8, 1e-6):
        oracle.set_f32_emulation(True)
        t0 = time.perf_counter()
        p, r = oracle.lm_fit(d, st.guess(), st.fixed, st.psf, img, sig, method=1,
                             opts=oracle.default_opts(ftol=tol, xtol=tol))
        dt = time.perf_counter() - t0
        oracle.set_f32_emulation(False)
        x64, _ = oracle.evaluate(d, p, st.psf, img, sig, method=1)
        dist = np.abs(p - p64)[free] / sigma
        out["fits"][f"{tol:g}"] = dict(params=p.tolist(), chi2_emulated=r["chi2"], chi2_fp64=x64,
                                       iters=r["iters"], accepted=r["accepted"],
                                       status=r["status"], max_sigma_distance=float(dist.max()),
                                       sigma_distance=dist.tolist(), cpu_s=dt)
        print(tol, r, "chi2 fp64", x64, "max |dp|/sigma", dist.max(), flush=True)
    with open(os.path.join(HERE, "stamp512_f32.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
