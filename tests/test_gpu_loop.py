"""The batched LM loop run on the device (Sec. 3, residency): one CUDA-graph
launch per fit whose WHILE node repeats the LM body until the body's control
kernel finds no stamp still fitting, the body cap reached, or the time budget
spent.

- The graph loop takes exactly the steps of the same body launched directly
  (the profiled path), and on an explicit stream the same as on the legacy one.
- A time budget that runs out ends every stamp still fitting with GF_ETIMEOUT,
  keeping its last accepted parameters (the oracle's chi^2 there matches the
  reported one), and the call returns.  The wait that runs out is the
  budget's own check on the device's global timer; nothing faults or hangs.
- A budget that does not run out changes nothing; one that runs out part way
  leaves every stamp either as the unbudgeted fit left it, bit for bit, or
  stopped with GF_ETIMEOUT after no more trials than the unbudgeted fit took.
"""
import numpy as np
import pytest

import oracle
from paper_1101_2254_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gf():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1101_2254_gb300 import build, gf as gf_
    build.build()
    return gf_


@pytest.fixture(scope="module")
def case(gf):
    sts = synth.batch_stamps(24, seed=5, smin=32, smax=96)
    imgs, sigs, descs = [], [], []
    for st in sts:
        od = oracle.make_desc(st.H, st.W, st.P, st.kinds, st.os_factor, st.os_box)
        img, sig = synth.add_noise(oracle.render(od, st.params, st.psf), st.noise_seed)
        imgs.append(img); sigs.append(sig); descs.append(od)
    T = lambda xs: torch.as_tensor(np.concatenate([x.ravel() for x in xs])).cuda()  # noqa: E731
    s0 = sts[0]
    return dict(sts=sts, imgs=imgs, sigs=sigs, descs=descs, img=T(imgs), sig=T(sigs),
                psf=T([st.psf for st in sts]), p0=np.array([st.guess() for st in sts]),
                d=gf.make_desc(1, 1, s0.P, s0.kinds, s0.os_factor, 8),
                b=gf.make_batch([st.H for st in sts], [st.W for st in sts], psf_size=s0.P),
                fixed=s0.fixed)


def fit(gf, c, stream=None, **kw):
    opts = gf.default_opts(**kw)
    return gf.lm_fit_batch(c["d"], c["b"], c["p0"], c["fixed"], c["img"], c["sig"], c["psf"],
                           opts=opts, stream=stream)


def same(a, b):
    pa, ra = a
    pb, rb = b
    return np.array_equal(pa, pb) and all(x == y for x, y in zip(ra, rb))


def test_graph_loop_equals_direct_body_launches(gf, case):
    graph = fit(gf, case)
    with gf.Profiler():  # profiled calls launch the body directly, host-polled
        direct = fit(gf, case)
    assert same(graph, direct)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        other = fit(gf, case, stream=side)
    torch.cuda.synchronize()
    assert same(graph, other)
    assert all(r["status"] in (gf.OK, gf.EMAXITER) for r in graph[1])


def test_time_budget_runs_out(gf, case):
    p, res = fit(gf, case, time_budget_s=1e-9)
    assert all(r["status"] == gf.ETIMEOUT for r in res), [r["status"] for r in res]
    for i, r in enumerate(res):
        st = case["sts"][i]
        assert r["iters"] >= 1
        x_o = oracle.evaluate(case["descs"][i], p[i], st.psf, case["imgs"][i], case["sigs"][i])[0]
        assert abs(r["chi2"] - x_o) <= 1e-4 * x_o, (i, r["chi2"], x_o)
    # the context is still usable: a normal fit afterwards completes
    p2, res2 = fit(gf, case)
    assert all(r["status"] in (gf.OK, gf.EMAXITER) for r in res2)


def test_budget_that_does_not_run_out_changes_nothing(gf, case):
    assert same(fit(gf, case), fit(gf, case, time_budget_s=100.0))


def test_partial_budget(gf, case):
    full = fit(gf, case)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fit(gf, case)
    e1.record()
    e1.synchronize()
    t_full = e0.elapsed_time(e1) / 1e3
    p, res = fit(gf, case, time_budget_s=0.4 * t_full)
    for i, r in enumerate(res):
        if r["status"] == gf.ETIMEOUT:
            assert r["iters"] <= full[1][i]["iters"]
        else:
            assert np.array_equal(p[i], full[0][i]) and r == full[1][i], i


def test_bad_budget_rejected_before_launch(gf, case):
    with pytest.raises(gf.GFError) as e:
        fit(gf, case, time_budget_s=-1.0)
    assert e.value.status == gf.EINVAL
