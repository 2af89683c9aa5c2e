"""The checked build (libcde_checked.so: device index checks at every index the
kernels derive from tile, unit, chunk, split or sample positions -- the stand-in
for sanitizers, which are closed on this pool).  Every entry point runs on
ragged cases in a fresh process with each library; the checked build must
report no failed check, and its results must equal the normal library's."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT_PATH)
from paper_1206_5278_gb300 import cde, synth

def L(a):
    return np.asarray(a, dtype=np.float64).ravel().tolist()

ctx = cde.cde_init(0)
out = {}
cases = [(1031, 9, 33, 5, "gauss"), (257, 3, 9, 17, "gauss"), (333, 2, 5, 7, "epan"), (700, 1, 16, 8, "gauss")]
dss = []
for n, d, g1, g2, k in cases:
    x, y = synth.random_small(n, d, seed=n + d)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=(d > 1), kernel=k)
    dss.append(ds)
    h1 = synth.bandwidth_grid(0.05, 3.0, g1)
    h2 = synth.bandwidth_grid(0.02, 2.0, g2)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    out["loo_%d" % n] = L(Lc) + L(Le)
    out["rows_%d" % n] = L(cde.cde_loo_rows(ctx, ds, h1, h2, [0, n // 2, n - 1]))
    if g1 <= 32 and g2 <= 32:
        import torch
        dc = torch.empty(g1 * g2, dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        cde.cde_loo_loglik_noalloc(ctx, ds, h1, h2, dc, None, stream=s)
        s.synchronize()
        out["noalloc_%d" % n] = L(dc.cpu().numpy())
bh1 = [synth.bandwidth_grid(0.1, 2.0, g) for g in (8, 16, 5)]
bh2 = [synth.bandwidth_grid(0.05, 1.0, g) for g in (8, 16, 7)]
Lc, Le = cde.cde_loo_loglik_batch(ctx, dss[1:], bh1, bh2)
out["batch"] = sum((L(a) + L(b) for a, b in zip(Lc, Le)), [])
for d, h1, h2, n in ((3, 0.05, 0.005, 900), (20, 0.3, 0.005, 517)):
    w = synth.grad_workload(N=n, d=d, seed=7)
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True)
    out["grad_%d" % d] = L(cde.cde_loo_grad_rows(ctx, ds, h1, h2))
for k in ("gauss", "epan"):
    x, y = synth.gmm_sine(1000, 3, seed=5)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True, kernel=k)
    xq = synth.query_points(x, 37, seed=1)
    yg = synth.y_grid(y, 0.2, 300)
    out["density_" + k] = L(cde.cde_density(ctx, ds, 0.6, 0.2, xq, yg))
    m, f = cde.cde_cond_stats(ctx, ds, 0.6, 0.2, xq, y[:37])
    out["stats_" + k] = L(m) + L(f)
    lo, hi, sm = cde.cde_cond_interval(ctx, ds, 0.6, 0.2, xq[:5], S=300, alpha=0.1, seed=3, samples=True)
    out["interval_" + k] = L(lo) + L(hi) + L(sm)
    sel = cde.cde_select_random(ctx, ds, 5.0, 2.0, 1, 5, 7, seed=9)
    out["select_" + k] = [sel["h1"], sel["h2"], sel["L_cond"], sel["L_eq3"]]
code, enabled = cde.cde_check_status(ctx)
out["check"] = [code, enabled]
cde.cde_shutdown(ctx)
print(json.dumps(out))
'''.replace("ROOT_PATH", repr(ROOT))


def _run(variant):
    env = dict(os.environ)
    env.pop("CDE_LIBRARY", None)
    if variant == "checked":
        env["CDE_LIBRARY"] = "checked"
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_reports_no_failed_check_and_matches():
    from paper_1206_5278_gb300 import _build
    _build.build(checks=True)
    normal = _run("normal")
    checked = _run("checked")
    assert normal["check"] == [0, False]
    assert checked["check"] == [0, True], "failed device index check, code %d" % checked["check"][0]
    for key, v in normal.items():
        if key == "check":
            continue
        a = [x if x == x else "nan" for x in v]
        b = [x if x == x else "nan" for x in checked[key]]
        assert a == b, key
