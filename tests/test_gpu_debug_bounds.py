"""The index-checked build (libcert_debug.so, -DCERT_DEBUG_BOUNDS) on the GPU:
its kernels check, at run time, the indices the release build relies on by
construction (search ranges inside their scene, neighbour indices written
into certificates, the kNN slot ranges and lists) and would return
CERT_EINTERNAL on a violation.  The workloads below -- a mixed batch under
every strategy, a batch large enough for 16-bit counts, the kNN search with
its far and heavy paths, the all-pairs pass -- must finish with CERT_OK and
match the oracle (the 16-bit batch: the all-pairs pass, itself checked
against the oracle).  Runs in a child
process, which loads the debug library instead of the release one."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import numpy as np, torch
import oracle
from oracle import knn as K
from paper_2606_18314_b300 import cert, scenes
assert cert.LIB_PATH.endswith("libcert_debug.so"), cert.LIB_PATH
m = scenes.BatchMotion.mixed(n_scenes=12, lo=300, hi=5000, eps=2e-3, seed=41)
off, fr = m.offsets, m.frames(5)
ctx = cert.Context(torch.from_numpy(fr[0]).cuda(), offsets=off, cell_scale=2.0, audit=("rho", "geometry"))
refs = [oracle.top2(fr[0][off[s]:off[s + 1]]) for s in range(12)]
for t, strat in enumerate(["incremental", "rebuild", "allpairs", "threshold", "incremental"], start=1):
    ctx.step(torch.from_numpy(fr[t]).cuda(), 2e-3, strat)
    res, rc = ctx.sync(raise_on_status=False)
    assert rc == cert.CERT_OK, (t, cert.STATUS_NAMES[rc])
    nn = ctx.views()["nn"].cpu().numpy()
    for s in range(12):
        r = oracle.step(fr[t - 1][off[s]:off[s + 1]], fr[t][off[s]:off[s + 1]], refs[s])
        assert np.array_equal(nn[off[s]:off[s + 1]], r.cert.nn) and int(res[s]["n_failed"]) == r.n_failed
        refs[s] = r.cert
ctx.rebuild()
_, rc = ctx.sync(raise_on_status=False)
assert rc == cert.CERT_OK
ctx.close()
# a context of more than 262,144 points with every scene below 65,536: 16-bit counts
mb = scenes.BatchMotion([scenes.Motion("uniform_clusters", 60000, 3, 1e-3, seed=60 + k, steps=8) for k in range(5)])
ob, fb = mb.offsets, mb.frames(3)
cb = cert.Context(torch.from_numpy(fb[0]).cuda(), offsets=ob)
for t, strat in enumerate(["incremental", "allpairs", "incremental"], start=1):
    cb.step(torch.from_numpy(fb[t]).cuda(), 1e-3, strat)
    _, rc = cb.sync(raise_on_status=False)
    assert rc == cert.CERT_OK, ("16-bit counts", t, cert.STATUS_NAMES[rc])
    nn = cb.views()["nn"].cpu().numpy()
    for s in range(5):
        ref = cert.cert_allpairs(torch.from_numpy(fb[t][ob[s]:ob[s + 1]]).cuda())[0].cpu().numpy()
        assert np.array_equal(nn[ob[s]:ob[s + 1]], ref), ("16-bit counts", t, s)
cb.close()
mk = scenes.Motion("uniform_clusters", 6000, 3, 1e-3, seed=2, steps=20)
fk = mk.frames(3)
for scale in (0.05, 1.0, 3.0):
    kc = cert.KnnContext(torch.from_numpy(fk[0]).cuda(), 8, cell_scale=scale)
    kref = K.cert(fk[0], 8)
    for t in range(1, 4):
        kc.step(torch.from_numpy(fk[t]).cuda(), 1e-3, "incremental" if t % 2 else "rebuild")
        kres, rc = kc.sync(raise_on_status=False)
        assert rc == cert.CERT_OK, (scale, t, cert.STATUS_NAMES[rc])
        r = K.step(fk[t - 1], fk[t], kref)
        assert np.array_equal(kc.views()["idx"].cpu().numpy().T, r.cert.idx)
        kref = r.cert
    kc.close()
p = np.random.default_rng(5).random((5000, 3)).astype(np.float32)
nn, d1, d2 = cert.cert_allpairs(torch.from_numpy(p).cuda())
assert np.array_equal(nn.cpu().numpy(), oracle.top2(p).nn)
print("debug ok")
'''


def test_debug_build_runs_clean():
    from paper_2606_18314_b300 import build
    build.build(debug=True)
    env = dict(os.environ, CERT_LIB_VARIANT="debug", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    out = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0 and "debug ok" in out.stdout, (out.stdout[-2000:], out.stderr[-4000:])
