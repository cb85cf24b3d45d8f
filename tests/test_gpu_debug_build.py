"""The bounds-checked build (compiled with FST_DEBUG): the frontier kernels
check every computed index into the staging buffers, the live pool, the
dense accumulators and the arc records against its buffer.  The batched and
single-string paths run through that build in a child process (the library
is loaded once per process) on inputs that exercise the drivers, layouts
and failure paths; the results must match the oracle and no check may have
fired."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    import numpy as np, torch
    import oracle
    from paper_1701_03038_gb300 import synth, _lib
    from paper_1701_03038_gb300.fst import Fst, debug_checks
    from gpu_util import assert_counts_close, assert_logz_close, assert_viterbi_equal

    assert debug_checks()["violations"] == 0
    fa, strs = synth.make_config("c2", scale=0.02, strings=40)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    ids = torch.from_numpy(strs.ids).cuda(); off = torch.from_numpy(strs.offsets).cuda()
    B, N = strs.count, len(strs.ids)
    ofb = o.fb_batch(strs.ids, strs.offsets, nthreads=8)
    ov = [o.viterbi(strs.get(b)) for b in range(B)]
    def check(pv, pf):
        torch.cuda.synchronize()
        sc, pa, ol, st = pv.scores.cpu().numpy(), pv.paths.cpu().numpy(), pv.olabels.cpu().numpy(), pv.status.cpu().numpy()
        for b in range(B):
            lo, hi = strs.offsets[b], strs.offsets[b + 1]
            assert_viterbi_equal(sc[b], pa[lo:hi], ol[lo:hi], st[b], ov[b])
            assert_logz_close(pf.logz[b].item(), ofb["logz"][b])
        assert_counts_close(pf.counts.cpu().numpy(), ofb["counts"], batch=True)
    for flags, parts, driver, pull in ((0, 1, 0, 0), (_lib.PLAN_DENSE_ACC, 1, 0, 0), (_lib.PLAN_DENSE_ACC, 3, 0, 1),
                                       (0, 3, 0, 0), (_lib.PLAN_DENSE_ACC, 1, 1, 0), (0, 1, 1, 0)):
        pv = f.plan(ids, off, flags=_lib.PLAN_NO_FB | flags, parts=parts)
        pf = f.plan(ids, off, flags=_lib.PLAN_NO_VITERBI | flags, parts=parts)
        if driver:
            pv.set_driver(_lib.DRIVER_PERSISTENT); pf.set_driver(_lib.DRIVER_PERSISTENT)
        pf.set_pull(pull)
        for _ in range(2):
            pv.viterbi(); pf.forward_backward()
            check(pv, pf)
        if not driver:
            # an overflowing run and the exact run after it
            pv.limit_pool(8); pf.limit_pool(8)
            pv.viterbi(); pf.forward_backward(); torch.cuda.synchronize()
            assert (pf.status[:B].cpu().numpy() == _lib.OOM).all()
            pv.limit_pool(0); pf.limit_pool(0)
            pv.viterbi(); pf.forward_backward()
            check(pv, pf)
    # single strings: frontier kernels, both drivers
    for driver in (_lib.DRIVER_LAUNCH, _lib.DRIVER_PERSISTENT):
        f.set_plain_driver(driver, 0)
        f.set_plain_method(_lib.PLAIN_FRONTIER)
        for b in range(0, B, 5):
            x = strs.get(b)
            s, p, ol, st = f.viterbi(x)
            assert_viterbi_equal(s, p, ol, st, ov[b])
            lz, cnt, _ = f.forward_backward(x)
            assert_logz_close(lz, o.forward_backward(x)["logz"])
    r = debug_checks()
    print("VIOLATIONS", r["violations"], r["code"], r["index"], r["bound"])
""")


def test_debug_build_has_no_violations(tmp_path):
    from paper_1701_03038_gb300 import build
    lib = build.build_debug(str(tmp_path / "libfstgpu_debug.so"))
    env = dict(os.environ, FSTGPU_LIB=lib)
    script = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", script], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("VIOLATIONS")][-1]
    assert line.split()[1] == "0", line
