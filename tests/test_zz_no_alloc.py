"""fst_viterbi_noalloc, the Viterbi entry point that allocates nothing.

It serves callers that cannot allocate device memory while decoding (a host
memory manager that owns every allocation, a latency-critical loop that must
not synchronise on cudaMalloc/cudaFree, a hard memory cap): its working
memory is a fixed device array inside the library.  These tests call it
through the C ABI and compare it with fst_viterbi, the allocating entry
point, on two calls in a row, and with the oracle, including a string with
no accepting path and the empty string.  This file is collected last on
purpose.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import synth

from gpu_util import assert_viterbi_equal, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _noalloc(lib, f, x, stream):
    import torch
    n = len(x)
    x = np.ascontiguousarray(x, np.int32)
    score = torch.full((1,), 7.0, dtype=torch.float32, device="cuda")
    path = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    olab = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    rc = lib.fst_viterbi_noalloc(f.handle, x.ctypes.data_as(ctypes.c_void_p), n,
                                 ctypes.c_void_p(score.data_ptr()), ctypes.c_void_p(path.data_ptr()),
                                 ctypes.c_void_p(olab.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    return rc, score, path[:n], olab[:n]


def test_noalloc_matches_fst_viterbi_on_two_calls_in_a_row():
    import torch
    from paper_1701_03038_gb300 import _lib
    from paper_1701_03038_gb300.fst import Fst
    lib = _lib.load()
    fa, strs = synth.make_config("c2", scale=0.02, strings=4)
    f = Fst.from_arrays(fa)
    o = oracle.Fst(fa)
    # a longer string, then a shorter one: the second call starts from the
    # first call's leftovers in the shared array
    order = sorted(range(strs.count), key=lambda b: -len(strs.get(b)))[:2]
    stream = torch.cuda.current_stream()
    for call, b in enumerate(order):
        x = strs.get(b)
        ref_score, ref_path, ref_olab, ref_rc = f.viterbi(x)  # the allocating entry point
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc, score, path, olab = _noalloc(lib, f, x, stream)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert rc == 0, lib.fst_last_error()
        # Viterbi is compared bit for bit, with fst_viterbi and with the oracle
        assert score.item() == ref_score, (call, score.item(), ref_score)
        assert np.array_equal(path.cpu().numpy(), ref_path), call
        assert np.array_equal(olab.cpu().numpy(), ref_olab), call
        assert_viterbi_equal(score.item(), path.cpu().numpy(), olab.cpu().numpy(), oracle.OK, o.viterbi(x))
        if call == 1:  # the first call may load kernel code; the second must not change free memory
            assert free_after == free_before, (free_before, free_after)


def test_noalloc_no_path_and_empty_string():
    # i.i.d. strings mostly have no accepting path: the outputs say so (-inf
    # score, -1 path) while the return code stays FST_OK (the call is
    # asynchronous); the empty string scores the best start-and-final state
    import torch
    from paper_1701_03038_gb300 import _lib
    from paper_1701_03038_gb300.fst import Fst
    lib = _lib.load()
    fa, _ = synth.make_config("c1", scale=0.2, strings=1)
    f, o = Fst.from_arrays(fa), oracle.Fst(fa)
    stream = torch.cuda.current_stream()
    iid = synth.make_strings(fa, 6, 20, 40, seed=77, kind="iid")
    seen_nopath = 0
    for b in range(iid.count):
        x = iid.get(b)
        ov = o.viterbi(x)
        rc, score, path, olab = _noalloc(lib, f, x, stream)
        torch.cuda.synchronize()
        assert rc == 0, lib.fst_last_error()
        if ov["status"] == oracle.NO_PATH:
            seen_nopath += 1
            assert score.item() == -math.inf
            assert (path.cpu().numpy() == -1).all() and (olab.cpu().numpy() == -1).all()
        else:
            assert_viterbi_equal(score.item(), path.cpu().numpy(), olab.cpu().numpy(), oracle.OK, ov)
        s_ref, p_ref, _, _ = f.viterbi(x)
        assert score.item() == s_ref and np.array_equal(path.cpu().numpy(), p_ref)
    assert seen_nopath > 0
    # n = 0: no path array is touched; the score is the best start state's
    # start plus final weight (-inf here: state 0 is not final)
    empty = np.zeros(0, np.int32)
    rc, score, _, _ = _noalloc(lib, f, empty, stream)
    torch.cuda.synchronize()
    assert rc == 0, lib.fst_last_error()
    ov = o.viterbi(empty)
    assert np.float32(score.item()) == ov["best"] or (math.isinf(ov["best"]) and score.item() == ov["best"])


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    from paper_1701_03038_gb300 import _lib
    from paper_1701_03038_gb300.fst import Fst
    lib = _lib.load()
    q = 3_000_000  # 16 bytes of frontier per state already exceed the fixed array
    fa = synth.FstArrays(q, 2, 2, np.array([0, 1], np.int32), np.array([1, 2], np.int32),
                         np.array([0, 1], np.int32), np.array([0, 1], np.int32),
                         np.array([0.5, 0.5], np.float32),
                         np.where(np.arange(q) == 0, 0, np.inf).astype(np.float32),
                         np.where(np.arange(q) == 2, 0, np.inf).astype(np.float32))
    f = Fst.from_arrays(fa)
    rc, score, _, _ = _noalloc(lib, f, np.array([0, 1], np.int32), torch.cuda.current_stream())
    assert rc == _lib.UNSUPPORTED
    assert b"beyond the fixed" in lib.fst_last_error()
    torch.cuda.synchronize()
    assert score.item() == 7.0  # nothing was launched
    s, p, _, _ = f.viterbi(np.array([0, 1], np.int32))  # the allocating entry point still works
    assert list(p) == [0, 1]
