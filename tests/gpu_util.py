"""Shared helpers of the GPU parity tests: build once, compare with the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1701_03038_gb300 import build as gbuild

# Tolerances fixed for forward-backward against the float64 oracle: log Z
# within 1e-5 relative, per-string posteriors within 1e-5 absolute; batch
# sums of posteriors within 1e-5 * max(1, |count|).
LOGZ_RTOL = 1e-5
POST_ATOL = 1e-5


def ensure_built():
    try:
        import torch
    except ImportError:  # pragma: no cover
        pytest.skip("torch missing")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gbuild.build()
    oracle.build()


def assert_viterbi_equal(got_score, got_path, got_olab, got_status, ov):
    assert got_status == ov["status"], (got_status, ov["status"])
    assert np.float32(got_score) == ov["best"] or (math.isinf(ov["best"]) and got_score == ov["best"]), \
        (got_score, ov["best"])
    assert np.array_equal(np.asarray(got_path), ov["path"]), (got_path, ov["path"])
    if got_olab is not None:
        assert np.array_equal(np.asarray(got_olab), ov["olabels"])


def assert_logz_close(got, want):
    if want == -math.inf:
        assert got == -math.inf, got
        return
    assert abs(got - want) <= LOGZ_RTOL * max(1.0, abs(want)), (got, want, got - want)


def assert_counts_close(got, want, batch=False):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    tol = POST_ATOL * np.maximum(1.0, np.abs(want)) if batch else POST_ATOL
    err = np.abs(got - want)
    bad = np.flatnonzero(err > tol)
    assert bad.size == 0, (bad[:10], got[bad[:10]], want[bad[:10]], float(err.max()))
