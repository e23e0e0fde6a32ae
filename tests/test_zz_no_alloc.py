"""The allocation-free entry point, twed_batch_f32_noalloc.

Some callers cannot call cudaMalloc (code running during another thread's
global-mode graph capture, device-synchronization-free loops, plug-ins with a
fixed memory budget), so the library offers one batched call that works in
a static device array instead of allocated workspace.  Its results must
equal those of twed_batch_f32, the allocating entry point, call after call,
although every call reuses (and inherits the contents of) the same array.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2007_16135_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2007_16135_gb300 import twed
    twed.load()
    return twed


def _set(seed, nseries, lo, hi, dim):
    rng = np.random.default_rng(seed)
    out = []
    for n in rng.integers(lo, hi + 1, size=nseries):
        out.append((np.cumsum(rng.normal(size=(n, dim)), axis=0), np.cumsum(rng.exponential(1.0, n))))
    return W.pack(out).astype(np.float32)


def _call_noalloc(tw, A, B, pairs, out, nu, lam, p, stream):
    # straight through the C ABI: no handle, no allocation by the library
    lib = tw.load()
    sa, sb = A.cstruct(), B.cstruct()
    return lib.twed_batch_f32_noalloc(ctypes.byref(sa), ctypes.byref(sb),
                                      ctypes.c_void_p(pairs.data_ptr()), pairs.shape[0], A.dim,
                                      float(nu), float(lam), p, ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_batch_on_two_calls_in_a_row(tw):
    import torch
    stream = torch.cuda.current_stream()
    SA, SB = _set(1, 30, 1, 900, 4), _set(2, 21, 1, 1300, 4)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch.float32)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch.float32)
    rng = np.random.default_rng(3)
    cases = [
        (A, B, np.stack([rng.integers(0, SA.n, 400), rng.integers(0, SB.n, 400)], 1), 1.0, 1.0),
        (A, A, np.stack([rng.integers(0, SA.n, 250), rng.integers(0, SA.n, 250)], 1), 0.5, 0.25),
    ]
    for X, Y, pairs, nu, lam in cases:
        d_pairs = torch.as_tensor(pairs, dtype=torch.int64).cuda()
        want = tw.twed_batch(X, Y, d_pairs, nu, lam, 2).cpu().numpy()
        out = torch.full((len(pairs),), float("nan"), dtype=torch.float32, device="cuda")
        st = _call_noalloc(tw, X, Y, d_pairs, out, nu, lam, 2, stream)
        assert st == tw.TWED_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-30)
        assert np.all(np.isfinite(got)) and rel.max() <= 1e-5, rel.max()


def test_noalloc_rejects_requests_beyond_its_array(tw):
    import torch
    # one 2.5e6-point dim-8 series: its records alone exceed the static array;
    # the call must refuse on the host before enqueuing anything
    n = 2_500_000
    vals = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    ts = torch.arange(1, n + 1, dtype=torch.float32, device="cuda")
    offs = np.array([0, n], dtype=np.int64)
    S = tw.DeviceSet(vals, ts, torch.as_tensor(offs).cuda(), offs)
    pairs = torch.zeros((1, 2), dtype=torch.int64, device="cuda")
    out = torch.zeros(1, dtype=torch.float32, device="cuda")
    st = _call_noalloc(tw, S, S, pairs, out, 1.0, 1.0, 2, torch.cuda.current_stream())
    assert st == tw.TWED_ERR_UNSUPPORTED
