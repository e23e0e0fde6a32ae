"""The allocation-free entry point, twed_batch_f32_noalloc.

Some callers cannot call cudaMalloc (loops that must not synchronize the
device, latency-bound paths that must not wait on the allocator, plug-ins
with a fixed memory budget), so the library offers one batched call that works in
a static device array instead of allocated workspace.  Its results must
equal those of twed_batch_f32, the allocating entry point, call after call,
although every call reuses (and inherits the contents of) the same array;
they are also checked against the FP64 oracle directly, and the device's
free memory must not change across the calls after the first.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
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


def _free_bytes():
    import torch
    free, _total = torch.cuda.mem_get_info()
    return free


def test_noalloc_matches_batch_on_two_calls_in_a_row(tw):
    import torch
    stream = torch.cuda.current_stream()
    SA, SB = _set(1, 30, 1, 900, 4), _set(2, 21, 1, 1300, 4)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch.float32)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch.float32)
    rng = np.random.default_rng(3)
    cases = [
        (A, B, SA, SB, np.stack([rng.integers(0, SA.n, 400), rng.integers(0, SB.n, 400)], 1), 1.0, 1.0),
        (A, A, SA, SA, np.stack([rng.integers(0, SA.n, 250), rng.integers(0, SA.n, 250)], 1), 0.5, 0.25),
    ]
    prepared = []
    for X, Y, SX, SY, pairs, nu, lam in cases:
        d_pairs = torch.as_tensor(pairs, dtype=torch.int64).cuda()
        want = tw.twed_batch(X, Y, d_pairs, nu, lam, 2).cpu().numpy()
        ref = oracle.twed_pairs(SX.astype(np.float64).as_tuple(), SY.astype(np.float64).as_tuple(),
                                pairs, nu, lam, 2)
        out = torch.full((len(pairs),), float("nan"), dtype=torch.float32, device="cuda")
        prepared.append((X, Y, d_pairs, nu, lam, want, ref, out))
    torch.cuda.synchronize()
    for call, (X, Y, d_pairs, nu, lam, want, ref, out) in enumerate(prepared):
        reserved = torch.cuda.memory_reserved()
        free0 = _free_bytes()
        st = _call_noalloc(tw, X, Y, d_pairs, out, nu, lam, 2, stream)
        assert st == tw.TWED_OK
        torch.cuda.synchronize()
        if call > 0:  # the first call on the device may load kernels; later ones allocate nothing
            assert _free_bytes() == free0
        assert torch.cuda.memory_reserved() == reserved
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        # the allocating entry point's result, within the FP32 tolerance of the tests
        rel = np.abs(got - want) / np.maximum(np.abs(want), 1e-30)
        assert rel.max() <= 1e-5, rel.max()
        # and the oracle's (FP64 on the same FP32-rounded inputs)
        rel_o = np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1e-300)
        assert rel_o.max() <= 1e-5, rel_o.max()


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


def _fits(total_points, max_len, rec_bytes):
    """The documented size rule: 256 bytes of control words, the records
    (256-byte aligned) and four boundary rows of 8 x (longest + 2) bytes."""
    cap = 32 * 1024 * 1024
    rows_at = -(-(256 + rec_bytes * total_points) // 256) * 256
    row = 8 * ((max_len + 2) & ~1)
    return rows_at <= cap and (cap - rows_at) // row >= 4


def test_noalloc_size_limit_is_the_documented_one(tw):
    import torch
    # dim 1: 16-byte records.  One long series sets the boundary-row size; the
    # only pair run is between two short series, so the kernel work is tiny.
    short = 10
    L = 600_000
    while _fits(L + 2 + short, L + 2, 16):
        L += 2
    assert _fits(L + short, L, 16) and not _fits(L + 2 + short, L + 2, 16)
    stream = torch.cuda.current_stream()
    for n, ok in ((L, True), (L + 2, False)):
        rng = np.random.default_rng(n)
        S = W.pack([(np.cumsum(rng.normal(size=(n, 1)), axis=0), np.arange(1, n + 1, dtype=np.float64)),
                    (rng.normal(size=(short, 1)), np.arange(1, short + 1, dtype=np.float64))]).astype(np.float32)
        D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
        pairs = torch.tensor([[1, 1]], dtype=torch.int64, device="cuda")
        out = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
        st = _call_noalloc(tw, D, D, pairs, out, 1.0, 1.0, 2, stream)
        torch.cuda.synchronize()
        if ok:
            assert st == tw.TWED_OK
            assert out.item() == 0.0  # TWED(a, a) = 0
        else:
            assert st == tw.TWED_ERR_UNSUPPORTED


def test_noalloc_wide_dim_two_calls(tw):
    # dim 28 at p = 2 runs the wide strips here (their kernel loaded at the
    # first call's set-up), series of up to 300 points; the second call
    # allocates nothing and both match the oracle
    import torch
    stream = torch.cuda.current_stream()
    SA, SB = _set(11, 12, 1, 300, 28), _set(12, 9, 1, 260, 28)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch.float32)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch.float32)
    rng = np.random.default_rng(13)
    pairs = np.stack([rng.integers(0, SA.n, 90), rng.integers(0, SB.n, 90)], 1)
    d_pairs = torch.as_tensor(pairs, dtype=torch.int64).cuda()
    ref = oracle.twed_pairs(SA.astype(np.float64).as_tuple(), SB.astype(np.float64).as_tuple(), pairs, 1.0, 1.0, 2)
    out = torch.full((len(pairs),), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    for call in range(2):
        free0 = _free_bytes()
        assert _call_noalloc(tw, A, B, d_pairs, out, 1.0, 1.0, 2, stream) == tw.TWED_OK
        torch.cuda.synchronize()
        if call > 0:
            assert _free_bytes() == free0
        got = out.cpu().numpy().astype(np.float64)
        assert (np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)).max() <= 1e-5
        out.fill_(float("nan"))
