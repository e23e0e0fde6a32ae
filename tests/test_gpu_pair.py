"""GPU parity of the one-pair entry points against the CPU oracle.

FP64: bit-identical to the oracle for p = 1, 2 (same IEEE operations in the
same order), else within 1e-12 relative.  FP32: within 1e-5 relative of the
FP64 oracle run on the same FP32-rounded inputs (arithmetic error only).
Shapes straddle the strip heights (32 * rows-per-lane) and the 32-column
boundary chunks, and include 1 x 1, 1 x m, n x 1 and prime lengths.
"""
import numpy as np
import pytest

import oracle
from paper_2007_16135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 7), (9, 1), (2, 2), (31, 33), (32, 32), (33, 65), (64, 1), (97, 3),
          (257, 300), (513, 129), (1000, 17), (300, 1031)]


@pytest.fixture(scope="module")
def tw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2007_16135_gb300 import twed
    twed.load()
    return twed


def rel_err(got, want):
    if want == 0:
        return abs(got)
    return abs(got - want) / abs(want)


def series(rng, n, dim, dtype=np.float64):
    a = np.cumsum(rng.normal(size=(n, dim)), axis=0).astype(dtype)
    t = np.cumsum(rng.exponential(1.0, n)).astype(dtype)
    return a, t


def test_w1_pair_f64_bitwise(tw):
    a, ta, b, tb = W.pair_w1()
    got = tw.twed_f64(a, ta, b, tb, 1.0, 1.0, 2)
    want = oracle.twed(a, ta, b, tb, 1.0, 1.0, 2)
    assert got == want


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("dim,p", [(1, 2), (2, 1), (3, 2), (4, 2), (5, 2), (7, 1), (8, 1), (8, 2), (3, 3),
                                   (9, 2)])
def test_pair_f64(tw, n, m, dim, p):
    rng = np.random.default_rng(n * 1000 + m * 10 + dim + 100 * p)
    a, ta = series(rng, n, dim)
    b, tb = series(rng, m, dim)
    nu, lam = 0.37, 0.81
    got = tw.twed_f64(a, ta, b, tb, nu, lam, p)
    want = oracle.twed(a, ta, b, tb, nu, lam, p)
    if p in (1, 2):
        assert got == want, (got, want)
    else:
        assert rel_err(got, want) <= 1e-12


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("dim,p", [(1, 2), (3, 2), (4, 1), (8, 2), (6, 2), (2, 3)])
def test_pair_f32(tw, n, m, dim, p):
    rng = np.random.default_rng(7 + n * 1000 + m * 10 + dim + 100 * p)
    a, ta = series(rng, n, dim, np.float32)
    b, tb = series(rng, m, dim, np.float32)
    nu, lam = 0.25, 1.0
    got = tw.twed_f32(a, ta, b, tb, nu, lam, p)
    want = oracle.twed(a.astype(np.float64), ta.astype(np.float64), b.astype(np.float64),
                       tb.astype(np.float64), nu, lam, p)
    assert rel_err(got, want) <= 1e-5, (got, want)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rows_per_lane_schedules_agree(tw, dtype):
    # every strip height must give the same value (bit-identical in FP64)
    import torch
    rng = np.random.default_rng(3)
    a, ta = series(rng, 2100, 3)
    b, tb = series(rng, 700, 3)
    td = torch.float64 if dtype == "f64" else torch.float32
    dev = lambda x: torch.as_tensor(x).to(td).cuda()
    vals = []
    for R in (1, 2, 4, 8):
        out = tw.twed_dev(dev(a), dev(ta), dev(b), dev(tb), 0.5, 1.0, 2,
                          opts=tw.make_opts(rows_per_lane=R))
        torch.cuda.synchronize()
        vals.append(out.item())
    if dtype == "f64":
        assert len(set(vals)) == 1, vals
        assert vals[0] == oracle.twed(a, ta, b, tb, 0.5, 1.0, 2)
    else:
        assert max(vals) - min(vals) <= 1e-6 * max(vals), vals


def test_device_entry_point_on_torch_stream(tw):
    import torch
    rng = np.random.default_rng(5)
    a, ta = series(rng, 640, 2)
    b, tb = series(rng, 555, 2)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        A, TA, B, TB = (torch.as_tensor(x).cuda() for x in (a, ta, b, tb))
        out = tw.twed_dev(A, TA, B, TB, 1.0, 0.5, 2, stream=s)
    s.synchronize()
    assert out.item() == oracle.twed(a, ta, b, tb, 1.0, 0.5, 2)
    tw.default_handle().sync_status(s)


def test_w2_shape_f64_long_pair(tw):
    # the 3-D workload with exponential time gaps at n = m = 20000 (the full
    # 1e5 size is checked against the oracle in test_gpu_full.py)
    a, ta, b, tb = W.pair_w2(20000)
    got = tw.twed_f64(a, ta, b, tb, 0.001, 1.0, 2)
    want = oracle.twed_rolling(a, ta, b, tb, 0.001, 1.0, 2)
    assert got == want


def test_identity_and_symmetry_on_gpu(tw):
    rng = np.random.default_rng(9)
    a, ta = series(rng, 700, 4)
    b, tb = series(rng, 333, 4)
    assert tw.twed_f64(a, ta, a, ta, 1.0, 1.0, 2) == 0.0
    assert tw.twed_f64(a, ta, b, tb, 1.0, 1.0, 2) == tw.twed_f64(b, tb, a, ta, 1.0, 1.0, 2)


def test_wait_timeout_is_reported_and_context_survives(tw):
    # fault injection on the host side: strip 0 never publishes its progress,
    # so strip 1's bounded wait expires and the call reports TIMEOUT
    rng = np.random.default_rng(11)
    a, ta = series(rng, 3000, 1, np.float32)
    b, tb = series(rng, 500, 1, np.float32)
    opts = tw.make_opts(rows_per_lane=1, timeout_s=0.2, stall_strip=0)
    with pytest.raises(tw.TwedError) as ei:
        tw.twed_f32(a, ta, b, tb, 1.0, 1.0, 2, opts=opts)
    assert ei.value.status == tw.TWED_ERR_TIMEOUT
    got = tw.twed_f32(a, ta, b, tb, 1.0, 1.0, 2)  # the context is still usable
    want = oracle.twed(a.astype(np.float64), ta.astype(np.float64), b.astype(np.float64),
                       tb.astype(np.float64), 1.0, 1.0, 2)
    assert rel_err(got, want) <= 1e-5


@pytest.mark.parametrize("bad", ["len0", "dim0", "p0", "nu", "lam", "nan_nu", "nan_input"])
def test_invalid_arguments_rejected(tw, bad):
    a, t = np.zeros((4, 2)), np.arange(4.0)
    args = dict(a=a, ta=t, b=a, tb=t, nu=1.0, lam=1.0, p=2)
    if bad == "len0":
        args.update(a=a[:0], ta=t[:0])
    elif bad == "dim0":
        args.update(a=np.zeros((4, 0)), b=np.zeros((4, 0)))
    elif bad == "p0":
        args.update(p=0)
    elif bad == "nu":
        args.update(nu=-1.0)
    elif bad == "lam":
        args.update(lam=-0.5)
    elif bad == "nan_nu":
        args.update(nu=float("nan"))
    elif bad == "nan_input":
        a2 = a.copy()
        a2[1, 1] = np.inf
        args.update(a=a2)
    with pytest.raises(tw.TwedError) as ei:
        tw.twed_f64(**args)
    assert ei.value.status == tw.TWED_ERR_INVALID_ARG


@pytest.mark.parametrize("n,m", [(1, 1), (33, 65), (257, 300), (1000, 17), (2100, 700)])
@pytest.mark.parametrize("dim,p", [(1, 2), (3, 2), (4, 1), (8, 2), (2, 2), (5, 2), (7, 1)])
def test_pair_f32_compensated(tw, n, m, dim, p):
    # compensated (TwoSum) FP32 running cost against the FP64 oracle on the
    # same FP32-rounded inputs
    rng = np.random.default_rng(17 + n * 1000 + m * 10 + dim + 100 * p)
    a, ta = series(rng, n, dim, np.float32)
    b, tb = series(rng, m, dim, np.float32)
    got = tw.twed_f32(a, ta, b, tb, 0.25, 1.0, p, opts=tw.make_opts(accum=tw.ACCUM_KAHAN))
    want = oracle.twed(a.astype(np.float64), ta.astype(np.float64), b.astype(np.float64),
                       tb.astype(np.float64), 0.25, 1.0, p)
    assert rel_err(got, want) <= 1e-5, (got, want)


def test_compensated_unsupported_layout_is_reported(tw):
    # dim 9 has no compiled point layout (dims 5-7 are zero-padded to 8): an
    # explicit request is refused
    rng = np.random.default_rng(1)
    a, ta = series(rng, 50, 9, np.float32)
    with pytest.raises(tw.TwedError) as ei:
        tw.twed_f32(a, ta, a, ta, 1.0, 1.0, 2, opts=tw.make_opts(accum=tw.ACCUM_KAHAN))
    assert ei.value.status == tw.TWED_ERR_UNSUPPORTED
