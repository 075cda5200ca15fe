"""The FP64 helper functions the kernels are built on, against correctly
rounded references and the IEEE-754 layout: the pivot reciprocal square root
(FP32 seed + one third-order Householder step) within 2 ulp and the
reciprocal (FP32 seed + one third-order Newton step) within 1 ulp of the
correctly rounded values over the whole double range and where the seed
truncates the most, the bit-layout splits
and float round trip exact, and the integer-unit max / min equal to fmax /
fmin on non-negative operands (a NaN operand ignored)."""
import numpy as np
import pytest

from tests.gpu_common import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    ensure_built()


def _positive(rng):
    """Log-uniform over the normal range, mantissas near every binade edge,
    both sides of the fast-path bounds (1e-30, 1e30), subnormals."""
    x = 10.0 ** rng.uniform(-307, 307, 200_000)
    m = 1.0 + rng.random(50_000)
    scaled = m * 2.0 ** rng.integers(-99, 99, 50_000).astype(float)
    edges = []
    for b in (1e-30, 1e30, 1.0, 2.0, 0.5, np.finfo(float).tiny):
        edges += [b, np.nextafter(b, 0.0), np.nextafter(b, np.inf)]
    edges += [np.finfo(float).max, np.nextafter(np.finfo(float).max, 0.0)]
    edges += [3.0, 7.0, 1.0 - 2.0 ** -53, 5e-324, 1e-310, 2.2e-308]
    return np.concatenate([x, m, scaled, np.array(edges)])


def _run(fn, x):
    torch = torch_cuda()
    from paper_2403_15913_gb300.solver import eval_fn
    y = eval_fn(fn, torch.from_numpy(np.ascontiguousarray(x)).cuda())
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _ulps(y, ref):
    return np.abs(y - ref) / np.spacing(np.abs(ref))


def test_pivot_rsqrt_within_two_ulp():
    from paper_2403_15913_gb300 import _native as nat
    x = _positive(np.random.default_rng(0))
    y = _run(nat.KKT_FN_RSQRT, x)
    ref = (1 / np.sqrt(x.astype(np.longdouble))).astype(np.float64)
    err = _ulps(y, ref)
    assert np.max(err) <= 2.0, (np.max(err), x[np.argmax(err)])
    special = np.array([0.0, np.inf, np.nan, -1.0, -0.0])
    ys = _run(nat.KKT_FN_RSQRT, special)
    assert ys[0] == np.inf and ys[1] == 0.0 and np.isnan(ys[2]) and np.isnan(ys[3]) and ys[4] == -np.inf


def test_reciprocal_within_one_ulp():
    from paper_2403_15913_gb300 import _native as nat
    x = _positive(np.random.default_rng(1))
    x = x[x > 1e-307]                       # 1/x of a subnormal overflows either way
    y = _run(nat.KKT_FN_RCP, x)
    ref = (1 / x.astype(np.longdouble)).astype(np.float64)
    err = _ulps(y, ref)
    assert np.max(err) <= 1.0, (np.max(err), x[np.argmax(err)])
    # the fast path is within one rounding of the IEEE quotient almost everywhere
    assert np.mean(y == 1.0 / x) > 0.99
    special = np.array([0.0, np.inf, np.nan, -2.0])
    ys = _run(nat.KKT_FN_RCP, special)
    assert ys[0] == np.inf and ys[1] == 0.0 and np.isnan(ys[2]) and ys[3] == -0.5


def _worst_truncation(rng):
    """Mantissas whose low 29 bits are all ones (the FP32 seeds truncate them
    away, moving the seed the most) and the largest mantissa, at scales across
    the fast-path range and next to its ends (1e-30, 1e30)."""
    hi = rng.integers(0, 1 << 23, 4000, dtype=np.int64)
    mant = (hi << 29) | ((1 << 29) - 1)
    mant = np.concatenate([mant, [(1 << 52) - 1, (1 << 29) - 1]])
    ex = np.concatenate([rng.integers(-99, 99, mant.size - 10), [-99, -99, -98, 98, 98, 99, 0, 0, -1, 1]])
    x = ((ex + 1023) << 52 | mant).view(np.float64)
    edge = np.array([1e-30, 1e30])
    ends = np.concatenate([np.nextafter(edge, np.inf), np.nextafter(edge, 0.0),
                           (edge.view(np.int64) | ((1 << 29) - 1)).view(np.float64)])
    return np.concatenate([x, ends])


def test_reciprocal_worst_truncation_and_range_ends():
    """The reciprocal within one ulp where its FP32 seed loses the most bits,
    and at the ends of the range its fast path covers."""
    from paper_2403_15913_gb300 import _native as nat
    x = _worst_truncation(np.random.default_rng(6))
    y = _run(nat.KKT_FN_RCP, x)
    ref = (1 / x.astype(np.longdouble)).astype(np.float64)
    err = _ulps(y, ref)
    assert np.max(err) <= 1.0, (np.max(err), x[np.argmax(err)])


def test_split_is_frexp_on_normal_numbers():
    from paper_2403_15913_gb300 import _native as nat
    x = _positive(np.random.default_rng(2))
    normal = (x >= np.finfo(float).tiny) & np.isfinite(x)
    m = _run(nat.KKT_FN_SPLIT_M, x)
    e = _run(nat.KKT_FN_SPLIT_E, x)
    rm, re = np.frexp(x[normal])
    assert np.array_equal(m[normal], rm) and np.array_equal(e[normal], re.astype(float))
    assert np.all(np.isnan(m[~normal]))
    bad = np.array([0.0, -1.0, np.inf, np.nan, 5e-324, -0.0])
    assert np.all(np.isnan(_run(nat.KKT_FN_SPLIT_M, bad)))


def test_float_round_trip_truncates_mantissa():
    from paper_2403_15913_gb300 import _native as nat
    x = _positive(np.random.default_rng(3))
    x = x[(x > 1e-30) & (x < 1e30)]
    y = _run(nat.KKT_FN_F32_ROUNDTRIP, x)
    ref = ((x.view(np.int64) >> 29) << 29).view(np.float64)
    assert np.array_equal(y, ref)
    assert np.all(np.abs(y - x) <= 2.0 ** -23 * x)


def _pairs(rng, signed):
    a = np.concatenate([10.0 ** rng.uniform(-300, 300, 50_000), [0.0, np.inf, 1.0, 1.0]])
    b = 10.0 ** rng.uniform(-300, 300, a.size)
    b[:7] = [np.nan, 0.0, np.inf, 1.0, 1e-320, 2.0, 0.5]
    b[-4:] = [np.nan, 1.0, 0.0, np.inf]
    if signed:
        flip = rng.random(a.size) < 0.5
        b = np.where(flip, -b, b)
        b[8] = -0.0
    return a, b


@pytest.mark.parametrize("which", ["max_abs", "max", "min"])
def test_integer_unit_max_min(which):
    from paper_2403_15913_gb300 import _native as nat
    rng = np.random.default_rng(4)
    a, b = _pairs(rng, signed=(which == "max_abs"))
    fn = {"max_abs": nat.KKT_FN_MAX_ABS, "max": nat.KKT_FN_MAX_NN, "min": nat.KKT_FN_MIN_NN}[which]
    y = _run(fn, np.stack([a, b]))
    ref = {"max_abs": np.fmax(a, np.abs(b)), "max": np.fmax(a, b), "min": np.fmin(a, b)}[which]
    assert np.array_equal(y, ref)
