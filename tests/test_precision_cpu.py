"""The precision argument behind the tensor-core near field of FP32 products, checked on the CPU.

Every FP32 value x is split into hi = x rounded to TF32 (nearest, ties away from zero: the low 13
mantissa bits cleared) and lo = x - hi, which is exact in FP32. The tensor cores read each operand
as TF32, so lo enters with its own low 13 bits dropped. Three products, hi*hi + hi*lo + lo*hi,
then reproduce a*b to about 2^-22 relative: the dropped lo*lo term and the truncation of lo are
both of that order. The bar for a dot product is the one plain FP32 arithmetic meets, a few units
of 2^-24 times sum |a||b| over its length. Plain TF32 (hi*hi alone) misses it by orders of
magnitude, which is why the near field does not use it."""
import numpy as np

TF32_DROP = np.uint32(0x1FFF)  # the 13 low mantissa bits a TF32 value does not carry


def _tf32_round(x: np.ndarray) -> np.ndarray:
    """x rounded to TF32: to nearest, ties away from zero (finite inputs)."""
    b = x.astype(np.float32).view(np.uint32)
    r = (b + np.uint32(0x1000)) & ~TF32_DROP
    return r.view(np.float32)


def _tf32_truncate(x: np.ndarray) -> np.ndarray:
    """x as the tensor cores read a 32-bit operand in TF32 mode: the low 13 mantissa bits dropped."""
    return (x.astype(np.float32).view(np.uint32) & ~TF32_DROP).view(np.float32)


def _split_dot(a: np.ndarray, b: np.ndarray, three: bool) -> np.ndarray:
    """Dot products of the rows of a with the rows of b, from the TF32 split, summed exactly."""
    ah, bh = _tf32_round(a), _tf32_round(b)
    al, bl = _tf32_truncate(a - ah), _tf32_truncate(b - bh)
    f = lambda x: x.astype(np.float64)
    out = f(ah) @ f(bh).T
    if three:
        out += f(ah) @ f(bl).T + f(al) @ f(bh).T
    return out


def test_tf32_rounding_is_the_documented_one():
    x = np.array([1.0, 1.0 + 2.0 ** -10, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -12, -(1.0 + 2.0 ** -11)], np.float32)
    h = _tf32_round(x)
    # 10 explicit mantissa bits survive; a tie rounds away from zero
    assert list(h) == [1.0, 1.0 + 2.0 ** -10, 1.0 + 2.0 ** -10, 1.0 + 2.0 ** -10, -(1.0 + 2.0 ** -10)]
    lo = x - h
    assert np.array_equal(h.astype(np.float64) + lo.astype(np.float64), x.astype(np.float64))  # exact split


def test_three_tf32_products_reach_fp32_accuracy():
    rng = np.random.default_rng(7)
    K = 64  # a dense leaf's inner dimension
    for scale in (1.0, 1e-20, 3e15):
        a = (rng.standard_normal((64, K)) * scale).astype(np.float32)
        b = rng.uniform(-1.0, 1.0, (64, K)).astype(np.float32)
        exact = a.astype(np.float64) @ b.astype(np.float64).T
        mag = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64).T
        err3 = np.abs(_split_dot(a, b, True) - exact) / mag
        err1 = np.abs(_split_dot(a, b, False) - exact) / mag
        # three products: within a few units of 2^-22 of sum |a||b| (plain FP32 summation of K
        # terms is bounded by K 2^-24 = 2^-18 here, and usually sits near sqrt(K) 2^-24)
        assert err3.max() <= 4 * 2.0 ** -22, err3.max()
        # one TF32 product: about 2^-11, far outside any FP32-level bar
        assert err1.max() >= 2.0 ** -14, err1.max()
