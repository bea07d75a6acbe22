"""How well the tensor-core forms' terms represent an FP64 operand (CPU).

The GPU tolerance for the BF16 split and FP16 scaled forms rests on two
facts about the operand terms, restated here in numpy from their definition
(every element rounded once to FP32, then split in FP32 by round-to-nearest):
  BF16 split : a = b0 + b1 + b2 + r with |r| <= 2^-24 |a|
  FP16 scaled: a 2^e = h0 + h1 + r with |r| <= 2^-22 |a 2^e| + 2^-25,
               max |a 2^e| over the leaf in [2^14, 2^15)
(the FP16 term's absolute floor 2^-25 is half its smallest subnormal step).
Each product of terms is exact in FP32 (8 x 8 and 11 x 11 significant bits)."""
import numpy as np
import pytest


def _bf16_rn(x32: np.ndarray) -> np.ndarray:
    """Round FP32 to the nearest BF16 (ties to even), as FP32."""
    b = x32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _split_bf16(a: np.ndarray):
    x = a.astype(np.float32)
    b0 = _bf16_rn(x)
    r1 = x - b0
    b1 = _bf16_rn(r1)
    b2 = _bf16_rn(r1 - b1)
    return b0, b1, b2


def _leaf_shift(a: np.ndarray) -> int:
    m = float(np.max(np.abs(a)))
    if m == 0.0:
        return 0
    return int(np.clip(14 - np.floor(np.log2(m)), -120, 120))


def _split_fp16(a: np.ndarray):
    e = _leaf_shift(a)
    x = (a * 2.0 ** e).astype(np.float32)
    h0 = x.astype(np.float16).astype(np.float32)
    h1 = (x - h0).astype(np.float16).astype(np.float32)
    return e, x, h0, h1


def _leaves(seed):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 1.0, (64, 64))
    d = np.abs(np.subtract.outer(np.arange(64), np.arange(64)))
    yield u                                   # uniform
    yield u * np.exp(-0.3 * d)                # decay across the leaf (1e-8 range)
    yield u * np.exp(-0.6 * d) * 1e-9         # small leaf, wide range
    yield np.ldexp(u, rng.integers(-30, 30, (64, 64)))  # wild exponents
    yield np.where(rng.random((64, 64)) < 0.5, 0.0, u)  # half zeros


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bf16_three_terms_represent_the_operand_to_2_pow_minus_24(seed):
    for a in _leaves(seed):
        b0, b1, b2 = _split_bf16(a)
        for t in (b0, b1, b2):
            assert np.array_equal(t, _bf16_rn(t))  # each term is a BF16 value
        rep = b0.astype(np.float64) + b1 + b2
        assert np.all(np.abs(a - rep) <= 2.0 ** -24 * np.abs(a))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fp16_two_scaled_terms_represent_the_operand_to_2_pow_minus_22(seed):
    for a in _leaves(seed):
        e, x, h0, h1 = _split_fp16(a)
        m = np.max(np.abs(x))
        assert m == 0.0 or 2.0 ** 14 <= m < 2.0 ** 15
        assert np.all(np.isfinite(h0)) and np.all(np.abs(h0) <= 65504.0)
        scaled = a * 2.0 ** e
        rep = h0.astype(np.float64) + h1
        assert np.all(np.abs(scaled - rep) <= 2.0 ** -22 * np.abs(scaled) + 2.0 ** -25)


def test_term_products_are_exact_in_fp32():
    rng = np.random.default_rng(7)
    a, b = rng.uniform(-1, 1, 4096), rng.uniform(-1, 1, 4096)
    for ta, tb in zip(_split_bf16(a), _split_bf16(b)):
        assert np.array_equal((ta * tb).astype(np.float64), ta.astype(np.float64) * tb.astype(np.float64))
    _, _, h0, h1 = _split_fp16(a)
    _, _, g0, g1 = _split_fp16(b)
    for p, q in ((h0, g0), (h0, g1), (h1, g0)):
        assert np.array_equal((p * q).astype(np.float64), p.astype(np.float64) * q.astype(np.float64))
