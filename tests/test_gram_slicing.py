"""The two IEEE single-precision identities the Gram kernels' slicing rests
on, checked on the host in numpy float32 (round to nearest even, the mode of
the kernels' __fadd_rn / __fsub_rn):

1. For |r| < 2^(k-1) and C = 1.5 * 2^(k+23), (r + C) - C is r rounded to the
   nearest multiple of 2^k, ties to even: rint(r 2^-k) 2^k.
2. A float with at most 8 significant bits is exact in bfloat16, and its
   bfloat16 bits are the float's upper 16 bits.

With both, the fixed-grid slices y_s = q_s 2^(-8 s) of an x in (-1, 1) are
the same as with round-to-integer and a conversion, and each slice is exact
in bf16 with |q_1| <= 256 and |q_s| <= 128 for s >= 2 (the error-free split
of the Gram products, Alg. 8 with FP64-accurate accumulation)."""
import numpy as np

F32 = np.float32


def grid_round(r, k):
    c = F32(1.5) * F32(2.0) ** F32(k + 23)
    return (r + c) - c


def rint_round(r, k):
    s = F32(2.0) ** F32(-k)
    return np.rint(r * s) / s          # both scalings are exact powers of two


def bf16_rne_bits(x):
    """bfloat16 bits of float32 x, round to nearest even (finite x)."""
    u = x.view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def test_grid_rounding_equals_rint():
    rng = np.random.default_rng(7)
    for k in (-8, -16, -24, -32, -40):
        # residuals of every size below the grid's bound, plus exact ties
        mags = F32(2.0) ** rng.uniform(k - 30, k + 6, 200_000).astype(F32)
        r = (mags * rng.choice([-1, 1], mags.size)).astype(F32)
        ties = ((rng.integers(-2**10, 2**10, 20_000) + F32(0.5)) * F32(2.0) ** F32(k)).astype(F32)
        r = np.concatenate([r, ties, -ties, np.zeros(4, F32)])
        r = r[np.abs(r) < F32(2.0) ** F32(k + 6)]
        a = grid_round(r, k)
        b = rint_round(r, k)
        assert a.dtype == np.float32 and b.dtype == np.float32
        assert np.array_equal(a, b), k
        # and the residual is exact
        assert np.array_equal((r - a).astype(np.float64), r.astype(np.float64) - a.astype(np.float64))


def test_fixed_grid_slices_are_exact_bf16_upper_halves():
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, 100_000).astype(F32)
    x = np.concatenate([x, np.array([0.99999994, -0.99999994, 2.0**-126, -2.0**-40, 0.5], F32)])
    r = x.copy()
    total = np.zeros(x.size, np.float64)
    for s in range(1, 6):
        y = grid_round(r, -8 * s)
        q = y.astype(np.float64) * 2.0 ** (8 * s)
        assert np.all(q == np.rint(q))
        assert np.all(np.abs(q) <= (256 if s == 1 else 128))
        # exact in bf16: rounding to bf16 changes nothing, and the bits are the upper half
        upper = (y.view(np.uint32) >> 16).astype(np.uint16)
        assert np.array_equal(bf16_rne_bits(y), upper)
        back = (upper.astype(np.uint32) << 16).view(np.float32)
        assert np.array_equal(back, y)
        total += y.astype(np.float64)
        r = (r - y).astype(F32)
    # five slices reproduce x to within the last grid's half step
    assert np.max(np.abs(total - x.astype(np.float64))) <= 2.0 ** -41


def test_bf16_rounding_reference_on_known_values():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa (1.0) wins;
    # 1 + 3 * 2^-8 ties to 1 + 2^-6 (even); 1 + 2^-8 + 2^-20 rounds up
    v = np.array([1 + 2.0**-8, 1 + 3 * 2.0**-8, 1 + 2.0**-8 + 2.0**-20], F32)
    got = (bf16_rne_bits(v).astype(np.uint32) << 16).view(np.float32)
    assert list(got) == [F32(1.0), F32(1 + 2.0**-6), F32(1 + 2.0**-7)]
