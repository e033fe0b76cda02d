"""Pins of the oracle's bfloat16 rounding (`oracle.mlp_oracle.bf16`), the comparator of every
tensor-core inference check.

bfloat16 keeps float32's sign and 8-bit exponent and 7 stored fraction bits (8 significant bits).
Round-to-nearest-even then fixes every result below by hand: values halfway between two
neighbours go to the one whose last stored bit is 0; the largest finite value is 255 * 2^120;
values at or above the midpoint 255.5 * 2^120 overflow to infinity; below 2^-126 the spacing is
the subnormal quantum 2^-133; zeros keep their sign; NaN stays NaN.  On float32 inputs (where no
earlier rounding intervenes) the result must also equal PyTorch's float32 -> bfloat16 conversion.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

MAXF = 255.0 * 2.0 ** 120          # largest finite bfloat16
SUB = 2.0 ** -133                  # bfloat16 subnormal quantum

# (input, expected) pairs fixed by round-to-nearest-even
CASES = [
    (1.0, 1.0),
    (1.0 + 2.0 ** -8, 1.0),                                  # tie, lower neighbour even
    (1.0 + 3.0 * 2.0 ** -8, 1.0 + 2.0 ** -6),                # tie, upper neighbour even
    (1.0 + 2.0 ** -8 + 2.0 ** -30, 1.0 + 2.0 ** -7),         # just above a tie
    (1.0 + 2.0 ** -8 - 2.0 ** -30, 1.0),                     # just below a tie
    (1.0 + 2.0 ** -8 + 2.0 ** -40, 1.0 + 2.0 ** -7),         # above the tie by less than a float32 ulp
    (-(1.0 + 3.0 * 2.0 ** -8), -(1.0 + 2.0 ** -6)),          # sign symmetric
    (3.0, 3.0),
    (1.0 / 3.0, 0.333984375),                                # 0x3EAB: 171 * 2^-9
    (MAXF, MAXF),
    (254.5 * 2.0 ** 120, 254.0 * 2.0 ** 120),                # tie below the maximum, even = 254
    (255.5 * 2.0 ** 120 - 2.0 ** 100, MAXF),                 # just below the overflow midpoint
    (255.5 * 2.0 ** 120, np.inf),                            # the midpoint rounds to even = 2^128
    (1e39, np.inf),
    (-1e39, -np.inf),
    (2.0 ** -126, 2.0 ** -126),                              # smallest normal
    (SUB, SUB),                                              # smallest subnormal
    (1.5 * SUB, 2.0 * SUB),                                  # subnormal tie to even
    (2.5 * SUB, 2.0 * SUB),
    (0.5 * SUB, 0.0),                                        # tie with zero: zero is even
    (0.75 * SUB, SUB),
    (2.0 ** -140, 0.0),
    (np.inf, np.inf),
    (-np.inf, -np.inf),
]


def check_bf16_pins(fn):
    """Raises AssertionError if `fn` breaks any of the hand-fixed round-to-nearest-even pins."""
    x = np.array([c[0] for c in CASES])
    want = np.array([c[1] for c in CASES])
    got = np.asarray(fn(x), dtype=np.float64)
    for xi, gi, wi in zip(x, got, want):
        assert gi == wi, f"bf16({xi!r}) = {gi!r}, expected {wi!r}"
    z = np.asarray(fn(np.array([0.0, -0.0])), dtype=np.float64)
    assert z[0] == 0.0 and not np.signbit(z[0]) and z[1] == 0.0 and np.signbit(z[1]), "signed zeros"
    nan = np.asarray(fn(np.array([np.nan, -np.nan])), dtype=np.float64)
    assert np.isnan(nan).all(), "NaN must stay NaN"


def test_bf16_round_to_nearest_even_pins():
    check_bf16_pins(M.bf16)


def test_bf16_nan_payloads_stay_nan():
    # float32 NaNs whose payload sits only in the low 16 bits (an add-and-shift rounding turns
    # these into infinities or zero)
    bits = np.array([0x7F800001, 0x7FFFFFFF, 0xFF800001, 0x7FC00000], dtype=np.uint32)
    got = M.bf16(bits.view(np.float32).astype(np.float64))
    assert np.isnan(got).all()


def test_bf16_matches_torch_on_float32_inputs():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    # random float32 bit patterns over the whole finite range, plus exact ties in every binade
    bits = rng.integers(0, 0x7F7FFFFF, size=200000, dtype=np.uint64).astype(np.uint32)
    ties = (rng.integers(1, 254, size=4000, dtype=np.uint64).astype(np.uint32) << 23) | np.uint32(0x8000) \
        | (rng.integers(0, 128, size=4000, dtype=np.uint64).astype(np.uint32) << 16)
    f = np.concatenate([bits, ties]).view(np.float32)
    f = np.concatenate([f, -f])
    want = torch.from_numpy(f.copy()).to(torch.bfloat16).to(torch.float64).numpy()
    got = M.bf16(f.astype(np.float64))
    assert np.array_equal(got, want)


def test_planted_truncation_fails_the_pins():
    """A bfloat16 conversion that truncates (drops the low bits) instead of rounding, or rounds
    ties away from zero, must fail the pins above."""
    def truncate(x):
        f = np.asarray(x, dtype=np.float64).astype(np.float32)
        u = f.view(np.uint32) & np.uint32(0xFFFF0000)
        return u.view(np.float32).astype(np.float64)

    def ties_away(x):
        a = np.asarray(x, dtype=np.float64)
        fin = np.isfinite(a)
        af = np.where(fin, a, 0.0)
        _, e = np.frexp(af)
        q = np.ldexp(1.0, np.maximum(e, -125) - 8)
        r = np.sign(af) * np.floor(np.abs(af) / q + 0.5) * q
        r = np.where(np.abs(r) >= 2.0 ** 128, np.copysign(np.inf, af), r)
        return np.where(fin, r, a)

    for planted in (truncate, ties_away):
        with pytest.raises(AssertionError):
            check_bf16_pins(planted)
