"""Pins of the oracle's low-precision copies (precision form of the re-rank).

The copies follow the definitions of the two formats, so they are pinned
against what those definitions fix: special values, ties to even, saturation,
the subnormal grids, and brute-force nearest representable values.
"""

import numpy as np
import pytest

import oracle


def _f32(bits):
    return float(np.array([bits], dtype=np.uint32).view(np.float32)[0])


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


# ---------------------------------------------------------------- bfloat16
@pytest.mark.parametrize("x, bits", [
    (1.0, 0x3F80),
    (-2.0, 0xC000),
    (0.0, 0x0000),
    (-0.0, 0x8000),
    (1.0 + 2.0 ** -8, 0x3F80),           # halfway between 1 and 1 + 2^-7: even (1)
    (1.0 + 3 * 2.0 ** -8, 0x3F82),       # halfway between 1 + 2^-7 and 1 + 2^-6: even
    (1.0 + 2.0 ** -8 + 2.0 ** -20, 0x3F81),   # just above halfway: up
    (2.0 ** -133, 0x0001),               # smallest subnormal bfloat16
    (3 * 2.0 ** -134, 0x0002),           # halfway between 1 and 2 subnormal steps: even
    (2.0 ** -134, 0x0000),               # halfway between 0 and 1 step: even (0)
    (float(np.finfo(np.float32).max), 0x7F80),   # rounds past the largest finite: inf
    (float("inf"), 0x7F80),
])
def test_bf16_definition_values(x, bits):
    assert int(oracle.bf16_bits([x])[0]) == bits


def test_bf16_is_nearest_with_ties_to_even():
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 30, 2000),
                        rng.uniform(-1e-39, 1e-39, 300)]).astype(np.float32)
    b = oracle.bf16_bits(x)
    for xi, bi in zip(x, b):
        v = oracle.bf16_value([bi])[0]
        # neighbours one code away on either side (same sign half-line)
        for nb in (int(bi) - 1, int(bi) + 1):
            if (nb & 0x7FFF) > 0x7F7F or nb < 0 or (nb ^ int(bi)) & 0x8000:
                continue
            w = oracle.bf16_value([nb])[0]
            dv, dw = abs(float(xi) - v), abs(float(xi) - w)
            assert dv < dw or (dv == dw and (int(bi) & 1) == 0), (xi, hex(bi), hex(nb))


def test_bf16_relative_error_half_ulp():
    rng = np.random.default_rng(12)
    x = (rng.standard_normal(5000) * 1e3).astype(np.float32)
    v = oracle.bf16_value(oracle.bf16_bits(x))
    assert np.all(np.abs(v - x.astype(np.float64)) <= 2.0 ** -8 * np.abs(x))   # half of 2^-7 ulp


# ---------------------------------------------------------------- E4M3
@pytest.mark.parametrize("x, bits", [
    (1.0, 0x38),
    (-1.0, 0xB8),
    (448.0, 0x7E),                        # largest finite
    (464.0, 0x7E),                        # beyond: saturates
    (1e9, 0x7E),
    (-1e9, 0xFE),
    (2.0 ** -9, 0x01),                    # smallest subnormal
    (2.0 ** -10, 0x00),                   # halfway between 0 and 2^-9: even (0)
    (3 * 2.0 ** -10, 0x02),               # halfway between 1 and 2 steps: even
    (7 * 2.0 ** -9, 0x07),                # largest subnormal
    (2.0 ** -6, 0x08),                    # smallest normal
    (1.0625, 0x38),                       # halfway between 1 and 1.125: even
    (1.1875, 0x3A),                       # halfway between 1.125 and 1.25: even
    (240.0, 0x77),                        # 1.875 * 2^7
    (0.0, 0x00),
])
def test_e4m3_definition_values(x, bits):
    assert int(oracle.e4m3_bits([x])[0]) == bits


def test_e4m3_value_table():
    vals = oracle.e4m3_value(np.arange(256, dtype=np.uint8))
    finite = [c for c in range(256) if (c & 0x7F) != 0x7F]
    pos = sorted(vals[c] for c in finite if c < 128)
    assert pos[0] == 0.0 and pos[1] == 2.0 ** -9 and pos[-1] == 448.0
    assert len(set(pos)) == 127                      # 0 plus 126 positive finite values
    # every finite code round-trips
    for c in finite:
        assert int(oracle.e4m3_bits([vals[c]])[0]) == c


def test_e4m3_is_nearest_with_ties_to_even():
    grid = np.array(sorted(set(oracle.e4m3_value(np.arange(0x7F, dtype=np.uint8)))), dtype=np.float64)
    rng = np.random.default_rng(13)
    x = np.concatenate([rng.uniform(0, 448, 1500), rng.uniform(0, 2.0 ** -5, 500),
                        (grid[:-1] + grid[1:]) / 2]).astype(np.float32)
    b = oracle.e4m3_bits(x)
    for xi, bi in zip(x.astype(np.float64), b):
        v = oracle.e4m3_value([bi])[0]
        dist = np.abs(grid - xi)
        best = dist.min()
        assert abs(v - xi) == best, (xi, v)
        if np.sum(dist == best) > 1:                 # a tie: the even code wins
            assert (int(bi) & 1) == 0


# ---------------------------------------------------------------- copies
@pytest.mark.parametrize("prec", [1, 2])
def test_copy_error_and_norm(prec):
    rng = np.random.default_rng(14)
    x = (rng.standard_normal((50, 40)) * rng.uniform(1e-3, 1e3, (50, 1))).astype(np.float32)
    rows, meta = oracle.prec_copy(x, prec)
    assert rows.shape == (50, 48)
    assert np.all(rows[:, 40:] == 0)
    for i in range(50):
        xi = x[i].astype(np.float64)
        s = meta[i, 0]
        if prec == 1:
            v = oracle.bf16_value(rows[i, :40])
            assert s == 1.0
        else:
            assert s == float(np.float32(np.abs(x[i]).max()) / np.float32(448.0))
            v = oracle.e4m3_value(rows[i, :40]) * s
        assert meta[i, 1] == pytest.approx(np.linalg.norm(xi - v), rel=1e-12)
        assert meta[i, 2] == pytest.approx(np.linalg.norm(xi), rel=1e-12)
        # per-component error bounds fixed by the formats
        if prec == 1:
            assert np.all(np.abs(xi - v) <= 2.0 ** -8 * np.abs(xi))
        else:
            y = np.abs(xi) / s
            bound = np.where(y >= 2.0 ** -6, 2.0 ** -4 * y, 2.0 ** -10) * s * (1 + 1e-6)
            assert np.all(np.abs(xi - v) <= bound)


def test_copy_fp8_uses_full_range_and_zero_vector():
    x = np.zeros((2, 16), dtype=np.float32)
    x[1, 3] = -5.0
    rows, meta = oracle.prec_copy(x, 2)
    assert meta[0, 0] == 1.0 and meta[0, 1] == 0.0 and np.all(rows[0] == 0)
    assert int(rows[1, 3]) == 0xFE                   # -448: the largest magnitude maps to the top code
    # -5 ~ -448 * fl(5 / 448): only the rounding of the FP32 scale remains
    assert meta[1, 1] <= 5.0 * 2.0 ** -23
