"""Pins of the E4M3 oracle (oracle/fp8.py) to things other than itself: hand
values of the format definition, brute force over all codes, torch's own
float8_e4m3fn conversion (a library routine), a brute-force loop for the
scale rule and a worked example."""
import math

import numpy as np
import pytest
import torch

import oracle


def test_decode_matches_hand_values_of_the_format():
    hand = {0x00: 0.0, 0x01: 2.0 ** -9, 0x07: 7 * 2.0 ** -9, 0x08: 2.0 ** -6,
            0x09: 1.125 * 2.0 ** -6, 0x38: 1.0, 0x3F: 1.875, 0x40: 2.0, 0x77: 240.0,
            0x78: 256.0, 0x7E: 448.0, 0xB8: -1.0, 0xFE: -448.0, 0x81: -(2.0 ** -9)}
    v = oracle.e4m3_decode(list(hand))
    assert np.array_equal(v, np.array(list(hand.values())))
    assert np.signbit(oracle.e4m3_decode([0x80]))[0]
    nan = np.isnan(oracle.e4m3_decode(np.arange(256)))
    assert list(np.flatnonzero(nan)) == [0x7F, 0xFF]
    pos = oracle.e4m3_decode(np.arange(0x7F))
    assert np.all(np.diff(pos) > 0)                # 127 finite values, in code order
    assert np.array_equal(oracle.e4m3_decode(np.arange(0x80, 0xFF)), -pos)


def test_encode_inverts_decode_on_every_finite_code():
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF)])
    assert np.array_equal(oracle.e4m3_encode(oracle.e4m3_decode(codes)), codes.astype(np.uint8))


def _nearest_brute(x):
    """Nearest finite E4M3 value by a loop over all codes, ties to the even
    code, magnitudes above 448 saturated, the sign kept."""
    a = min(abs(x), 448.0)
    best, bd = None, math.inf
    for c in range(0x7F):
        v = float(oracle.e4m3_decode([c])[0])
        d = abs(a - v)
        if d < bd or (d == bd and c % 2 == 0):
            best, bd = c, d
    return best | (0x80 if math.copysign(1.0, x) < 0 else 0)


def test_encode_is_the_nearest_value_with_ties_to_even():
    g = np.random.default_rng(3)
    xs = list(g.standard_normal(300) * np.exp2(g.uniform(-12, 10, 300)))
    # exact midpoints and edges
    xs += [1.0625, 1.1875, 2.0 ** -10, 3 * 2.0 ** -10, 2.0 ** -6 - 2.0 ** -10, 464.0,
           465.0, 1e6, -1e-5, -0.0, 0.0, 240.0 + 8.0, 448.0 - 16.0]
    got = oracle.e4m3_encode(np.array(xs))
    want = [_nearest_brute(float(x)) for x in xs]
    assert list(got) == want
    # the midpoints by hand: 1.0625 -> 1.0 (M = 0), 1.1875 -> 1.25 (M = 2),
    # 2^-10 -> 0, 3 * 2^-10 -> 2^-8 (M = 2), past 448 -> 448
    assert list(got[300:305]) == [0x38, 0x3A, 0x00, 0x02, 0x08]
    assert list(got[305:308]) == [0x7E, 0x7E, 0x7E]


def test_encode_agrees_with_torch_float8_conversion():
    g = torch.Generator().manual_seed(5)
    x = torch.randn(200000, generator=g) * torch.exp2(torch.empty(200000).uniform_(-16, 9,
                                                                               generator=g))
    x = x.clamp(-448, 448)  # torch maps larger magnitudes to NaN, not to 448
    want = x.to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(oracle.e4m3_encode(x.double().numpy()), want)


def _scale_brute(t):
    if t == 0:
        return 1.0
    for es in range(-149, 129):
        if t <= 448.0 * 2.0 ** es:
            return 2.0 ** es
    raise AssertionError


def test_row_scale_is_the_smallest_power_of_two_that_fits():
    ts = [0.0, 448.0, 896.0, 447.0, 449.0, 224.0, 224.0 * (1 + 2 ** -40), 1.0,
          448.0 * 2.0 ** -140, 448.0 * 2.0 ** -149, 2.0 ** -149, 2.0 ** -130, 1e-37,
          3.0e38, 448.0 * 2.0 ** 100 * (1 - 2 ** -50)]
    g = np.random.default_rng(9)
    ts += list(np.exp2(g.uniform(-140, 120, 200)))
    got = oracle.row_scale(np.array(ts))
    assert list(got) == [_scale_brute(t) for t in ts]
    for t, s in zip(ts, got):
        if t >= 448.0 * 2.0 ** -148:
            assert 224.0 < t / s <= 448.0


def test_quantize_worked_example():
    # nine matrices (two groups of eight and one), two rows, two columns
    A = np.zeros((9, 2, 2))
    A[0] = [[448.0, -1.0], [0.0, 0.0]]          # group 0, row 0: t = 448 -> s = 1
    A[3] = [[3.0, 0.5], [0.0, 0.0]]             # row 1 of group 0 stays zero: s = 1
    A[8] = [[1000.0, 1.0], [0.001, -0.0005]]    # group 1: t = 1000 -> s = 4; t = 0.001 -> 2^-18
    codes, scales = oracle.quantize_e4m3(list(A))
    assert np.array_equal(scales, [[1.0, 1.0], [4.0, 2.0 ** -18]])
    assert list(codes[0, 0]) == [0x7E, 0xB8]    # 448, -1
    assert list(codes[3, 0]) == [0x44, 0x30]    # 3 = 1.5 * 2^1 (E = 8, M = 4), 0.5
    # 1000 / 4 = 250 -> 256 (between 240 and 256, nearer 256); 1 / 4 = 0.25
    assert list(codes[8, 0]) == [0x78, 0x28]
    # 0.001 * 2^18 = 262.144 -> 256; -0.0005 * 2^18 = -131.072 -> -128
    assert list(codes[8, 1]) == [0x78, 0xF0]
    back = oracle.dequantize_e4m3(codes, scales)
    assert back[8, 0, 0] == 1024.0 and back[8, 1, 1] == -128.0 * 2.0 ** -18
