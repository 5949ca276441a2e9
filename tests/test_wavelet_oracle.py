"""Pins of the oracle's per-cube wavelet compression (R21 in oracle/bcm_oracle.c, the
paper's section "Data compression") to things other than itself: perfect
reconstruction of the transform; a constant cube keeps one coefficient (the constant)
and its stream is worked out by hand bit for bit; a profile linear along x leaves
exactly one finest-level detail per x line, at the end of the line, equal to the
slope (the symmetric extension); the quantized reconstruction error stays within the
bound (1/2 + 7.3125 L) step that the inverse lifting steps give (each 1-D inverse pass
maps coefficient errors E_s, E_d to at most E_s + 1.5 E_d); the stream header."""
import math

import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("B", [4, 8, 16])
def test_perfect_reconstruction(B):
    x = np.random.default_rng(B).standard_normal(B ** 3)
    y = O.dwt3(O.dwt3(x, B), B, inverse=True)
    assert np.abs(y - x).max() <= 4e-15 * np.abs(x).max()


@pytest.mark.parametrize("B", [4, 8, 16])
def test_constant_cube_keeps_one_coefficient(B):
    c = 0.7371
    y = O.dwt3(np.full(B ** 3, c), B)
    assert y[0] == c and np.count_nonzero(y[1:]) == 0


def _payload_bits(words, nbits):
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")
    return bits[:nbits]


@pytest.mark.parametrize("c,step", [(0.0125, 1e-3), (3.0, 1e-3), (-0.0031, 1e-3)])
def test_constant_cube_stream_by_hand(c, step):
    """One cube: q = rint(c / step) at index 0, zeros elsewhere; z = zigzag(q) (2q, or
    -2q - 1 below zero); k = floor(log2(z // B^3)) (0 when that is 0); the first value
    is written as u = z >> k one-bits, a zero-bit and the k low bits of z (or 16
    one-bits and the 32 bits of z when u >= 16), every other value as k + 1 zero-bits."""
    B = 8
    w = O.wavelet_compress(np.full(B ** 3, c), B, step)
    q = int(round(c / step))
    z = 2 * q if q >= 0 else -2 * q - 1
    mean = z // B ** 3
    k = 0 if mean == 0 else min(24, mean.bit_length() - 1)
    u = z >> k
    if u < 16:
        first = np.concatenate([np.ones(u, np.uint8), [0],
                                [(z >> e) & 1 for e in range(k)]]).astype(np.uint8)
    else:
        first = np.concatenate([np.ones(16, np.uint8),
                                [(z >> e) & 1 for e in range(32)]]).astype(np.uint8)
    want = np.concatenate([first, np.zeros((B ** 3 - 1) * (k + 1), np.uint8)])
    nbits = want.size
    assert w[8] == 1 + math.ceil(nbits / 32)            # record words
    assert w[9] == k | (nbits << 5)                      # k, nbits
    assert np.array_equal(_payload_bits(w[10:], nbits), want)
    f = O.wavelet_decompress(w)
    assert np.all(f == q * step)


@pytest.mark.parametrize("B", [4, 8, 16])
def test_linear_profile_leaves_one_detail_per_line(B):
    a, b = 0.375, -0.125  # dyadic: every value and every lifting step exact
    i = np.arange(B)
    x = np.broadcast_to(a + b * i, (B, B, B)).reshape(-1)  # varies along x only
    y = O.dwt3(x, B).reshape(B, B, B)  # [k, j, i]
    h = B // 2
    # finest-level x details of every line (all j, k below h: y and z low bands) ...
    assert np.all(y[:h, :h, h:B - 1] == 0.0)
    assert np.all(y[:h, :h, B - 1] == b)
    # ... and no finest-level detail along y or z
    assert np.count_nonzero(y[h:, :, :]) == 0 and np.count_nonzero(y[:, h:, :]) == 0


@pytest.mark.parametrize("B", [4, 8, 16])
def test_quantized_error_within_the_lifting_bound(B):
    L = int(round(math.log2(B)))
    rng = np.random.default_rng(10 + B)
    n_cubes = 6
    g = np.linspace(0, 1, B)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    fields = [rng.standard_normal(n_cubes * B ** 3),
              np.concatenate([np.sin(2 + 3 * X + c) * np.cos(Y - 2 * Z * c)
                              for c in range(n_cubes)]).reshape(-1)]
    for f in fields:
        for step in (1e-2, 1e-4):
            g2 = O.wavelet_decompress(O.wavelet_compress(f, B, step))
            assert np.abs(g2 - f).max() <= (0.5 + 7.3125 * L) * step


def test_stream_header_and_smooth_fields_compress():
    B, n_cubes, step = 16, 3, 1e-4
    g = np.linspace(0, 1, B)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    f = np.concatenate([np.sin(1 + X + 0.5 * c) * np.exp(-Y * Z) for c in range(n_cubes)])
    w = O.wavelet_compress(f.reshape(-1), B, step)
    assert w[0] == 0x57434D42 and w[1] == 1 and w[2] == B and w[3] == n_cubes
    assert w[6:8].view(np.float64)[0] == step
    assert 8 + n_cubes + int(w[8:8 + n_cubes].sum()) == w.size
    noise = np.random.default_rng(0).standard_normal(f.size) * np.abs(f).max()
    assert w.size * 2 < O.wavelet_compress(noise, B, step).size
