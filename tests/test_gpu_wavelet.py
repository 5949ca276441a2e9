"""Wavelet compression of cell fields on the GPU (bcm_compress_field / bcm_decompress_field)
against the oracle (R21 in oracle/bcm_oracle.c): the stream is integer data decided by
FP64 arithmetic done the same way on both sides, so it must match word for word, and
the decoded field bit for bit (after rounding to the field's storage type); error
codes for a short buffer, a step too small for the field and foreign streams."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1808_04099_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1808_04099_gb300 import bcm  # noqa: E402

GRIDS = {
    "cavity_B4": lambda: W.cavity(2, 4),
    "sphere_B8": lambda: W.sphere_channel(4, 2, 2, 8, radius=0.3),
    "sphere_B16": lambda: W.sphere_channel(2, 1, 1, 16, length=(2.0, 1.0, 1.0), radius=0.2,
                                           center=(0.6, 0.5, 0.5)),
}


def stepped_grid(spec, prec):
    g = bcm.Grid(spec, prec)
    g.load_state(W.initial_state(spec, seed=61, noise=1e-2))
    g.step(2, rtol=1e-10)
    return g


@pytest.mark.parametrize("prec", [bcm.PREC_F64, bcm.PREC_F32_REFINE])
@pytest.mark.parametrize("name", sorted(GRIDS))
def test_stream_and_decoded_field_match_oracle(name, prec):
    spec = GRIDS[name]()
    g = stepped_grid(spec, prec)
    for fid in (bcm.U, bcm.W, bcm.P):
        f = g.numpy(fid)
        for rel in (1e-3, 1e-5):
            step = rel * np.abs(f).max()
            s = g.compress_field(fid, step).cpu().numpy().view(np.uint32)
            ref = O.wavelet_compress(f, spec.B, step)
            assert np.array_equal(s, ref), (fid, rel)
            g.decompress_field(fid, torch.from_numpy(s.view(np.int32)))
            got = g.numpy(fid)
            want = O.wavelet_decompress(ref)
            if g.field(fid).dtype == torch.float32:
                want = want.astype(np.float32).astype(np.float64)
            assert np.array_equal(got, want), (fid, rel)
            assert np.abs(got - f).max() <= (0.5 + 7.3125 * np.log2(spec.B)) * step * 1.0001
            # put the original values back for the next round
            dst = g.field(fid)
            dst.copy_(torch.from_numpy(f).to(dst.device, dst.dtype))


def test_errors():
    spec = GRIDS["sphere_B8"]()
    g = stepped_grid(spec, bcm.PREC_F64)
    L = bcm.lib()
    buf = torch.empty(64, dtype=torch.int32, device=g.device)
    n = C.c_size_t()
    rc = L.bcm_compress_field(g._h, bcm.U, 1e-3, C.c_void_p(buf.data_ptr()), 256, C.byref(n))
    assert rc == bcm.BCM_E_INVALID  # capacity below the stream
    big = torch.empty(L.bcm_compress_bound(g._h) // 4, dtype=torch.int32, device=g.device)
    rc = L.bcm_compress_field(g._h, bcm.U, 1e-12, C.c_void_p(big.data_ptr()),
                              big.numel() * 4, C.byref(n))
    assert rc == bcm.BCM_E_BOUNDS  # coefficients beyond 2^30 steps
    s = g.compress_field(bcm.U, 1e-3)
    bad = s.clone()
    bad[0] = 0
    with pytest.raises(bcm.BCMError) as ei:
        g.decompress_field(bcm.U, bad)
    assert ei.value.status == bcm.BCM_E_INVALID
    other = stepped_grid(GRIDS["cavity_B4"](), bcm.PREC_F64).compress_field(bcm.U, 1e-3)
    with pytest.raises(bcm.BCMError) as ei:
        g.decompress_field(bcm.U, other)
    assert ei.value.status == bcm.BCM_E_INVALID


def test_full_size_sphere_streams_match_oracle():
    """The 4.19M-cell sphere flow after two mixed steps: the streams of u and p at a
    step of 1e-4 of the field's largest value equal the oracle's word for word."""
    spec = W.config_sphere(2)
    g = bcm.Grid(spec, bcm.PREC_F32_REFINE)
    g.load_state(W.initial_state(spec))
    g.step(2, rtol=1e-8)
    for fid in (bcm.U, bcm.P):
        f = g.numpy(fid)
        step = 1e-4 * np.abs(f).max()
        s = g.compress_field(fid, step).cpu().numpy().view(np.uint32)
        assert np.array_equal(s, O.wavelet_compress(f, spec.B, step))


def rice_bits(zs, k):
    """LSB-first bits of the codes of values zs with Rice parameter k (the stream format
    of the compressor: u < 16 one-bits, a zero-bit, the k low bits; else 16 one-bits and
    the 32 bits of z)."""
    bits = []
    for z in zs:
        u = int(z) >> k
        if u < 16:
            bits += [1] * u + [0] + [(int(z) >> e) & 1 for e in range(k)]
        else:
            bits += [1] * 16 + [(int(z) >> e) & 1 for e in range(32)]
    return bits


def crafted_stream(B, records, step):
    """A stream of the compressor's layout from (k, bits, nbits) per cube."""
    sb = np.array([step], np.float64).view(np.uint32)
    head = [0x57434d42, 1, B, len(records), 0, 0, int(sb[0]), int(sb[1])]
    sizes, body = [], []
    for k, bits, nbits in records:
        w = np.zeros((len(bits) + 31) // 32, np.uint64)
        for i, b in enumerate(bits):
            w[i >> 5] |= np.uint64(b) << np.uint64(i & 31)
        sizes.append(1 + w.size)
        body += [k | (nbits << 5)] + [int(v) for v in w]
    return np.array(head + sizes + body, np.uint32)


def crafted_records(B, n_cubes, seed):
    """Records the encoder would not write but a decoder must read as the format says:
    a parameter of 1 with every value 0 (a code boundary every second bit, so a decode
    started at an odd bit never falls into step), values that mostly escape, the
    largest parameter, geometric values, and trailing bits past what B^3 codes can use
    (beyond 48 B^3 bits)."""
    rng = np.random.default_rng(seed)
    B3 = B ** 3
    recs = []
    for c in range(n_cubes):
        kind = (c + seed) % 5
        if kind == 0:
            k, zs = 1, np.zeros(B3, np.int64)
        elif kind == 1:
            k, zs = 0, rng.integers(0, 2 ** 32, B3)
        elif kind == 2:
            k, zs = 24, rng.integers(0, 2 ** 29, B3)
        else:
            k = int(rng.integers(0, 8))
            zs = np.minimum(rng.geometric(1.0 / (2 ** k + 1), B3) - 1, 2 ** 32 - 1)
        bits = rice_bits(zs, k)
        if kind == 4:
            bits += list(rng.integers(0, 2, 48 * B3 + 77))
        recs.append((k, bits, len(bits)))
    return recs


@pytest.mark.parametrize("name", ["cavity_B4", "sphere_B8", "sphere_B16"])
def test_crafted_records_decode_as_the_oracle(name):
    """Block-parallel decoding of records whose code boundaries are hard to find equals
    the oracle's sequential decoder bit for bit (4^3 cubes: one partial warp per
    block), and a record cut one bit short is malformed on both sides."""
    spec = GRIDS[name]()
    g = bcm.Grid(spec, bcm.PREC_F64)
    for seed in range(5):  # every kind of record in every cube
        recs = crafted_records(spec.B, spec.n_cubes, seed)
        s = crafted_stream(spec.B, recs, 0.37)
        want = O.wavelet_decompress(s)
        g.decompress_field(bcm.P, torch.from_numpy(s.view(np.int32)))
        assert np.array_equal(g.numpy(bcm.P), want), seed
    k1, bits1, nb1 = recs[1]  # seed 4: cube 1 holds the all-zero record, no spare bits
    short = crafted_stream(spec.B, recs[:1] + [(k1, bits1, nb1 - 1)] + recs[2:], 0.37)
    with pytest.raises(ValueError):
        O.wavelet_decompress(short)
    with pytest.raises(bcm.BCMError) as ei:
        g.decompress_field(bcm.P, torch.from_numpy(short.view(np.int32)))
    assert ei.value.status == bcm.BCM_E_INVALID
