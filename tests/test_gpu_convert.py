"""The kernels' FP32 <-> FP64 conversions (integer operations on the IEEE 754 fields) against
numpy's IEEE 754 conversions, bit for bit: FP64 -> FP32 rounds to nearest, ties to even, and
FP32 -> FP64 is exact.  Inputs cover every class: random bit patterns, values across the
binary32 range, exact ties of both parities and their neighbours, the edges of the normal
range, subnormals, zeros, infinities and NaN."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _doubles():
    rng = np.random.default_rng(11)
    parts = [rng.integers(0, 2 ** 64, 400000, dtype=np.uint64, endpoint=False)]
    vals = rng.standard_normal(400000) * np.exp(rng.uniform(-90, 90, 400000))
    parts.append(vals.view(np.uint64))
    f = rng.standard_normal(200000).astype(np.float32).astype(np.float64).view(np.uint64)
    tie = f | np.uint64(0x10000000)          # exactly half an ulp of binary32 above f
    parts += [tie, tie + np.uint64(1), tie - np.uint64(1), f]
    edges = [0x47EFFFFFE0000000, 0x47EFFFFFF0000000, 0x47EFFFFFEFFFFFFF, 0x47F0000000000000,  # max float, ties to inf
             0x3810000000000000, 0x380FFFFFFFFFFFFF, 0x3800000000000000, 0x36A0000000000000,  # min normal, subnormals
             0x0000000000000000, 0x8000000000000000, 0x7FF0000000000000, 0xFFF0000000000000,  # zeros, infinities
             0x7FF8000000000000, 0x0000000000000001, 0x3FF0000000000000, 0xBFF0000010000000]
    parts.append(np.array(edges, dtype=np.uint64))
    return np.concatenate(parts).view(np.float64)


def test_f64_to_f32_is_round_to_nearest_even():
    import torch
    from paper_1701_04900_gb300 import native
    d = _doubles()
    got = native.convert_check(torch.from_numpy(d).cuda()).cpu().numpy()
    with np.errstate(over="ignore", invalid="ignore"):
        ref = d.astype(np.float32)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint32), ref[~nan].view(np.uint32))


def test_f32_to_f64_is_exact():
    import torch
    from paper_1701_04900_gb300 import native
    rng = np.random.default_rng(12)
    bits = np.concatenate([rng.integers(0, 2 ** 32, 1000000, dtype=np.uint64).astype(np.uint32),
                           np.array([0, 0x80000000, 1, 0x807FFFFF, 0x00800000, 0x7F7FFFFF, 0x7F800000, 0xFF800000,
                                     0x7FC00000], dtype=np.uint32)])
    f = bits.view(np.float32)
    got = native.convert_check(torch.from_numpy(f).cuda()).cpu().numpy()
    ref = f.astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint64), ref[~nan].view(np.uint64))


def test_rejects_bad_arguments():
    from paper_1701_04900_gb300 import native
    L = native.lib()
    assert L.asyflexa_convert_check(2, None, None, 1, None) == native.EINVAL
    assert L.asyflexa_convert_check(0, None, None, 5, None) == native.EINVAL
    assert L.asyflexa_convert_check(0, None, None, -1, None) == native.EINVAL
    assert L.asyflexa_convert_check(0, None, None, 0, None) == native.OK


def _e4m3_value(code):
    """FP8-e4m3 (OCP 8-bit floating point, E4M3: bias 7, no infinities) from its definition:
    (-1)^s 2^(e-7) (1 + f/8) for e > 0, (-1)^s 2^-6 (f/8) for e = 0."""
    s, e, f = code >> 7, (code >> 3) & 0xF, code & 0x7
    mag = 2.0 ** (e - 7) * (1 + f / 8) if e else 2.0 ** -6 * (f / 8)
    return -mag if s else mag


def test_fp8_decode_every_code():
    """Every one of the 256 codes, in buffer order (code i at byte i of 16 units), decodes to
    its exact value; the two NaN codes give NaN."""
    import torch
    from paper_1701_04900_gb300 import native
    codes = np.arange(256, dtype=np.uint8)
    got = native.convert_check(torch.from_numpy(codes).cuda(), storage="fp8").cpu().numpy()
    ref = np.array([_e4m3_value(c) for c in range(256)], dtype=np.float64)
    nan = (codes & 0x7F) == 0x7F
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].astype(np.float64), ref[~nan])
    assert np.array_equal(np.signbit(got[~nan]), codes[~nan] >= 0x80)     # -0 keeps its sign
    assert ref[0x7E] == 448.0 and ref[0x01] == 2.0 ** -9 and ref[0x08] == 2.0 ** -6


def test_fp8_decode_random_layout():
    import torch
    from paper_1701_04900_gb300 import native
    rng = np.random.default_rng(13)
    codes = rng.integers(0, 256, 16 * 4099, dtype=np.uint8)
    got = native.convert_check(torch.from_numpy(codes).cuda(), storage="fp8").cpu().numpy()
    table = np.array([_e4m3_value(c) for c in range(256)], dtype=np.float64)
    table[0x7F] = table[0xFF] = np.nan
    ref = table[codes]
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].astype(np.float64), ref[~nan])


def test_bf16_decode_is_exact():
    import torch
    from paper_1701_04900_gb300 import native
    rng = np.random.default_rng(14)
    bits = rng.integers(0, 2 ** 16, 8 * 5003, dtype=np.uint32).astype(np.uint16)
    src = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()
    got = native.convert_check(src, storage="bf16").cpu().numpy()
    ref = (bits.astype(np.uint32) << 16).view(np.float32)     # bf16 is the top half of binary32
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint32), ref[~nan].view(np.uint32))


def test_decode_rejects_partial_units():
    import torch
    from paper_1701_04900_gb300 import native
    with pytest.raises(native.AsyflexaError):
        native.convert_check(torch.zeros(24, dtype=torch.uint8, device="cuda"), storage="fp8")
    with pytest.raises(native.AsyflexaError):
        native.convert_check(torch.zeros(12, dtype=torch.bfloat16, device="cuda"), storage="bf16")
