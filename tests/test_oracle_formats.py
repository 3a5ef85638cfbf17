"""Pins for the oracle's stored formats: BF16 and OCP FP8-E4M3 encode/decode
and the per-row FP8 quantiser, against torch's own CPU conversions."""
import numpy as np
import pytest
import torch


def _special_floats():
    rng = np.random.default_rng(5)
    parts = [
        rng.standard_normal(20000).astype(np.float32) * 100,
        rng.uniform(-1e-38, 1e-38, 2000).astype(np.float32),  # subnormal FP32
        np.array([0.0, -0.0, 1.0, -1.0, 3.0e38, -3.0e38, 1.17549435e-38], np.float32),
    ]
    # exact ties for BF16: low 16 bits == 0x8000, both parities of bit 16
    bits = rng.integers(0, 2**32, 4000, dtype=np.uint64).astype(np.uint32)
    bits = (bits & np.uint32(0xFFFF0000)) | np.uint32(0x8000)
    bits = bits[((bits >> 23) & 0xFF) != 0xFF]  # finite only
    parts.append(bits.view(np.float32))
    return np.concatenate(parts)


def test_bf16_encode_matches_torch(oracle_mod):
    x = _special_floats()
    ours = oracle_mod.quantize_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)


def test_bf16_decode_matches_torch(oracle_mod):
    codes = np.arange(0, 2**16, 37, dtype=np.uint16)
    codes = codes[((codes >> 7) & 0xFF) != 0xFF]
    ours = oracle_mod.decode_bf16(codes)
    ref = torch.from_numpy(codes.view(np.int16)).view(torch.bfloat16).double().numpy()
    assert np.array_equal(ours, ref)


def test_e4m3_decode_all_codes_match_torch(oracle_mod):
    codes = np.arange(256, dtype=np.uint8)
    ours = oracle_mod.decode_e4m3(codes)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).double().numpy()
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])
    assert np.nanmax(ours) == 448.0


def test_e4m3_encode_matches_torch_below_overflow(oracle_mod):
    rng = np.random.default_rng(9)
    # all representable values, all midpoints (ties), random values
    vals = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).double().numpy()
    vals = np.sort(vals[np.isfinite(vals)])
    mids = (vals[1:] + vals[:-1]) / 2
    x = np.concatenate([vals, mids, rng.uniform(-463, 463, 20000),
                        rng.uniform(-0.02, 0.02, 5000)]).astype(np.float32)
    x = x[np.abs(x) < 464]  # torch does not saturate; below 464 both round to finite
    ours = oracle_mod.encode_e4m3(x)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)


def test_e4m3_encode_saturates(oracle_mod):
    codes = oracle_mod.encode_e4m3(np.array([464.0, 1e30, -1e30, np.inf, 448.0]))
    assert codes.tolist() == [0x7E, 0x7E, 0xFE, 0x7E, 0x7E]


def test_fp8_row_quantiser(oracle_mod):
    rng = np.random.default_rng(11)
    x = (rng.standard_normal((300, 24)) * rng.uniform(0.01, 300, (300, 1))).astype(np.float32)
    x[7] = 0.0  # all-zero row: scale 1
    q, s = oracle_mod.quantize_fp8(x)
    xt = torch.from_numpy(x)
    s_ref = xt.abs().amax(1) / 448.0
    s_ref = torch.where(s_ref > 0, s_ref, torch.ones_like(s_ref))
    assert np.array_equal(s, s_ref.numpy())
    q_ref = (xt / s_ref[:, None]).clamp(-448, 448).to(torch.float8_e4m3fn).view(torch.uint8)
    assert np.array_equal(q, q_ref.numpy())
    # every row uses the top of the range, and decoding recovers x to e4m3 precision
    dq = oracle_mod.decode_e4m3(q) * s[:, None].astype(np.float64)
    assert np.all(np.abs(dq - x) <= 2.0**-4 * np.abs(x) + s[:, None] * 2.0**-9 + 1e-30)
