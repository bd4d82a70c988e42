"""Pins of the oracle's prefilter encodings (bfloat16, FP8 E4M3 with a
per-row scale) and of its block-mean embedding, against library routines
(torch's dtype conversions) and closed forms."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def test_bf16_rounding_against_torch():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.random(5000, dtype=np.float32),
                           np.arange(513, dtype=np.float32) / np.float32(512),
                           # exact ties at bit 16: odd and even upper halves
                           np.array([0x3F808000, 0x3F818000, 0x3F7F8000, 0x3E808000],
                                    dtype=np.uint32).view(np.float32)])
    ref = torch.from_numpy(vals).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = np.array([oracle.bf16_bits(float(v)) for v in vals], dtype=np.uint16)
    np.testing.assert_array_equal(got, ref)
    for h in ref[:50]:
        assert oracle.bf16_value(int(h)) == float(torch.tensor(int(h), dtype=torch.int16)
                                                  .view(torch.bfloat16).float())


def test_e4m3_decode_all_codes_against_torch():
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    got = np.array([oracle.e4m3_value(int(c)) for c in codes])
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], ref[~nan])
    assert oracle.e4m3_value(0x7E) == 448.0 and oracle.e4m3_value(0x01) == 2.0 ** -9


def test_e4m3_rounding_against_torch_in_range():
    rng = np.random.default_rng(1)
    vals = np.concatenate([rng.uniform(-448, 448, 3000), rng.uniform(-1, 1, 3000),
                           rng.uniform(-2 ** -6, 2 ** -6, 1000),
                           # midpoints between neighbouring codes (ties to even)
                           (np.array([oracle.e4m3_value(c) for c in range(0, 0x7E)]) +
                            np.array([oracle.e4m3_value(c) for c in range(1, 0x7F)])) / 2])
    vals = vals.astype(np.float32)
    ref = torch.from_numpy(vals).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = np.array([oracle.e4m3_code(float(v)) for v in vals], dtype=np.uint8)
    np.testing.assert_array_equal(got, ref)
    assert oracle.e4m3_code(1e6) == 0x7E and oracle.e4m3_code(-1e6) == 0xFE   # saturation


def test_embed_closed_forms():
    nx = ny = nz = 32
    f = 8
    d = (nx // f) ** 3
    m = np.zeros(nx * ny * nz, np.uint8)
    b, q, s = oracle.embed(m, nx, ny, nz)
    assert not b.any() and not q.any() and s == np.float32(1.0)
    # a single voxel: one block at 1/512, scale (1/512)/448, code of 448
    x, y, z = 13, 30, 2
    m[x + nx * (y + ny * z)] = 1
    b, q, s = oracle.embed(m, nx, ny, nz)
    j = (x // f) + (nx // f) * ((y // f) + (ny // f) * (z // f))
    assert oracle.bf16_value(int(b[j])) == 1.0 / 512 and b.sum() == b[j]
    assert s == np.float32(np.float32(1.0 / 512) / np.float32(448.0))
    assert q[j] == 0x7E and q.sum() == 0x7E
    # a full block plus a half block: values 1 and 1/2
    m[:] = 0
    vol = m.reshape(nz, ny, nx)
    vol[0:8, 0:8, 0:8] = 1
    vol[8:16, 8:16, 8:12] = 1
    b, q, s = oracle.embed(vol.reshape(-1), nx, ny, nz)
    j1, j2 = 0, 1 + 4 * (1 + 4 * 1)
    assert oracle.bf16_value(int(b[j1])) == 1.0 and oracle.bf16_value(int(b[j2])) == 0.5
    assert s == np.float32(1.0 / 448.0)
    assert oracle.e4m3_value(int(q[j1])) == 448.0 and oracle.e4m3_value(int(q[j2])) == 224.0
    assert np.count_nonzero(b) == 2 and np.count_nonzero(q) == 2
    assert d == b.size


def test_embed_bf16_rounds_counts_above_256():
    nx = ny = nz = 8
    m = np.zeros(512, np.uint8)
    m[:257] = 1                                     # 257/512 is not a bfloat16
    b, _, _ = oracle.embed(m, nx, ny, nz)
    assert oracle.bf16_value(int(b[0])) == 256 / 512     # ties to even
    m[:259] = 1
    b, _, _ = oracle.embed(m, nx, ny, nz)
    assert oracle.bf16_value(int(b[0])) == 260 / 512
