"""Pins of the oracle's random-projection (count sketch) and Hamming-code
encodings against a published generator test vector, closed forms and
invariants."""
import numpy as np

import oracle

rng = np.random.default_rng(7)


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: the first outputs of the reference generator
    assert oracle.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64(0, 2) == 0x06C45D188009454F


def test_single_voxel_lands_in_its_bucket_with_its_sign():
    v, d = 5000, 256
    for x in (0, 1, 31, 32, 4999):
        m = np.zeros(v, np.uint8)
        m[x] = 1
        sk = oracle.sketch(m, d)
        h = oracle.splitmix64(0, x)
        j = (h >> 32) & (d - 1)
        assert np.count_nonzero(sk) == 1
        assert sk[j] == (-1 if (h >> 31) & 1 else 1)


def test_sketch_is_linear_over_disjoint_masks():
    v, d = 20000, 1024
    a = (rng.random(v) < 0.1).astype(np.uint8)
    b = ((rng.random(v) < 0.1) & (a == 0)).astype(np.uint8)
    np.testing.assert_array_equal(oracle.sketch(a | b, d), oracle.sketch(a, d) + oracle.sketch(b, d))
    assert oracle.sketch(np.zeros(v, np.uint8), d).sum() == 0


def test_sketch_distance_estimates_symmetric_difference():
    """E || S(a) - S(b) ||^2 = |a xor b| for a count sketch; averaged over
    pairs the ratio is close to 1."""
    v, d = 50000, 4096
    ratios = []
    for _ in range(30):
        a = (rng.random(v) < 0.05).astype(np.uint8)
        b = a.copy()
        flip = rng.random(v) < 0.02
        b[flip] ^= 1
        diff = oracle.sketch(a, d).astype(np.int64) - oracle.sketch(b, d)
        ratios.append(float((diff * diff).sum()) / float((a ^ b).sum()))
    assert abs(np.mean(ratios) - 1.0) < 0.05


def test_sign_codes_and_hamming():
    sk = np.array([3, -1, 0, 5] * 8 + [-2] * 32, dtype=np.int32)
    code = oracle.sign_code(sk)
    assert code.shape == (2,)
    assert code[0] == sum(1 << j for j in range(32) if j % 4 in (0, 3)) and code[1] == 0
    a = rng.integers(0, 2 ** 32, 128, dtype=np.uint64).astype(np.uint32)
    assert oracle.hamming(a, a) == 0
    assert oracle.hamming(a, ~a) == 128 * 32
    b = a.copy()
    b[5] ^= np.uint32(0b1011)
    assert oracle.hamming(a, b) == 3


def test_encode_values_integer_rows():
    vals = np.array([0, 1, -1, 255, 256, 257, -300, 448], dtype=np.int32)
    bf, q, s = oracle.encode_values(vals)
    assert [oracle.bf16_value(int(x)) for x in bf[:5]] == [0.0, 1.0, -1.0, 255.0, 256.0]
    assert oracle.bf16_value(int(bf[5])) == 256.0          # 257 -> nearest-even bfloat16
    assert s == np.float32(1.0)                              # max |v| = 448
    assert oracle.e4m3_value(int(q[7])) == 448.0 and oracle.e4m3_value(int(q[6])) == -288.0
