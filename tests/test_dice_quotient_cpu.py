"""The library's computation of the binary64 Dice quotient
(``csrc/dice.cuh``, used by every scan kernel: integer long division whose
18-bit digits are estimated from a binary32 reciprocal and corrected by the
exact remainder) against the host's IEEE division, bit for bit.  Removing
either digit correction fails these cases.

The header is compiled for the host with g++ into a small shared library;
the expected values come from numpy's binary64 division, which is correctly
rounded to nearest-even.  Cases: every numerator below every denominator up
to 2,048; random pairs over the whole 32-bit range; numerators next to the
denominator and powers of two; the conventions for empty and equal masks.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2205_04550_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("dice")
    src = d / "dice_host.cpp"
    src.write_text(
        '#include "dice.cuh"\n'
        'extern "C" void quotients(const unsigned* num, const unsigned* den, long n,\n'
        '                          unsigned long long* out) {\n'
        '    for (long i = 0; i < n; ++i) out[i] = dbq::quotient_bits(num[i], den[i]);\n'
        '}\n'
        'extern "C" unsigned long long dice(unsigned i, unsigned a, unsigned b) {\n'
        '    return dbq::dice_bits(i, a, b);\n'
        '}\n')
    so = d / "libdice_host.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", HDR, str(src),
                    "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.quotients.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p]
    lib.dice.argtypes = [ctypes.c_uint, ctypes.c_uint, ctypes.c_uint]
    lib.dice.restype = ctypes.c_ulonglong
    return lib


def _check(lib, num, den):
    num = np.ascontiguousarray(num, dtype=np.uint32)
    den = np.ascontiguousarray(den, dtype=np.uint32)
    assert np.all(num > 0) and np.all(num < den)
    got = np.empty(num.size, dtype=np.uint64)
    lib.quotients(num.ctypes.data, den.ctypes.data, num.size, got.ctypes.data)
    want = (num.astype(np.float64) / den.astype(np.float64)).view(np.uint64)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, [(int(num[i]), int(den[i]), hex(int(got[i])), hex(int(want[i])))
                           for i in bad[:5]]


def test_all_pairs_below_2048(lib):
    den = np.repeat(np.arange(2, 2049, dtype=np.uint32), np.arange(1, 2048))
    num = np.concatenate([np.arange(1, d, dtype=np.uint32) for d in range(2, 2049)])
    _check(lib, num, den)


def test_random_pairs_over_32_bits(lib):
    rng = np.random.default_rng(2205)
    for bits in (12, 20, 24, 26, 28, 31, 32):
        den = rng.integers(2, 2 ** bits, size=200_000, dtype=np.uint64)
        num = (rng.random(den.size) * (den - 1)).astype(np.uint64) + 1
        num = np.minimum(num, den - 1)
        _check(lib, num, den)


def test_numerators_next_to_the_denominator_and_powers_of_two(lib):
    rng = np.random.default_rng(7)
    den = rng.integers(2 ** 20, 2 ** 32, size=50_000, dtype=np.uint64)
    for off in (1, 2, 3):
        ok = den > off
        _check(lib, den[ok] - off, den[ok])
    p2 = np.array([2 ** j for j in range(1, 32)], dtype=np.uint64)
    _check(lib, p2 - 1, p2)
    _check(lib, np.ones(p2.size, np.uint64), p2)
    _check(lib, p2[:-1], p2[1:] + 1)
    _check(lib, np.full(31, 1, np.uint64), np.array([2 ** 32 - 1] * 31, np.uint64))


def test_dice_conventions(lib):
    one = np.float64(1.0).view(np.uint64)
    assert lib.dice(0, 0, 0) == one            # both masks empty
    assert lib.dice(5, 5, 5) == one            # identical masks
    assert lib.dice(0, 3, 4) == 0              # disjoint
    want = (np.float64(2 * 3) / np.float64(7 + 11)).view(np.uint64)
    assert lib.dice(3, 7, 11) == want


def test_denominators_next_to_powers_of_two(lib):
    rng = np.random.default_rng(11)
    dens = []
    for j in range(2, 33):
        for off in (-3, -1, 1, 3):
            d = 2 ** j + off
            if 2 < d < 2 ** 32:
                dens.append(d)
    den = np.repeat(np.array(dens, dtype=np.uint64), 4000)
    num = (rng.random(den.size) * (den - 1)).astype(np.uint64) + 1
    num = np.minimum(num, den - 1)
    _check(lib, num, den)
    half = den // 2
    _check(lib, np.maximum(half, 1), den)
    _check(lib, np.minimum(half + 1, den - 1), den)
