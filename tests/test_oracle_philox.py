"""Pins of the oracle's Philox4x32-10 against cuRAND's host-side generator.

cuRAND's host Philox generator (a library routine, run on the CPU) emits, for
seed s, Philox4x32-10 blocks under key (s lo, s hi): block b of its output has
counter (b div 65536, 0, b mod 65536, 0), and an offset of 4*65536*c numbers
moves the first counter word to c (low 32 bits) and the second to c >> 32
(the offset is a 64-bit count, so c < 2^46).
Agreement over thousands of blocks pins the oracle's round function, key
schedule and counter words 0, 1 and 2.
"""
import ctypes

import numpy as np
import pytest

import oracle as O

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def _generate(lib, seed, n, offset=0):
    g = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        if offset:
            assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out


@pytest.mark.parametrize("seed", [0, 1, 3, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host(seed):
    lib = _curand()
    nblk = 65536 * 3
    out = _generate(lib, seed, 4 * nblk).reshape(-1, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    rng = np.random.default_rng(seed & 0xFFFF)
    picks = np.concatenate([np.arange(8), rng.integers(0, nblk, 600), [nblk - 1, 65535, 65536]])
    for b in picks:
        ctr = [int(b) // 65536, 0, int(b) % 65536, 0]
        assert np.array_equal(O.philox(ctr, key), out[b]), (seed, b)


@pytest.mark.parametrize("c0,c1", [(3, 1), (7, 2), (0xFFFFFFFF, 0x3FFF), (12345, 777)])
def test_philox_second_counter_word(c0, c1):
    lib = _curand()
    seed = 0xDEADBEEF12345678
    out = _generate(lib, seed, 8, offset=4 * 65536 * ((c1 << 32) + c0))
    key = [seed & 0xFFFFFFFF, seed >> 32]
    assert np.array_equal(O.philox([c0, c1, 0, 0], key), out[:4])


def test_philox_is_keyed():
    # different keys or counters give different blocks (no accidental aliasing)
    a = O.philox([1, 2, 3, 4], [5, 6])
    assert not np.array_equal(a, O.philox([1, 2, 3, 5], [5, 6]))
    assert not np.array_equal(a, O.philox([1, 2, 3, 4], [5, 7]))
