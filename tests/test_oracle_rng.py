"""Pins for the oracle's Philox generator (Salmon et al. 2011).

The 4x64 instantiation is checked word for word against numpy's Philox
bit generator (the published Philox4x64-10); the 4x32 instantiation is
the same macro text with the 32-bit constants, and is checked for the
statistical properties the method relies on.
"""
import numpy as np
import pytest


def _numpy_block(ctr, key):
    """numpy's Philox increments its counter before each block."""
    g = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    return g.random_raw(4).astype(np.uint64)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_philox4x64_matches_numpy(orc, seed):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        ctr = rng.integers(0, 2 ** 63, size=4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 63, size=2, dtype=np.uint64)
        ctr[0] = ctr[0] & np.uint64(0x7FFFFFFFFFFFFFFF)  # no carry on the increment
        nxt = ctr.copy()
        nxt[0] += np.uint64(1)
        assert np.array_equal(orc.philox4x64(nxt, key), _numpy_block(ctr, key))


def test_philox4x64_zero_counter(orc):
    assert np.array_equal(orc.philox4x64([1, 0, 0, 0], [0, 0]), _numpy_block([0, 0, 0, 0], [0, 0]))


def _words(orc, n, key=(7, 9), word3=0):
    out = np.zeros((n, 4), np.uint32)
    for i in range(n):
        out[i] = orc.philox4x32([i, 0, 0, word3], key)
    return out.ravel()


def test_philox4x32_uniform_bytes(orc):
    w = _words(orc, 20000)
    # chi-square of the 256 byte values of every byte lane
    for shift in (0, 8, 16, 24):
        b = (w >> np.uint32(shift)) & np.uint32(0xFF)
        counts = np.bincount(b, minlength=256)
        exp = w.size / 256.0
        chi2 = ((counts - exp) ** 2 / exp).sum()
        # 255 dof: mean 255, sd ~22.6; 6 sd band
        assert 120 < chi2 < 390, chi2


def test_philox4x32_avalanche(orc):
    rng = np.random.default_rng(5)
    flips = []
    for _ in range(400):
        ctr = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
        bit = int(rng.integers(0, 128))
        c2 = ctr.copy()
        c2[bit // 32] ^= np.uint32(1 << (bit % 32))
        a = orc.philox4x32(ctr, key)
        b = orc.philox4x32(c2, key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    m = np.mean(flips)
    assert 62 < m < 66, m          # 128 output bits, half should flip


def test_philox4x32_key_sensitivity(orc):
    a = orc.philox4x32([1, 2, 3, 4], [10, 20])
    b = orc.philox4x32([1, 2, 3, 4], [11, 20])
    c = orc.philox4x32([1, 2, 3, 4], [10, 21])
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def test_philox4x32_uniform_mean_and_serial_correlation(orc):
    w = _words(orc, 25000, key=(123, 456), word3=(3 << 16) | 7)
    u = (w.astype(np.float64) + 0.5) / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 5 / np.sqrt(u.size)


def test_draw_layout(orc):
    """Draw j of a packet is word j&3 of the block with counter word 2 = j>>2;
    key = (seed_lo ^ job, seed_hi ^ iter), counter = (pkt_lo, pkt_hi, j>>2, stream)."""
    seed = 0x0123456789ABCDEF
    job, it, stream, pkt = 5, 9, (2 << 16) | 3, (7 << 32) | 11
    key = [(seed & 0xFFFFFFFF) ^ job, (seed >> 32) ^ it]
    for j in range(13):
        blk = orc.philox4x32([pkt & 0xFFFFFFFF, pkt >> 32, j >> 2, stream], key)
        assert orc.draw_u32(seed, job, it, stream, pkt, j) == int(blk[j & 3])
