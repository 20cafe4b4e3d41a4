"""Pins of the oracle's random-number stream (Philox4x32-10, uniform map,
Box-Muller) against published vectors and mathematical identities."""
import json
import math
import os

import numpy as np
import pytest

from oracle import mc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hex(v):
    return [int(x, 16) for x in v]


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox_kat.json")) as f:
        kat = json.load(f)
    for v in kat["vectors"]:
        out = mc.philox4x32_10(_hex(v["counter"]), _hex(v["key"]))
        assert [int(x) for x in out] == _hex(v["out"])


def test_philox_stream_counter_layout():
    # call c of stream (seed, key) uses counter (c_lo, c_hi, key_lo, key_hi), key (seed_lo, seed_hi)
    seed, key = 0x0123456789ABCDEF, 0xFEDCBA9876543210
    calls = [0, 1, 2**32 - 1, 2**32, 2**40 + 7]
    for c in calls:
        got = mc.philox_stream(seed, key, c, 1)
        ref = mc.philox4x32_10([c & 0xFFFFFFFF, c >> 32, key & 0xFFFFFFFF, key >> 32],
                               [seed & 0xFFFFFFFF, seed >> 32])
        assert list(got) == list(ref)


def test_uniform_map_range_and_exactness():
    # u = (2 floor(x / 2^9) + 1) 2^-24: odd multiples of 2^-24 strictly inside (0, 1)
    assert mc.uniform(0) == 2.0 ** -24
    assert mc.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert mc.uniform(511) == 2.0 ** -24 and mc.uniform(512) == 3 * 2.0 ** -24
    rng = np.random.default_rng(0)
    for x in rng.integers(0, 2**32, size=1000):
        u = mc.uniform(int(x))
        k = u * 2**24
        assert k == int(k) and int(k) % 2 == 1 and 0 < u < 1


def test_box_muller_identities():
    seed, key = 7, 11
    words = mc.philox_stream(seed, key, 0, 64).reshape(-1, 4)
    z = mc.normals(seed, key, 0, 256).reshape(-1, 4)
    for w, zz in zip(words, z):
        for p in range(2):
            u0, u1 = mc.uniform(int(w[2 * p])), mc.uniform(int(w[2 * p + 1]))
            r2 = zz[2 * p] ** 2 + zz[2 * p + 1] ** 2
            assert r2 == pytest.approx(-2.0 * math.log(u0), rel=1e-13)
            ang = math.atan2(zz[2 * p + 1], zz[2 * p]) % (2 * math.pi)
            assert ang == pytest.approx(2 * math.pi * u1, abs=1e-12)


def test_normals_offset_consistency():
    # the stream index m is global: a window equals the same slice of a longer run
    seed, key = 3, 5
    full = mc.normals(seed, key, 0, 1000)
    for b in [0, 1, 3, 4, 17, 501]:
        np.testing.assert_array_equal(mc.normals(seed, key, b, 100), full[b:b + 100])


def test_normal_moments():
    z = mc.normals(0, 1, 0, 2_000_000)
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    # fourth moment 3, variance of z^4 is 96
    assert abs(np.mean(z ** 4) - 3.0) < 5 * math.sqrt(96.0 / n)
    # the uniform map caps |z| at sqrt(-2 ln 2^-24) = sqrt(48 ln 2)
    assert np.abs(z).max() <= math.sqrt(48 * math.log(2)) + 1e-12


def test_streams_differ_by_key_and_seed():
    a = mc.normals(0, 0, 0, 64)
    assert not np.array_equal(a, mc.normals(0, 1, 0, 64))
    assert not np.array_equal(a, mc.normals(1, 0, 0, 64))


def test_cholesky():
    rng = np.random.default_rng(2)
    for d in [1, 2, 3, 7, 20]:
        A = rng.normal(size=(d, d))
        S = A @ A.T + d * np.eye(d)
        L = mc.cholesky(S)
        np.testing.assert_allclose(L @ L.T, S, rtol=0, atol=1e-12 * d)
        assert np.allclose(np.triu(L, 1), 0)
    with pytest.raises(np.linalg.LinAlgError):
        mc.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))
