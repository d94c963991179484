"""Seeded input generators: pinned to the generator's published test vectors
and to library routines (numpy log/exp), independent of the oracle."""
import numpy as np
import pytest

import synth


def test_philox_known_answers():
    # Known-answer vectors published with the Philox4x32-10 definition
    # (Salmon et al., SC'11; Random123 distribution).
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = synth.philox4x32_10(*ctr, *key)
        assert tuple(int(g) for g in got) == want


def test_uniform_ranges_and_exactness():
    idx = np.arange(200000, dtype=np.uint64)
    a = synth.uniform_f64(0, 0, idx)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 0.01 and abs(a.var() - 1.0 / 3.0) < 0.01
    # 53 random bits: every value is a multiple of 2^-52
    assert np.all(np.ldexp(a + 1.0, 52) == np.round(np.ldexp(a + 1.0, 52)))
    b = synth.uniform_f32(0, 0, idx)
    assert b.dtype == np.float32 and b.min() >= -1.0 and b.max() < 1.0
    assert np.all(np.ldexp(b.astype(np.float64) + 1.0, 23) % 1.0 == 0.0)
    # random access: element i does not depend on which other elements are drawn
    assert np.array_equal(synth.uniform_f64(0, 0, idx[1234:1240]), a[1234:1240])
    # streams and seeds differ
    assert not np.array_equal(synth.uniform_f64(0, 1, idx[:100]), a[:100])
    assert not np.array_equal(synth.uniform_f64(1, 0, idx[:100]), a[:100])


def test_ln_exp_against_numpy():
    x = np.concatenate([np.geomspace(1e-300, 1.0, 20001), np.linspace(0.01, 1.0, 20001)])
    rel = np.abs(synth.ln_f64(x) - np.log(x)) / np.maximum(np.abs(np.log(x)), 1e-300)
    assert rel.max() < 4e-15
    t = np.linspace(-4.0, 4.0, 40001)
    assert (np.abs(synth.exp_f64(t) - np.exp(t)) / np.exp(t)).max() < 1e-14


def test_gaussian_moments():
    g = synth.gaussian_f64(7, 3, np.arange(400000, dtype=np.uint64))
    assert abs(g.mean()) < 0.01
    assert abs(g.var() - 1.0) < 0.01
    assert abs(np.mean(g ** 4) - 3.0) < 0.05
    assert np.count_nonzero(g == 0.0) == 0


def test_lognormal_mix_range():
    v = synth.lognormal_mix_f64(0, 0, np.arange(100000, dtype=np.uint64))
    ratio = np.abs(v) / np.abs(synth.gaussian_f64(0, 0, np.arange(100000, dtype=np.uint64)))
    assert ratio.min() >= np.exp(-3.0) * (1 - 1e-12) and ratio.max() <= np.exp(3.0) * (1 + 1e-12)


def test_planted_structure():
    dims = [5, 6, 7]
    us = [synth.unit_gaussian(0, synth.stream_u(j), n) for j, n in enumerate(dims)]
    for u in us:
        assert abs(np.dot(u, u) - 1.0) < 1e-14
    A = synth.tensor("planted", 0, dims, us=us)
    R = 10.0 * np.einsum("i,j,k->ijk", *us)
    noise = (A - R) / 0.01
    assert abs(noise.std() - 1.0) < 0.2
