"""Pins for the oracle's Philox4x32-10 (Salmon et al., SC'11).

The counter-based generator draws the i.i.d. samples R_i that Eq. 4 averages
over (Sec. 3.1).  The oracle's rounds are checked against an independent
implementation (Triton's CPU interpreter) and for the properties a keyed
bijection of the counter space must have.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _random_inputs(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 2**32, size=(n, 6), dtype=np.uint64).astype(np.uint32)
    a[0] = 0                      # all-zero counter and key
    a[1] = 0xFFFFFFFF             # all-ones counter and key
    a[2, 4:] = 0
    return a


def test_philox_matches_triton_interpreter(tmp_path):
    pytest.importorskip("triton")
    a = _random_inputs(256, 7)
    fin, fout = tmp_path / "in.npy", tmp_path / "out.npy"
    np.save(fin, a)
    env = dict(os.environ, TRITON_INTERPRET="1")
    subprocess.run([sys.executable, os.path.join(HERE, "_philox_triton.py"), str(fin), str(fout)],
                   check=True, env=env, timeout=600)
    ref = np.load(fout).astype(np.uint32)
    got = oracle.philox(a[:, :4], a[:, 4:])
    assert np.array_equal(got, ref)


def test_philox_is_injective_in_the_counter():
    # For a fixed key the 10-round map is a bijection of the 128-bit counter.
    n = 1 << 16
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n)
    ctr[:, 1] = 12345
    out = oracle.philox(ctr, np.array([3, 4], np.uint32))
    as_bytes = out.view(np.dtype((np.void, 16)))
    assert np.unique(as_bytes).size == n


def test_philox_output_bits_are_uniform():
    n = 1 << 15
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 1] = np.arange(n)
    out = oracle.philox(ctr, np.array([0, 0], np.uint32))
    bits = np.unpackbits(out.view(np.uint8)).reshape(n, 128)
    p = bits.mean(axis=0)
    # each of the 128 output bits is a fair coin: 6-sigma band
    assert np.all(np.abs(p - 0.5) < 6 * 0.5 / np.sqrt(n))


def test_philox_key_and_counter_words_all_matter():
    base = np.array([[1, 2, 3, 4]], np.uint32)
    k = np.array([5, 6], np.uint32)
    ref = oracle.philox(base, k)
    for w in range(4):
        c = base.copy()
        c[0, w] ^= 1
        assert not np.array_equal(oracle.philox(c, k), ref)
    for w in range(2):
        kk = k.copy()
        kk[w] ^= 1
        assert not np.array_equal(oracle.philox(base, kk), ref)
