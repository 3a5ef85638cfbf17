"""Pins for the oracle's random draws (reading R1: Philox4x64-10, Salmon et al.
SC'11).  The reference is numpy's own Philox4x64-10 bit generator, an
implementation independent of ours."""
import numpy as np
import pytest
from scipy import stats


def _numpy_block(ctr, key):
    # numpy increments the 256-bit counter before producing a block, so the
    # block for counter c is the first output of a generator started at c - 1.
    c = [int(v) for v in ctr]
    borrow = 1
    for i in range(4):
        v = c[i] - borrow
        borrow = 1 if v < 0 else 0
        c[i] = v % (1 << 64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(c, dtype=np.uint64))
    return bg.random_raw(4)


def test_philox_matches_numpy_bit_for_bit(oracle_mod):
    rng = np.random.default_rng(123)
    cases = [((0, 0, 0, 0), (0, 0)), ((1, 0, 0, 0), (1, 0)),
             ((2**64 - 1, 2**64 - 1, 5, 0), (2**64 - 1, 2**64 - 1))]
    for _ in range(200):
        cases.append((tuple(int(v) for v in rng.integers(0, 2**64, 4, dtype=np.uint64)),
                      tuple(int(v) for v in rng.integers(0, 2**64, 2, dtype=np.uint64))))
    for ctr, key in cases:
        ours = oracle_mod.philox4x64_10(ctr, key)
        assert np.array_equal(ours, _numpy_block(ctr, key)), (ctr, key)


def test_uniform_is_word0_top53_bits(oracle_mod):
    for seed, stream, m in [(1, 0, 0), (1, 0, 1), (7, 3, 1000), (2**63, 2**40, 2**33)]:
        w0 = int(_numpy_block((m, 0, 0, 0), (seed, stream))[0])
        assert oracle_mod.uniform(seed, stream, m) == (w0 >> 11) * 2.0**-53


def test_uniform_draws_are_uniform(oracle_mod):
    u = np.array([oracle_mod.uniform(1, 0, m) for m in range(200_000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    # Different streams and seeds give unrelated sequences.
    v = np.array([oracle_mod.uniform(1, 1, m) for m in range(20_000)])
    w = np.array([oracle_mod.uniform(2, 0, m) for m in range(20_000)])
    assert abs(np.corrcoef(u[:20_000], v)[0, 1]) < 0.05
    assert abs(np.corrcoef(u[:20_000], w)[0, 1]) < 0.05
