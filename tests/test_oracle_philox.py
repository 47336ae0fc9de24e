"""Pins of the oracle's Philox4x32-10 generator and its uniform mapping."""
import os

import numpy as np
from scipy import stats

from oracle.philox import philox4x32_10, uniform23
from oracle import step as ostep
from oracle.plasma import Params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        words = [int(t, 16) for t in line.split()]
        rows.append((words[0:4], words[4:6], words[6:10]))
    return rows


def test_known_answer_vectors():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = philox4x32_10(np.array(ctr, dtype=np.uint32), key)
        assert [int(v) for v in got] == want


def test_vectorised_matches_scalar():
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x12345678, 0x9abcdef0)
    batch = philox4x32_10(ctr, key)
    for i in range(64):
        assert np.array_equal(batch[i], philox4x32_10(ctr[i], key))


def test_uniform23_exact_in_binary32():
    w = np.array([0, 1, 511, 512, 2 ** 31, 2 ** 32 - 1], dtype=np.uint32)
    u = uniform23(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u[0] == 0.5 * 2.0 ** -23 and u[-1] == 1.0 - 0.5 * 2.0 ** -23


def test_uniformity_chi_square():
    ctr = np.zeros((1 << 14, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(1 << 14)
    u = uniform23(philox4x32_10(ctr, (7, 0)).reshape(-1))
    counts = np.histogram(u, bins=64, range=(0, 1))[0]
    assert stats.chisquare(counts).pvalue > 1e-4


def test_decision_word_layout():
    p = Params(seed=0x0000000500000003)
    u = ostep.decision_uniforms(p, 9, 17, ostep.STREAM_EMIT_E, 10)
    for i in range(10):
        blk = philox4x32_10(np.array([9, 17, i >> 2, ostep.STREAM_EMIT_E << 24], dtype=np.uint32),
                            (3, 5))
        assert u[i] == uniform23(blk[i & 3])
