"""Host-side workload generators: the batched-box configuration's statistics
and structure (no GPU)."""
import numpy as np

from paper_2604_24627_gb300 import workloads


def test_config4_boxes():
    w = workloads.config4(nboxes=4096, seed=0)
    counts = np.bincount(w.box_of_cell)
    assert len(counts) == 4096 and counts.sum() == w.ncells
    assert counts.min() >= 16 and counts.max() <= 4096
    # log-normal with median 256 and sigma_ln = ln(16)/3, truncated to [16, 4096]
    assert abs(np.log(np.median(counts)) - np.log(256.0)) < 0.08
    assert abs(np.std(np.log(counts)) - np.log(16.0) / 3.0) < 0.05
    # per-box plasma: T uniform in [1, 5] keV, n_e log-uniform in [1e24, 1e26]
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    T_box = w.T_keV[starts]
    ne_box = w.n_ion[starts, 0]
    assert T_box.min() >= 1.0 and T_box.max() <= 5.0 and abs(T_box.mean() - 3.0) < 0.1
    lg = np.log10(ne_box)
    assert lg.min() >= 24.0 and lg.max() <= 26.0 and abs(lg.mean() - 25.0) < 0.05
    # every cell of a box carries the box's plasma
    assert np.array_equal(w.T_keV, T_box[w.box_of_cell])
    assert np.array_equal(w.n_ion[:, 0], ne_box[w.box_of_cell])
    assert w.caps[0] >= w.n_el and w.caps[1] >= w.n_ph


def test_config4_seeded():
    a = workloads.config4(nboxes=64, seed=7)
    b = workloads.config4(nboxes=64, seed=7)
    c = workloads.config4(nboxes=64, seed=8)
    assert np.array_equal(a.T_keV, b.T_keV) and np.array_equal(a.box_of_cell, b.box_of_cell)
    assert not np.array_equal(a.T_keV[:16], c.T_keV[:16])
