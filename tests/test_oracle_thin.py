"""Pins of the oracle's arc-length thinning of ordered pieces (the parallel
reading of the box means of Sec. 3.3.2): closed forms on equally spaced
samples, the centroid for a box longer than the piece, the identity for a box
shorter than every segment, gaps longer than a box, and the group mean."""
import numpy as np

from oracle import graph


def test_equally_spaced_line_groups_of_four():
    # samples every 0.25 h along x: boxes of 1 h hold 4 samples each
    P = np.column_stack([np.arange(13) * 0.25, np.zeros(13), np.zeros(13)])
    means, group = graph.thin_piece(P, False, 1.0)
    assert np.array_equal(group, np.arange(13) // 4)
    assert np.allclose(means[:3, 0], [0.375, 1.375, 2.375]) and means[3, 0] == 3.0
    assert np.all(means[:, 1:] == 0)


def test_box_longer_than_piece_gives_centroid():
    rng = np.random.default_rng(1)
    P = np.cumsum(rng.uniform(-0.3, 0.3, (20, 3)), axis=0)
    means, group = graph.thin_piece(P, True, 1e3)
    assert len(means) == 1 and np.all(group == 0)
    assert np.allclose(means[0], P.mean(axis=0), atol=1e-12)


def test_box_shorter_than_segments_keeps_samples():
    rng = np.random.default_rng(2)
    P = np.cumsum(rng.uniform(0.2, 0.5, (15, 3)), axis=0)
    means, group = graph.thin_piece(P, False, 0.1)
    assert np.array_equal(group, np.arange(15))
    assert np.array_equal(means, P)


def test_gap_longer_than_a_box_starts_one_group():
    P = np.array([[0, 0, 0], [0.2, 0, 0], [3.5, 0, 0], [3.6, 0, 0]], float)
    means, group = graph.thin_piece(P, False, 1.0)
    assert list(group) == [0, 0, 1, 1]
    assert np.allclose(means, [[0.1, 0, 0], [3.55, 0, 0]])


def test_single_sample_and_spacing():
    means, group = graph.thin_piece([[1.0, 2.0, 3.0]], False, 1.0)
    assert np.array_equal(means, [[1.0, 2.0, 3.0]]) and list(group) == [0]
    # a circle of radius 6 sampled densely: group spacing close to the box
    t = np.linspace(0, 2 * np.pi, 400, endpoint=False)
    P = np.column_stack([6 * np.cos(t), 6 * np.sin(t), np.zeros_like(t)])
    means, group = graph.thin_piece(P, True, 1.5)
    L = 2 * np.pi * 6 * (399 / 400)
    assert len(means) == int(L // 1.5) + 1
