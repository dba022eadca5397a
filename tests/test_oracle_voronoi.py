"""Pins of the oracle's periodic Voronoi labelling (Sec. 2.1) and twin split
against hand-derived partitions."""
import numpy as np

from oracle.voronoi import label_rve, voronoi_labels
from paper_2402_09996_gb300.inputs import RVEInputs


def test_two_seeds_split_the_cell_in_halves():
    lab = voronoi_labels((8, 8, 8), np.array([[0.25, 0.5, 0.5], [0.75, 0.5, 0.5]]))
    assert np.all(lab[:, :, :4] == 0) and np.all(lab[:, :, 4:] == 1)


def test_periodic_minimum_image():
    # voxel x = 15/16 is 0.1125 from a seed at 0.05 through the boundary
    lab = voronoi_labels((2, 2, 8), np.array([[0.05, 0.5, 0.5], [0.5, 0.5, 0.5]]))
    assert list(lab[0, 0]) == [0, 0, 1, 1, 1, 1, 0, 0]


def test_exact_tie_goes_to_lowest_index():
    # centres 0.125, 0.375, 0.625, 0.875: voxel 1 is exactly 0.125 from both seeds and
    # voxel 3 exactly 0.375 from both (through the periodic boundary for seed 0)
    lab = voronoi_labels((1, 1, 4), np.array([[0.25, 0.5, 0.5], [0.5, 0.5, 0.5]]))
    assert list(lab[0, 0]) == [0, 0, 1, 0]
    lab = voronoi_labels((1, 1, 4), np.array([[0.5, 0.5, 0.5], [0.25, 0.5, 0.5]]))
    assert list(lab[0, 0]) == [1, 0, 0, 0]


def test_sampled_labels_match_full_map():
    rng = np.random.default_rng(3)
    seeds = rng.uniform(size=(9, 3))
    full = voronoi_labels((6, 10, 12), seeds).reshape(-1)
    idx = rng.choice(full.size, 100, replace=False)
    assert np.array_equal(voronoi_labels((6, 10, 12), seeds, voxels=idx), full[idx])


def test_twin_split_of_a_whole_cell_grain_halves_it():
    """One grain filling the cell: the centroid is the seed voxel's centre minus half a
    voxel per axis (minimum-image offsets run over [-n/2, n/2)), and the plane x = centroid
    puts exactly half of the voxels on the twin side."""
    inp = RVEInputs((4, 6, 8), np.array([[0.3, 0.4, 0.6]]), np.zeros((2, 3)), np.array([1], np.uint8),
                    np.array([[1.0, 0.0, 0.0]]))
    lab = label_rve(inp)
    assert np.sum(lab == 1) == lab.size // 2
    # the seed voxel is i = 2; centroid x = 2.0; twin side is i + 1/2 - 2 > 0 (minimum image)
    assert np.all(lab[:, :, 2:6] == 1) and np.all(lab[:, :, [0, 1, 6, 7]] == 0)


def test_twin_split_slab_grain_along_y():
    seeds = np.array([[0.25, 0.5, 0.5], [0.75, 0.5, 0.5]])
    inp = RVEInputs((4, 8, 8), seeds, np.zeros((4, 3)), np.array([1, 0], np.uint8),
                    np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 0.0]]))
    lab = label_rve(inp)
    assert np.all(lab[:, :, 4:] == 1)
    left = lab[:, :, :4]
    assert np.sum(left == 2) == left.size // 2 and np.sum(left == 0) == left.size // 2
