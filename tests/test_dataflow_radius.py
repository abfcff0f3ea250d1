"""The dependency rule of the dataflow level launch, checked on the CPU.

A region of cell (i, j) covers cells i-1 .. i+1 and j-1 .. j+1, clipped to the image; its move
reads the labels of the region and of the one-pixel ring around it and writes the region's
labels.  The launch lets a region wait only for regions of earlier groups whose cells are
within three cells of its own in both directions.  These tests check, for every pair of
regions of small grids (cell sizes 1 to 6, images whose sides are not multiples of the cell),
that two regions that are farther apart neither read nor write each other's pixels, so their
moves commute, and that two regions of the same group never touch, so the group order is the
only order the launch has to keep.  They also check that the group index of the kernel,
4 (j mod 4) + (i mod 4), is the order of the 16 group launches.
"""
import itertools

import pytest


def region(i, j, s, W, H):
    return max(0, (i - 1) * s), min(W, (i + 2) * s), max(0, (j - 1) * s), min(H, (j + 2) * s)


def grow(b, W, H):
    return max(0, b[0] - 1), min(W, b[1] + 1), max(0, b[2] - 1), min(H, b[3] + 1)


def overlap(a, b):
    return a[0] < b[1] and b[0] < a[1] and a[2] < b[3] and b[2] < a[3]


def group(i, j):
    return 4 * (j % 4) + (i % 4)


@pytest.mark.parametrize("s,W,H", [(1, 13, 9), (2, 23, 17), (3, 31, 20), (5, 40, 31), (6, 47, 35)])
def test_regions_beyond_three_cells_commute(s, W, H):
    nx, ny = -(-W // s), -(-H // s)
    cells = [(i, j) for i in range(nx) for j in range(ny)]
    boxes = {c: region(*c, s, W, H) for c in cells}
    for a, b in itertools.combinations(cells, 2):
        A, B = boxes[a], boxes[b]
        touch = overlap(A, grow(B, W, H)) or overlap(B, grow(A, W, H))
        near = abs(a[0] - b[0]) <= 3 and abs(a[1] - b[1]) <= 3
        if touch:
            assert near, (a, b)
            assert group(*a) != group(*b), (a, b)


def test_group_index_is_the_launch_order():
    # the host builds the items of group g from cells with i % 4 = g & 3 and j % 4 = g >> 2
    for g in range(16):
        gi, gj = g & 3, g >> 2
        for i in range(gi, 20, 4):
            for j in range(gj, 20, 4):
                assert group(i, j) == g
