"""Host-side checks of the gather form's staging layout (bilinear streaming,
Eq. 33-38, gathered while the tensor-core step loads its operand): with the
constants read from the kernel header, every tap of every site of a 128-site
row tile falls inside the TMA box that the producer copies for its direction,
at the shared-memory offset the converter reads, within the direction's
region of the staging slot; the ghost fill writes only inside the box.  A
plain restatement of the index arithmetic in Python, run for every tap
offset the lattice projection can give and every box start parity, so that
a change of the constants or of the box rule that would read or write
outside the slot fails here rather than on the GPU."""
import os
import re

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(HERE, "..", "paper_2609_23057_b300", "csrc", "tc_common.cuh")


def _constants():
    src = open(HDR).read()
    tile = int(re.search(r"constexpr int kTileM = (\d+);", src).group(1))
    sites = int(re.search(r"#define RTLB_TC_GATHER_SITES (\d+)", src).group(1))
    dirs = int(re.search(r"constexpr int kGatherDirs = (\d+);", src).group(1))
    return tile, sites, dirs


def test_window_covers_every_tap():
    tile, G, dirs = _constants()
    assert G & (G - 1) == 0 and (tile % G) == 0
    cols = (tile + 1 + G - 1 + G - 1) // G * G           # kGatherCols
    box_bytes = 2 * cols * 16                              # kGatherBoxBytes
    dir_bytes = (box_bytes + 127) // 128 * 128             # kGatherDirBytes
    assert dir_bytes % 128 == 0 and dir_bytes * dirs % 128 == 0
    for n0x in range(-3, 3):                               # tap offsets n0 and n0 + 1 per axis
        for x0 in (0, tile, 2 * tile, 5 * tile):
            xs = x0 - n0x - 1                              # first site the taps read
            lead = xs & (G - 1)
            xe = xs - lead                                 # the box's first site
            assert xe % G == 0
            for r in range(tile):
                for bx in (0, 1):
                    for bz in (0, 1):
                        row, col = 1 - bz, r + 1 - bx
                        # the converter's offset and the site it stands for
                        off = row * cols * 16 + (col + lead) * 16
                        assert 0 <= off and off + 16 <= box_bytes <= dir_bytes
                        assert xe + col + lead == (x0 + r) - (n0x + bx)
            # the ghost fill's entries are the box's own
            for idx in range(2 * cols):
                assert idx * 16 + 16 <= box_bytes


@pytest.mark.parametrize("nx", [128, 256, 2048])
def test_tma_coordinate_is_aligned(nx):
    """The box's innermost coordinate is 0 (a group of G sites, 16 G bytes,
    is one box row, so the 16-byte rule on it holds), and the site-group
    coordinate is the group holding the first tap: the box starts at or below
    it by less than one group, and where it lies outside the lattice (left of
    0, right of nx) the copy fills zeros."""
    tile, G, _ = _constants()
    assert (16 * G) % 16 == 0
    cols = (tile + 1 + G - 1 + G - 1) // G * G
    for n0x in range(-3, 3):
        for x0 in range(0, nx, tile):
            xs = x0 - n0x - 1
            c1 = (xs - (xs & (G - 1))) // G
            assert c1 * G <= xs < c1 * G + G
            assert c1 * G + cols >= xs + tile + 1            # the last tap inside the box
