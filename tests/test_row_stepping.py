"""The division-free index stepping of the loss kernels' coalesced row staging
(k_loss, k_vloss; CPU): lane l of a warp takes the flat indices i = l + 32 k of a
block of rows of C floats, and its (row, column) advances by 32 as a mixed-radix
sum, (32 // C, 32 % C) with a carry.  For every class count the kernels accept
(1..32) and every lane, the stepped pair equals divmod(i, C), and the shared-memory
slot row * (C | 1) + column is in bounds and distinct across the block."""
import pytest


def _stepped(lane, C, n):
    """The (row, column) sequence a lane walks, as the kernels step it."""
    row, col = lane // C, lane % C
    drow, dcol = 32 // C, 32 % C
    out = []
    for i in range(lane, n, 32):
        out.append((i, row, col))
        row += drow
        col += dcol
        if col >= C:
            col -= C
            row += 1
    return out


@pytest.mark.parametrize("C", range(1, 33))
def test_stepping_equals_divmod(C):
    sp = C | 1
    for rows in (1, 7, 31, 32):  # a partial block and a whole one
        n = rows * C
        seen = set()
        for lane in range(32):
            for i, row, col in _stepped(lane, C, n):
                assert (row, col) == divmod(i, C)
                slot = row * sp + col
                assert 0 <= slot < 32 * sp
                assert slot not in seen
                seen.add(slot)
        assert len(seen) == n


def test_row_stride_spreads_lanes_over_banks():
    """Lane l's row starts at word l * (C | 1): an odd stride, so the 32 lanes reading
    column c of their own rows hit 32 distinct banks."""
    for C in range(1, 33):
        sp = C | 1
        for c in range(C):
            assert len({(lane * sp + c) % 32 for lane in range(32)}) == 32
