"""The rule the device uses to fill the holes of domino shuffling, checked on
the CPU against the column-walk rule.

After the destruction and sliding steps of order k -> K = k + 1, the empty
cells of the order-K diamond form disjoint 2x2 blocks whose lower-left cells
have x + y + K odd, stacked from the bottom of every run of empty cells in a
column.  The device lets each empty cell find its block from its 3x3
neighbourhood when only one of the two candidate blocks has its other three
cells empty, and from the parity of the run below it otherwise.  This replay
of the shuffling algorithm (with numpy coin flips for the blocks: the rule,
not the random stream, is under test) checks that every local decision names
the block the column walk names, that the walk is rarely needed, and that
every step ends in a tiling of the diamond.  No GPU.
"""
import numpy as np
import pytest

EMPTY, HL, HR, VB, VT = 0, 1, 2, 3, 4


def in_diamond(x, y, k):
    return abs(2 * x + 1) + abs(2 * y + 1) <= 2 * k


def move(A, k):
    """Destruction and sliding of the order-k tiling A (dict cell -> part)."""
    K = k + 1

    def cell(x, y):
        return A.get((x, y), EMPTY)

    def survives(ax, ay, horizontal):
        north_or_east = ((ax + ay + k) & 1) == 0
        if horizontal:
            return cell(ax, ay + 1) != HL if north_or_east else cell(ax, ay - 1) != HL
        return cell(ax + 1, ay) != VB if north_or_east else cell(ax - 1, ay) != VB

    B = {}
    for y in range(-K, K):
        for x in range(-K, K):
            if not in_diamond(x, y, K):
                continue
            out = EMPTY
            c = cell(x, y - 1)   # from below, going north
            if c in (HL, HR):
                ax = x if c == HL else x - 1
                if ((ax + y - 1 + k) & 1) == 0 and survives(ax, y - 1, True):
                    out = c
            c = cell(x, y + 1)   # from above, going south
            if c in (HL, HR):
                ax = x if c == HL else x - 1
                if ((ax + y + 1 + k) & 1) == 1 and survives(ax, y + 1, True):
                    out = c
            c = cell(x - 1, y)   # from the left, going east
            if c in (VB, VT):
                ay = y if c == VB else y - 1
                if ((x - 1 + ay + k) & 1) == 0 and survives(x - 1, ay, False):
                    out = c
            c = cell(x + 1, y)   # from the right, going west
            if c in (VB, VT):
                ay = y if c == VB else y - 1
                if ((x + 1 + ay + k) & 1) == 1 and survives(x + 1, ay, False):
                    out = c
            if out:
                B[(x, y)] = out
    return B


def block_by_walk(B, x, y, K):
    below, yy = 0, y - 1
    while yy >= -K and in_diamond(x, yy, K) and B.get((x, yy), EMPTY) == EMPTY:
        below += 1
        yy -= 1
    by = y - 1 if below & 1 else y
    bx = x if (x + by + K) & 1 else x - 1
    return bx, by


def block_local(B, x, y, K):
    """The block from the 3x3 neighbourhood, or None where two blocks fit."""
    def hole(dx, dy):
        return in_diamond(x + dx, y + dy, K) and B.get((x + dx, y + dy), EMPTY) == EMPTY
    odd = (x + y + K) & 1
    if odd:
        h1 = hole(1, 0) and hole(0, 1) and hole(1, 1)      # block at (x, y)
        h2 = hole(-1, 0) and hole(0, -1) and hole(-1, -1)  # block at (x - 1, y - 1)
        cand = ((x, y), (x - 1, y - 1))
    else:
        h1 = hole(-1, 0) and hole(-1, 1) and hole(0, 1)    # block at (x - 1, y)
        h2 = hole(0, -1) and hole(1, -1) and hole(1, 0)    # block at (x, y - 1)
        cand = ((x - 1, y), (x, y - 1))
    if h1 == h2:
        return None
    return cand[0] if h1 else cand[1]


@pytest.mark.parametrize("n,seed", [(5, 1), (12, 2), (30, 3), (45, 4)])
def test_local_block_rule_matches_column_walk(n, seed):
    rng = np.random.default_rng(seed)
    A = {}
    local = walked = empty = cells = 0
    for k in range(n):
        K = k + 1
        B = move(A, k)
        C = dict(B)
        draws = {}
        for y in range(-K, K):
            for x in range(-K, K):
                if not in_diamond(x, y, K):
                    continue
                cells += 1
                if B.get((x, y), EMPTY) != EMPTY:
                    continue
                empty += 1
                bx, by = block_by_walk(B, x, y, K)
                loc = block_local(B, x, y, K)
                if loc is None:
                    walked += 1
                else:
                    assert loc == (bx, by), (n, K, x, y)
                    local += 1
                if (bx, by) not in draws:
                    draws[(bx, by)] = rng.random() < 0.5
                if draws[(bx, by)]:
                    C[(x, y)] = HR if x > bx else HL
                else:
                    C[(x, y)] = VT if y > by else VB
        # a tiling of the order-K diamond: every cell covered, halves paired
        for y in range(-K, K):
            for x in range(-K, K):
                if in_diamond(x, y, K):
                    v = C.get((x, y), EMPTY)
                    assert v != EMPTY
                    if v == HL:
                        assert C.get((x + 1, y)) == HR
                    if v == VB:
                        assert C.get((x, y + 1)) == VT
        A = C
    assert local + walked == empty
    # the walk is the exception, and holes are far from rare
    assert walked <= 0.15 * empty
    if n >= 30:
        assert empty >= 0.2 * cells
