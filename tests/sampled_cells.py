"""One-cell check of a coarse step on sampled cells (test helper).

Away from walls, domain faces and refinement interfaces a level-l cell is
advanced by 2^l plain collide-stream updates per coarse step (Sec. 2.2; the
recursive sub-cycling of the octree refinement):
f_i(x, t + 1) = C(f(x - c_i, t))_i, with C the cumulant collision at the
level's rate omega1 = 1 / (3 nu_l + 1/2).  For a cell whose neighbourhood of
radius 2^l is all fluid, the populations after the coarse step follow from
the populations before it by that recursion alone, each collision computed
one cell at a time by the FP64 oracle.  This is how a run too large for the
oracle is checked: a sample of its cells, one by one.
"""
import numpy as np
from scipy import ndimage

import oracle as O

C27 = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)])


def interior(types, radius):
    """Cells whose (2 radius + 1)^3 neighbourhood lies in the level's box and
    holds only fluid cells (type 0: not solid, not covered by a finer level)."""
    return ndimage.binary_erosion(types == 0, structure=np.ones((2 * radius + 1,) * 3, bool), border_value=0)


def pick(mask, n, seed):
    """Up to n distinct (z, y, x) cells where mask is set, drawn with a seeded generator."""
    idx = np.flatnonzero(mask)
    sel = np.random.default_rng(seed).choice(idx, size=min(n, len(idx)), replace=False)
    return np.stack(np.unravel_index(np.sort(sel), mask.shape), -1)


class Recursion:
    """f(cell) after `updates` collide-stream updates of the state S
    (z, y, x, 27), each cell's collision computed once (memoised)."""

    def __init__(self, S, nu):
        self.S, self.r, self.memo, self.post_memo = S, O.rates(1.0 / (3.0 * nu + 0.5)), {}, {}

    def post(self, cell, updates):
        """The collision of cell's populations after `updates` updates."""
        key = (cell, updates)
        if key not in self.post_memo:
            self.post_memo[key] = O.collide(self.after(cell, updates), self.r)
        return self.post_memo[key]

    def after(self, cell, updates):
        cell = tuple(int(v) for v in cell)
        key = (cell, updates)
        if key in self.memo:
            return self.memo[key]
        if updates == 0:
            out = self.S[cell]
        else:
            out = np.empty(27)
            for i in range(27):
                cx, cy, cz = C27[i]
                out[i] = self.post((cell[0] - cz, cell[1] - cy, cell[2] - cx), updates - 1)[i]
        self.memo[key] = out
        return out


def window_all_fluid(types, cell, radius):
    """True when the (2 radius + 1)^3 window around cell (z, y, x) lies in the
    level's box and holds only fluid cells."""
    lo = [int(c) - radius for c in cell]
    if min(lo) < 0 or any(int(c) + radius >= types.shape[a] for a, c in enumerate(cell)):
        return False
    return bool((types[lo[0]:lo[0] + 2 * radius + 1, lo[1]:lo[1] + 2 * radius + 1,
                       lo[2]:lo[2] + 2 * radius + 1] == 0).all())


def check_level(S0, S1, types, level, nu_level, n, seed, atol):
    """Compare S1 on n sampled interior cells of a level with the one-cell
    recursion from S0; returns (cells checked, max error, max |S1 - S0|)."""
    k = 2 ** level
    cells = pick(interior(types, k), n, seed)
    rec = Recursion(S0, nu_level)
    err = moved = 0.0
    for c in cells:
        want = rec.after(c, k)
        got = S1[tuple(c)]
        e = float(np.abs(got - want).max())
        assert e < atol, "level %d cell (z,y,x) = %s: max |f - f_oracle| = %g" % (level, tuple(c), e)
        err = max(err, e)
        moved = max(moved, float(np.abs(got - S0[tuple(c)]).max()))
    return len(cells), err, moved
