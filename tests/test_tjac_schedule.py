"""Index schedules of the tensor-core block Jacobi (tjacobi.cu), checked on
the CPU: the same formulas as the host loop and the kernels, run over every
case they take.

  * Block slots paired in odd-even order (even rounds (0, 1), (2, 3), ...,
    odd rounds (1, 2), (3, 4), ..., the two blocks of a pair changing slots):
    in nb rounds every pair of blocks meets exactly once, and the block order
    is reversed, which is where the write-back finds each block.
  * The in-CTA sweep: the circle-method steps (first round) and the cross
    steps (i, b + (i + t) mod b) (later rounds) are disjoint within a step and
    cover their pairs once; the enumeration of the upper 2 x 2 blocks of a
    step's pairs in double rows covers each block once.
"""
import itertools

import pytest


def odd_even_rounds(nb):
    """Pairs of block slots per round, as the host loop issues them."""
    P0 = nb // 2
    for rnd in range(nb):
        par = rnd & 1
        P = P0 - 1 if par else P0
        yield [(par + 2 * p, par + 2 * p + 1) for p in range(P)]


def final_slot(B, nb, sweeps):
    """Slot of block B after `sweeps` outer sweeps (the store kernel's rule)."""
    return nb - 1 - B if sweeps & 1 else B


@pytest.mark.parametrize("nb", [2, 4, 6, 8, 10, 16, 32, 64])
def test_odd_even_pairs_meet_once_and_reverse(nb):
    slots = list(range(nb))                     # slot -> block
    for sweeps in range(1, 4):
        met = []
        for pairs in odd_even_rounds(nb):
            used = set()
            for a, b in pairs:
                assert a not in used and b not in used and b < nb
                used |= {a, b}
                met.append(frozenset((slots[a], slots[b])))
                slots[a], slots[b] = slots[b], slots[a]
        assert len(met) == len(set(met)) == nb * (nb - 1) // 2
        for B in range(nb):
            assert slots[final_slot(B, nb, sweeps)] == B


def circle(np_, t, p):
    q = np_ - 1
    if p == 0:
        return q, t
    return (t + p) % q, (t - p + q) % q


@pytest.mark.parametrize("TB", [64, 128])
def test_in_cta_steps_cover_their_pairs(TB):
    H = TB // 2
    # first round: circle method over all TB vectors, TB - 1 steps
    seen = set()
    for t in range(TB - 1):
        idx = set()
        for p in range(H):
            i, j = circle(TB, t, p)
            assert i != j and i not in idx and j not in idx
            idx |= {i, j}
            seen.add(frozenset((i, j)))
    assert seen == {frozenset(c) for c in itertools.combinations(range(TB), 2)}
    # later rounds: the b^2 pairs between the two blocks, b steps
    seen = set()
    for t in range(H):
        idx = set()
        for i in range(H):
            j = H + (i + t) % H
            assert i not in idx and j not in idx
            idx |= {i, j}
            seen.add((i, j))
    assert seen == {(i, j) for i in range(H) for j in range(H, TB)}


@pytest.mark.parametrize("H", [32, 64])
def test_upper_block_enumeration(H):
    seen = []
    for e in range(H // 2 * (H + 1)):
        d, jj = divmod(e, H + 1)
        if jj < H - d:
            k1, k2 = d, d + jj
        else:
            k1 = H - 1 - d
            k2 = k1 + (jj - (H - d))
        assert 0 <= k1 <= k2 < H
        seen.append((k1, k2))
    assert sorted(seen) == [(a, b) for a in range(H) for b in range(a, H)]
