"""Host-side checks of the FP32 correction solve's work distribution (the persistent kernel of the
refined forms' L^-T L^-1 r, Eq. 2's two substitutions): the item sequences come from the kernel's own
iterator, run on the host through gp_debug_solve_items.

For every shape (tile rows Mt, CTAs G): (1) coverage — across the CTAs every forward tile product
(I, J), J <= I - 2, every chain step beta_I = y_I - M_I beta_{I-1}, every y product and the first block
appear exactly once, and likewise backward; each item belongs to its block's owner (block mod G);
(2) order — a block's y product follows all its tile products and precedes its chain step, backward
items of a block follow its forward chain step; (3) progress — a simulation in which each CTA runs its
items in order, blocking until the block an item needs is published, publishes every block of both
sweeps in order, with no deadlock for any CTA count.
"""
import ctypes
import itertools

import numpy as np
import pytest

import __graft_entry__
from paper_2602_19683_gb300 import _native as N

FT, FF, FP, FD, BT, BF, BP, BD = range(8)


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return N.load()


def items(lib, Mt, G, c):
    n = lib.gp_debug_solve_items(Mt, G, c, None, 0)
    assert n >= 0
    out = np.zeros(3 * max(n, 1), dtype=np.int32)
    assert lib.gp_debug_solve_items(Mt, G, c, out.ctypes.data_as(ctypes.c_void_p), n) == n
    return [tuple(int(v) for v in out[3 * k:3 * k + 3]) for k in range(n)]


def expected(Mt):
    e = [(FT, I, J) for I in range(Mt) for J in range(I - 1)] + [(FD, 0, 0)]
    e += [(FP, I, I) for I in range(1, Mt)] + [(FF, I, I - 1) for I in range(1, Mt)]
    e += [(BT, I, J) for I in range(Mt) for J in range(I - 1)] + [(BD, Mt - 1, Mt - 1)]
    e += [(BP, J, J) for J in range(Mt - 1)] + [(BF, J + 1, J) for J in range(Mt - 1)]
    return sorted(e)


def block_of(kind, I, J):
    return I if kind < BT else J


@pytest.mark.parametrize("Mt,G", list(itertools.product([1, 2, 3, 4, 7, 40, 153, 256], [1, 2, 3, 5, 152])))
def test_solve_items_cover_order_and_progress(lib, Mt, G):
    Ge = min(G, Mt)
    seqs = [items(lib, Mt, G, c) for c in range(Ge)]
    assert sorted(x for s in seqs for x in s) == expected(Mt)
    for c, s in enumerate(seqs):
        assert all(block_of(*x) % Ge == c for x in s)
        pos = {x: k for k, x in enumerate(s)}
        for kind, I, J in s:
            if kind == FP:
                assert all(pos[(FT, I, j)] < pos[(FP, I, I)] for j in range(I - 1))
                assert pos[(FP, I, I)] < pos[(FF, I, I - 1)]
            if kind == BP:
                assert all(pos[(BT, i, J)] < pos[(BP, J, J)] for i in range(J + 2, Mt))
                assert pos[(BP, J, J)] < pos[(BF, J + 1, J)]
                fwd_final = (FD, 0, 0) if J == 0 else (FF, J, J - 1)
                assert pos[fwd_final] < pos[(BP, J, J)]
    # progress: forward blocks publish in order 0..Mt-1, backward blocks Mt-1..0
    front_f = front_b = 0
    idx = [0] * Ge
    while any(idx[c] < len(seqs[c]) for c in range(Ge)):
        moved = False
        for c in range(Ge):
            if idx[c] >= len(seqs[c]):
                continue
            kind, I, J = seqs[c][idx[c]]
            if kind in (FT, FF) and front_f < J + 1:
                continue
            if kind in (BT, BF) and front_b < Mt - I:
                continue
            if kind in (FD, FF):
                assert front_f == I
                front_f = I + 1
            if kind in (BD, BF):
                assert front_b == Mt - 1 - J
                front_b = Mt - J
            idx[c] += 1
            moved = True
        assert moved, f"no CTA can proceed (Mt={Mt}, G={G}, positions {idx})"
    assert front_f == Mt and front_b == Mt


def test_solve_items_reject_bad_arguments(lib):
    assert lib.gp_debug_solve_items(0, 1, 0, None, 0) == -1
    assert lib.gp_debug_solve_items(4, 0, 0, None, 0) == -1
    assert lib.gp_debug_solve_items(4, 2, 2, None, 0) == -1  # CTA index beyond the CTAs used
