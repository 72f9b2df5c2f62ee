"""Host-side checks of the C ABI: the library builds, loads and exports every declared entry point,
argument validation works without a GPU, and the persistent kernel's dispatch orders are
topological orders of the tiled algorithms' dependency graphs (Sec. 3.2, Fig. 1; Eqs. 2-3)."""
import ctypes
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_2602_19683_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return N.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gp_status|const char\*|int64_t|void)\s+(gp_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert name in N.SIGNATURES, f"binding lacks {name}"


def test_no_gpu_or_bad_args_are_rejected(lib):
    h = ctypes.c_void_p()
    s = lib.gp_create(ctypes.byref(h), 0, None, None)
    import torch
    if not torch.cuda.is_available():
        assert s == N.GP_ERR_NO_DEVICE
    else:
        assert s == N.GP_OK
        lib.gp_destroy(h)
    assert lib.gp_create(None, 0, None, None) == N.GP_ERR_INVALID_ARG
    assert lib.gp_cholesky(None, None) == N.GP_ERR_INVALID_ARG
    assert lib.gp_status_string(N.GP_ERR_NOT_PD) == b"matrix not positive definite"


def tasks(lib, graph, Mt, Mc, T, workers, mixed=0):
    cnt = lib.gp_schedule_tasks(graph, Mt, Mc, T, workers, mixed, None, 0)
    out = np.zeros((cnt, 4), dtype=np.int32)
    assert lib.gp_schedule_tasks(graph, Mt, Mc, T, workers, mixed, out.ctypes.data, cnt) == cnt
    return out


@pytest.mark.parametrize("Mt,workers,mixed", [(1, 4, 0), (2, 1, 0), (5, 3, 1), (9, 304, 0), (16, 304, 1),
                                               (16, 152, 3), (40, 152, 3)])
def test_cholesky_schedule_is_topological(lib, Mt, workers, mixed):
    """Every tile of the lower triangle receives POTRF/TRSM once and its updates J = 0..min-1 in order,
    and each task appears after the tasks whose tiles it reads (Fig. 1's dependencies)."""
    T = 128 if mixed else 64  # mixed 128-tiles group their updates
    t = tasks(lib, 0, Mt, 0, T, workers, mixed)
    if not mixed:
        assert len(t) == 2 * Mt + Mt * (Mt - 1) // 2 + sum((Mt - J - 1) * (Mt - J) // 2 for J in range(Mt))
    cnt = {}  # tile -> updates applied (+1 once final)
    inverted = set()
    paired = 0
    for kind, p, q, r in t:
        if kind == 0:
            assert cnt.get((p, p), 0) == p
            cnt[(p, p)] = p + 1
        elif kind == 14:  # TRTRI(J): after POTRF(J), once
            assert cnt.get((p, p), 0) == p + 1 and p not in inverted
            inverted.add(p)
        elif kind == 1:
            assert cnt.get((q, q), 0) == q + 1 and cnt.get((p, q), 0) == q and p > q
            cnt[(p, q)] = q + 1
        elif kind in (2, 19):  # columns [J0, J1) of updates, r = J0 | J1 << 16; 19: rows p and p + 1
            J0, J1 = r & 0xFFFF, (r >> 16) or (r & 0xFFFF) + 1
            rows = (p, p + 1) if kind == 19 else (p,)
            assert mixed or kind == 2
            for I in rows:
                assert I < Mt and I >= q >= J1 > J0 >= 0 and J1 - J0 <= 8
                for J in range(J0, J1):
                    assert cnt.get((I, J), 0) == J + 1 and cnt.get((q, J), 0) == J + 1
                assert cnt.get((I, q), 0) == J0
            for I in rows:
                cnt[(I, q)] = J1
            paired += kind == 19
        else:
            raise AssertionError(kind)
    assert all(cnt[(I, J)] == J + 1 for I in range(Mt) for J in range(I + 1))
    assert inverted == set(range(Mt))
    if mixed and Mt >= 16:  # tile 128 on the tensor cores: grouped updates of row pairs share L_KJ
        assert paired > 0


@pytest.mark.parametrize("Mt,workers,variant", [(1, 3, 4), (2, 1, 4), (9, 304, 4), (12, 152, 5), (5, 2, 5)])
def test_left_and_top_looking_schedules(lib, Mt, workers, variant):
    """The left-/top-looking Cholesky graphs (Sec. 3.2's other tile variants): every tile takes all its
    updates (columns 0..K-1) in one task after those columns are final, then its POTRF/TRSM; the order
    is topological, and the factor-final events follow the variant's column / row order."""
    t = tasks(lib, 0, Mt, 0, 64, workers, variant)
    assert len(t) == 2 * Mt + Mt * (Mt - 1) // 2 + Mt * (Mt + 1) // 2 - Mt
    cnt, final_order = {}, []
    for kind, p, q, r in t:
        if kind == 0:
            assert cnt.get((p, p), 0) == p
            cnt[(p, p)] = p + 1
            final_order.append((p, p))
        elif kind == 14:
            assert cnt.get((p, p), 0) == p + 1
        elif kind == 1:
            assert cnt.get((q, q), 0) == q + 1 and cnt.get((p, q), 0) == q
            cnt[(p, q)] = q + 1
            final_order.append((p, q))
        elif kind == 2:
            J0, J1 = r & 0xFFFF, r >> 16
            assert J0 == 0 and J1 == q >= 1 and p >= q
            for J in range(J1):
                assert cnt.get((p, J), 0) == J + 1 and cnt.get((q, J), 0) == J + 1
            assert cnt.get((p, q), 0) == 0
            cnt[(p, q)] = J1
        else:
            raise AssertionError(kind)
    assert all(cnt[(I, J)] == J + 1 for I in range(Mt) for J in range(I + 1))
    if workers == 1:  # one worker follows the variant's order exactly
        key = (lambda ij: (ij[1], ij[0])) if variant == 4 else (lambda ij: ij)
        assert final_order == sorted(final_order, key=key)


@pytest.mark.parametrize("Mt,Mc,workers,mixed", [(1, 1, 2, 0), (4, 3, 5, 0), (7, 2, 304, 0), (1, 1, 2, 1),
                                                 (9, 3, 5, 1), (13, 2, 304, 1)])
def test_cov_schedule_is_topological(lib, Mt, Mc, workers, mixed):
    """L V = K_{X,Xs} then S -= V^T V (Eq. 3): every block of V is solved after all its updates, in J
    order; mixed 128-tiles group the products (V_Ic over J0..J1 while far from its solve, S_ab over g
    consecutive J)."""
    t = tasks(lib, 1, Mt, Mc, 128 if mixed else 64, workers, mixed)
    cv, cs = {}, {}
    for kind, p, q, r in t:
        if kind == 3:
            assert cv.get((p, q), 0) == p
            cv[(p, q)] = p + 1
        elif kind == 4:
            assert cv.get((q, r), 0) == q + 1 and cv.get((p, r), 0) == q and p > q
            cv[(p, r)] = q + 1
        elif kind == 5:
            assert p >= q and cv.get((r, p), 0) == r + 1 and cv.get((r, q), 0) == r + 1 and cs.get((p, q), 0) == r
            cs[(p, q)] = r + 1
        elif kind == 15:  # V_Ic -= sum_{J0 <= J < J1} L_IJ V_Jc
            J0, J1 = r & 0xFFFF, r >> 16
            assert mixed and p >= J1 > J0 >= 0 and J1 - J0 <= 8 and cv.get((p, q), 0) == J0
            assert all(cv.get((J, q), 0) == J + 1 for J in range(J0, J1))
            assert J1 - J0 == 1 or J1 <= p - 2  # the two columns next to the solve stay single
            cv[(p, q)] = J1
        elif kind == 16:  # S_ab -= sum_{J0 <= J < J1} V_Ja^T V_Jb
            J0, J1 = r & 0xFFFF, r >> 16
            assert mixed and p >= q and J1 - J0 <= 8 and cs.get((p, q), 0) == J0
            assert all(cv.get((J, p), 0) == J + 1 and cv.get((J, q), 0) == J + 1 for J in range(J0, J1))
            cs[(p, q)] = J1
        else:
            raise AssertionError(kind)
    assert all(cs[(a, b)] == Mt for a in range(Mc) for b in range(a + 1))
    assert all(cv[(I, c)] == I + 1 for I in range(Mt) for c in range(Mc))


@pytest.mark.parametrize("Mt,T,workers", [(1, 32, 1), (3, 64, 2), (6, 96, 304)])
def test_mean_schedule_is_topological(lib, Mt, T, workers):
    """L beta = y then L^T alpha = beta (Eq. 2): each diagonal block is solved in 32-row chunks after
    every update of all its chunks; a block's updates of later blocks follow all its chunks."""
    t = tasks(lib, 2, Mt, 0, T, workers)
    nch = T // 32
    cf, cb, df, db = {}, {}, {}, {}
    for kind, p, q, r in t:
        if kind == 17:  # forward chunk q of block p
            assert all(cf.get((p, ch), 0) == p for ch in range(nch))
            df[p] = df.get(p, 0) + 1
        elif kind == 7:
            assert df.get(q, 0) == nch and cf.get((p, r), 0) == q and p > q
            cf[(p, r)] = q + 1
        elif kind == 18:  # backward chunk q of block p
            assert df.get(p, 0) == nch and all(cb.get((p, ch), 0) == Mt - 1 - p for ch in range(nch))
            db[p] = db.get(p, 0) + 1
        elif kind == 9:
            assert db.get(q, 0) == nch and df.get(p, 0) == nch and cb.get((p, r), 0) == Mt - 1 - q and q > p
            cb[(p, r)] = Mt - q
        else:
            raise AssertionError(kind)
    assert all(df[J] == nch and db[J] == nch for J in range(Mt))


@pytest.mark.parametrize("Mt,workers,mixed", [(1, 2, 0), (2, 1, 0), (5, 7, 1), (9, 304, 0)])
def test_adjoint_schedule_is_topological(lib, Mt, workers, mixed):
    """The reverse sweep (adjoint of Fig. 1): for each J from the last column down, RUPD(P, K, J) for
    all P, K > J with K descending per P, after the adjoint of tile (max(P,K), min(P,K)) is final;
    RTRSM(P, J) after all of them; RDIAG(P, J) in P order within each of 8 partial sums; RPOTRF(J)
    after every part. Mirrors the device's counter waits."""
    t = tasks(lib, 3, Mt, 0, 64, workers, mixed)
    assert len(t) == sum((Mt - 1 - J) ** 2 + 2 * (Mt - 1 - J) + 1 for J in range(Mt))
    parts = 8
    rc, fa, rd = {}, set(), {}
    for kind, p, q, r in t:
        if kind == 10:  # K descending per (P, J)
            hi, lo = max(p, q), min(p, q)
            assert p > r and q > r and (hi, lo) in fa and rc.get((p, r), 0) == Mt - 1 - q
            rc[(p, r)] = Mt - q
        elif kind == 11:
            assert rc.get((p, q), 0) == Mt - 1 - q
            fa.add((p, q))
        elif kind == 12:
            part, k = (p - q - 1) % parts, (p - q - 1) // parts
            assert (p, q) in fa and rd.get((q, part), 0) == k
            rd[(q, part)] = k + 1
        elif kind == 13:
            for part in range(parts):
                cnt = max(0, -(-(Mt - 1 - p - part) // parts))
                assert rd.get((p, part), 0) == cnt
            fa.add((p, p))
        else:
            raise AssertionError(kind)
    assert fa == {(I, J) for I in range(Mt) for J in range(I + 1)}


def test_schedule_rejects_bad_arguments(lib):
    assert lib.gp_schedule_tasks(0, 4, 0, 48, 1, 0, None, 0) == -1
    assert lib.gp_schedule_tasks(0, 4, 0, 64, 1, 6, None, 0) == -1
    assert lib.gp_schedule_tasks(5, 4, 0, 64, 1, 0, None, 0) == -1
    assert lib.gp_schedule_tasks(0, 4, 0, 64, 0, 0, None, 0) == -1
    assert lib.gp_schedule_tasks(0, 4, 0, 128, 1, 2, None, 0) == -1
    assert lib.gp_schedule_tasks(0, 4, 0, 128, 1, 7, None, 0) == -1


def _shared_neighbours(t):
    """Fraction of consecutive grouped updates (in dispatch order) that share a packed operand group
    (same row I or same column K, same first column J0) with the one started just before."""
    g = [(p, q, r & 0xFFFF) for kind, p, q, r in t if kind in (2, 19) and (r >> 16) - (r & 0xFFFF) > 1]
    same = sum(1 for a, b in zip(g, g[1:]) if a[2] == b[2] and (a[0] == b[0] or a[1] == b[1]))
    return same / max(1, len(g) - 1)


def test_locality_order_starts_operand_sharers_together(lib):
    """cfg.locality_order: the same tasks (a valid order, checked above) with far more grouped updates
    started right after one that reads the same packed operand group."""
    base = tasks(lib, 0, 128, 0, 128, 152, 1)
    loc = tasks(lib, 0, 128, 0, 128, 152, 3)
    assert sorted(map(tuple, base)) == sorted(map(tuple, loc))
    assert _shared_neighbours(loc) > 0.8 and _shared_neighbours(base) < 0.3


def test_autotune_cache_key_and_class_table():
    """Host logic of the autotuner's JSON cache: batches of the same coarse shape share a key, other
    shapes, precisions or GPUs do not; GPs take their size class's tile edge."""
    from paper_2602_19683_gb300 import api
    shape = [(n, 256, d) for n, d in zip((130, 900, 4000, 2100, 700, 3000), (4, 8, 16, 4, 8, 16))]
    k = api.autotune_cache_key("GB300", "fp64", shape, True)
    near = [(n + 7, m, d) for n, m, d in shape]  # same power-of-two buckets
    assert api.autotune_cache_key("GB300", "fp64", near, True) == k
    assert api.autotune_cache_key("GB300", "fp32", shape, True) != k
    assert api.autotune_cache_key("B200", "fp64", shape, True) != k
    assert api.autotune_cache_key("GB300", "fp64", shape, False) != k
    assert api.autotune_cache_key("GB300", "fp64", shape + [(5000, 256, 8)] * 3, True) != k
    assert api.autotune_cache_key("GB300", "fp64", shape, True, tiles=(64, 32)) == \
        api.autotune_cache_key("GB300", "fp64", shape, True, tiles=(32, 64, 0))
    table = [{"n_max": 700, "tile": 32}, {"n_max": 2100, "tile": 64}, {"n_max": 4000, "tile": 128}]
    assert api.tiles_from_classes(table, [1, 700, 701, 2100, 4000, 9999]) == [32, 32, 64, 64, 128, 128]
