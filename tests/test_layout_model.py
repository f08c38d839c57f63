"""Host-side checks of the symmetric panel layout, without a GPU.

A NumPy model of the layout arithmetic (slabs, steps, stored warp slices, the
[w][rt][lane][cc] order) is checked for: (1) the library's nsrgs_packed_bytes
(a host function of libnsrgs.so) agrees with it; (2) every element of the
strict block-upper triangle lands in exactly one stored slot and every other
slot holds a zero; (3) walking the steps as the stream kernel does (row
partials into Y[rows], column partials into Y[cols]) rebuilds A_off X; (4) the
reads and writes stay inside the buffers the library sizes (packed buffer,
X/Y padded to n*d + 64 rows) and every bulk copy is 16-byte aligned.
"""
import numpy as np
import pytest

import synth

from _panel_model import Geom, slot_coords, walk


CASES = [(2, 1, 0), (2, 3, 0), (5, 2, 1), (130, 3, 0), (131, 3, 1), (200, 3, 2), (257, 4, 0), (300, 1, 2), (513, 2, 0), (140, 4, 2),
         (257, 4, 1), (97, 4, 1), (300, 1, 1), (1100, 3, 1), (900, 4, 2), (1300, 2, 1),
         (3, 5, 0), (70, 5, 1), (67, 6, 0), (66, 7, 1), (130, 8, 0), (65, 8, 1)]


@pytest.mark.parametrize("n,d,storage", CASES)
def test_layout_is_a_bijection_and_rebuilds_AX(n, d, storage):
    g = Geom(n, d, storage)
    N = n * d
    inst = synth.make_instance(n, d, 0.7, seed=n + d)
    A = inst.dense()
    Aoff = A.copy()
    for i in range(n):
        Aoff[i * d : (i + 1) * d, i * d : (i + 1) * d] = 0.0
    hit = np.zeros((N, N), dtype=np.int64)
    X = np.random.default_rng(0).standard_normal((N + 64, d))
    X[N:] = 0.0
    Y = np.zeros((N + 64, d))
    xpad = N + 64
    total = 0
    for b, q, W, off in walk(g):
        rows, cols = slot_coords(g, b, q, W)
        assert rows.max() < (b + 1) * g.SB * d
        # bulk copies: 16-byte aligned sources and sizes; X rows inside the padding
        assert (g.header_bytes() + off) % 16 == 0 and (W * g.WB) % 16 == 0
        xcol = b * g.SB * d + q * g.SC
        assert (xcol * d * 4) % 16 == 0 and xcol + g.SC <= xpad
        inside = (rows < N) & (cols < N)
        ib = np.where(inside, rows // d, 0)
        jb = np.where(inside, cols // d, 0)
        upper = inside & (jb > ib)
        np.add.at(hit, (rows[upper], cols[upper]), 1)
        vals = np.zeros(rows.shape)
        vals[upper] = Aoff[rows[upper], cols[upper]]
        # stream-kernel walk: row partials -> Y[rows < N], column partials -> Y[cols] (padded)
        for rr, cc_, v in zip(rows, cols, vals):
            if v != 0.0:
                Y[rr] += v * X[cc_]
                Y[cc_] += v * X[rr]
        total += W * g.WB
    assert total == g.panel_bytes()
    iu = np.zeros((N, N), dtype=bool)
    for i in range(n):
        iu[i * d : (i + 1) * d, (i + 1) * d :] = True
    assert np.all(hit[iu] == 1), "an upper element is missing or duplicated"
    assert np.all(hit[~iu] == 0)
    assert np.allclose(Y[:N], Aoff @ X[:N], atol=1e-10)
    assert np.all(Y[N:] == 0.0)


@pytest.mark.parametrize("n,d,storage", CASES + [(10000, 3, 0), (10000, 3, 1), (10000, 3, 2), (2000, 4, 0), (3000, 8, 0), (2500, 6, 1)])
def test_packed_bytes_match_library(n, d, storage):
    L = pytest.importorskip("paper_2604_07372_gb300._lib")
    try:
        lib = L.lib()
    except RuntimeError:
        pytest.skip("libnsrgs.so not built")
    g = Geom(n, d, storage)
    assert lib.nsrgs_packed_bytes(n, d, storage) == g.header_bytes() + g.panel_bytes()


@pytest.mark.parametrize("n,d,storage", CASES + [(10000, 3, 0), (10000, 3, 1), (2000, 4, 2)])
def test_warp_count_nondecreasing_along_a_slab(n, d, storage):
    """The stream kernel recomputes a step's stored warp count only until it reaches NW."""
    g = Geom(n, d, storage)
    for b in range(g.nslabs):
        ws = [g.warps(b, q) for q in range(g.steps(b))]
        assert all(x <= y for x, y in zip(ws, ws[1:]))
        assert ws[0] >= 1
        # 32-bit step arithmetic in the kernel: the last column index fits easily
        assert b * g.SB * d + g.steps(b) * g.SC < 2**31


def test_stored_bytes_close_to_algorithmic():
    """At n = 10^4, d = 3 the stored panels exceed the packed triangle by < 0.5%."""
    n, d = 10000, 3
    for st in (0, 1, 2):
        g = Geom(n, d, st)
        alg = n * (n - 1) // 2 * d * d * g.E
        assert g.panel_bytes() / alg - 1.0 < 0.005
