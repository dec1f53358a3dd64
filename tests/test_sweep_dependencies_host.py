"""Dependency lists of the multi-step sweep (host logic, no GPU).

Before step k of a tile the persistent kernels wait for the tiles in its
list to finish step k - 1.  Here the lists the library builds are checked
against the tiles' read windows derived from the TMA geometry alone: a
tile of strip s and segment g reads rows ya - 4 .. yb + 4 and the window's
columns from x0 - 4 (124 for FP32, 128 for 16-bit storage); a position is
written by the tile owning its site, or -- for a ghost column or, without
walls, a ghost row -- the tile owning the site it is the periodic image of;
with walls the rows outside the lattice are never written, and neither are
the padded columns beyond the 4-column ghost band.  Every writer of a
position a tile reads must be in its list (it must have written the
previous step), and the tile must be in every such writer's list (the
writer must not overwrite the buffer before the tile has read it)."""
import numpy as np
import pytest

from paper_1307_6703_gb300 import LB_BF16DEV, LB_FP16DEV, LB_FP32, LBError, lb_sweep_dependencies

WINDOW = {LB_FP32: 124, LB_BF16DEV: 128, LB_FP16DEV: 128}
QUANTUM = {LB_FP32: 4, LB_BF16DEV: 8, LB_FP16DEV: 8}


def _required(prec, nx, ny, walls, nstrips, seg_h):
    q, cols = QUANTUM[prec], WINDOW[prec]
    base = q * (nx // (q * nstrips))
    extra = (nx - base * nstrips) // q
    x0s = [s * base + q * min(s, extra) for s in range(nstrips)]
    widths = [base + (q if s < extra else 0) for s in range(nstrips)]
    assert x0s[-1] + widths[-1] == nx
    strip_of = np.concatenate([np.full(w, s) for s, w in enumerate(widths)])
    seg = min(seg_h, ny)
    nseg = -(-ny // seg)
    seg_of = np.arange(ny) // seg
    req = []
    for g in range(nseg):
        ya, yb = g * seg, min(ny, (g + 1) * seg)
        for s in range(nstrips):
            X, Y = np.meshgrid(np.arange(x0s[s] - 4, x0s[s] - 4 + cols), np.arange(ya - 4, yb + 5))
            ok = (X >= -4) & (X < nx + 4)
            if walls:
                ok &= (Y >= 0) & (Y < ny)
            X, Y = X[ok] % nx, Y[ok] % ny
            req.append(set((strip_of[X] + nstrips * seg_of[Y]).tolist()))
    return req


CASES = [
    # (precision, nx, ny, walls, nstrips, seg_h)
    (LB_FP32, 4096, 1024, 1, 36, 52),       # the benchmark's tiling
    (LB_FP32, 4096, 1024, 1, 39, 24),
    (LB_BF16DEV, 4096, 1024, 1, 35, 32),
    (LB_FP32, 512, 256, 0, 5, 40),          # periodic: images in x and y
    (LB_FP32, 512, 256, 1, 8, 3),           # segments shorter than the halo
    (LB_FP32, 300, 130, 0, 3, 1),
    (LB_FP16DEV, 304, 130, 0, 3, 7),
    (LB_FP32, 8, 8, 0, 1, 2),               # lattice narrower than a window
    (LB_FP32, 8, 8, 1, 1, 8),
    (LB_BF16DEV, 16, 9, 0, 1, 4),
    (LB_FP32, 128, 64, 1, 16, 5),           # many narrow strips
    (LB_BF16DEV, 256, 100, 0, 16, 13),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "_".join(str(v) for v in c))
def test_lists_cover_every_read_in_both_directions(case):
    prec, nx, ny, walls, nstrips, seg_h = case
    ofs, idx = lb_sweep_dependencies(prec, nx, ny, walls, nstrips, seg_h)
    req = _required(*case)
    assert len(ofs) == len(req) + 1 and ofs[0] == 0 and ofs[-1] == len(idx)
    deps = [set(idx[ofs[t]:ofs[t + 1]].tolist()) for t in range(len(req))]
    for t, r in enumerate(req):
        assert t in deps[t]
        assert r <= deps[t], (t, sorted(r - deps[t]))
        for w in r:
            assert t in deps[w], (t, w)
    # the lists are symmetric and sorted without repeats
    for t, d in enumerate(deps):
        assert all(t in deps[u] for u in d)
        lst = idx[ofs[t]:ofs[t + 1]]
        assert np.all(np.diff(lst) > 0)


def test_lattices_and_tilings_the_sweep_does_not_take_are_refused():
    for args in ((LB_FP32, 4094, 64, 0, 36, 16),     # nx not a multiple of the quantum
                 (LB_BF16DEV, 4092, 64, 0, 36, 16),
                 (LB_FP32, 4096, 64, 0, 35, 16),     # fewer strips than the window allows
                 (LB_FP32, 4096, 64, 0, 600, 16),    # strips narrower than twice the quantum
                 (LB_FP32, 4096, 64, 0, 36, 0),      # no rows per segment
                 (LB_FP32, 4096, 4, 0, 36, 4)):      # too few rows for the sweep
        with pytest.raises(LBError):
            lb_sweep_dependencies(*args)
