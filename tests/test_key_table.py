"""The 2-D Hilbert keys of the CUDA path come from a four-state table (the curve of the
Skilling transform as a state machine, one level per step; `kHilbertStep2` in
paper_1805_01208_gb300/csrc/gk_bootstrap.cu).  Read as text from the source, the table is
walked here on the host and must give the oracle's key (its own level descent) for every
cell tried: random cells, the corners, single bits and cells along the diagonals."""
import os
import re

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _table():
    src = open(os.path.join(ROOT, "paper_1805_01208_gb300", "csrc", "gk_bootstrap.cu")).read()
    m = re.search(r"kHilbertStep2\[16\]\s*=\s*\{([^}]*)\}", src)
    assert m, "the step table is not in the source"
    t = [int(v) for v in m.group(1).split(",")]
    assert len(t) == 16
    return t


def _walk(t, x, y):
    key, st = 0, 0
    for lev in range(31, -1, -1):
        b = (((x >> lev) & 1) << 1) | ((y >> lev) & 1)
        v = t[st * 4 + b]
        key = (key << 2) | (v & 3)
        st = v >> 2
    return key


def test_step_table_gives_the_oracle_keys():
    t = _table()
    rng = np.random.default_rng(5)
    cells = [(0, 0), (2**32 - 1, 2**32 - 1), (0, 2**32 - 1), (2**32 - 1, 0)]
    cells += [(1 << i, 0) for i in range(32)] + [(0, 1 << i) for i in range(32)]
    cells += [(v, v) for v in rng.integers(0, 2**32, 200, dtype=np.uint64).tolist()]
    cells += [(v, 2**32 - 1 - v) for v in rng.integers(0, 2**32, 200, dtype=np.uint64).tolist()]
    cells += [tuple(c) for c in rng.integers(0, 2**32, (2000, 2), dtype=np.uint64).tolist()]
    small = rng.integers(0, 2**8, (500, 2), dtype=np.uint64).tolist()  # high levels all zero
    cells += [tuple(c) for c in small]
    for x, y in cells:
        assert _walk(t, int(x), int(y)) == oracle.hilbert_index(np.array([x, y], dtype=np.uint64), 32), (x, y)
