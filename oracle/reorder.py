"""Row and column permutations that expose a banded structure (Sec. 4.3), in plain Python.
Test infrastructure only: imported by the tests, never by the library.

Sec. 4.3 asks for a column permutation P_c (fewer fill-ins, narrower band) and a row
permutation P_r that together make P_r A P_c "as banded as possible", so that the banded
solver of Sec. 4.4 applies; it names no algorithm.  Reading used here (and by the library):

  P_c  reverse Cuthill-McKee on the column graph of A (columns adjacent when a row holds
       both, i.e. the graph of A^T A): while columns are unvisited, start a breadth-first
       search at the unvisited column of least degree (ties: lower index); a visited column's
       unvisited neighbours are appended in order of (degree, index); the visit order,
       reversed, is the new column order.
  P_r  rows in order of (first column, last column) under P_c, ties by row index (stable);
       an empty row sorts last.

Result: col_perm[k] = original column at new position k, row_perm[k] = original row at new
position k, row_start[k] = first new column of that row (cols for an empty row), and the band
width w = max over rows of (last - first + 1) (0 without non-zeros): row k of P_r A P_c lies
in columns row_start[k] .. row_start[k] + w - 1.

Pins (tests/test_oracle_reorder.py): a hand-worked example (5 rows, 4 columns) written out in that test,
banded patterns with scrambled rows and columns get their band width back, the permutations
are permutations, every row lies in its band, and rows are sorted by their starts.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def column_graph(cols: int, rows_cols):
    """Adjacency sets of the column graph: rows_cols[i] = the columns of row i."""
    adj = [set() for _ in range(cols)]
    for rc in rows_cols:
        for a in rc:
            for b in rc:
                if a != b:
                    adj[a].add(b)
    return adj


def reverse_cuthill_mckee(cols: int, rows_cols) -> list:
    adj = column_graph(cols, rows_cols)
    deg = [len(a) for a in adj]
    visited = [False] * cols
    order = []
    while len(order) < cols:
        start = min((c for c in range(cols) if not visited[c]), key=lambda c: (deg[c], c))
        visited[start] = True
        queue = deque([start])
        while queue:
            c = queue.popleft()
            order.append(c)
            for nb in sorted((x for x in adj[c] if not visited[x]), key=lambda x: (deg[x], x)):
                visited[nb] = True
                queue.append(nb)
    return order[::-1]


def band_order(rows: int, cols: int, row_ptr, col_idx):
    """P_c, P_r, row starts and band width of the pattern given in CSR form."""
    rows_cols = [sorted(set(int(c) for c in col_idx[row_ptr[i]:row_ptr[i + 1]])) for i in range(rows)]
    col_perm = reverse_cuthill_mckee(cols, rows_cols)
    newpos = [0] * cols
    for k, c in enumerate(col_perm):
        newpos[c] = k
    first, last = [], []
    for rc in rows_cols:
        if rc:
            p = [newpos[c] for c in rc]
            first.append(min(p))
            last.append(max(p))
        else:
            first.append(cols)
            last.append(cols - 1)
    row_perm = sorted(range(rows), key=lambda i: (first[i], last[i], i))
    row_start = [first[i] for i in row_perm]
    width = max([last[i] - first[i] + 1 for i in range(rows) if rows_cols[i]], default=0)
    return (np.array(col_perm, dtype=np.int32), np.array(row_perm, dtype=np.int64),
            np.array(row_start, dtype=np.int32), int(width))
