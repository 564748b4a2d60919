// Row and column permutations that expose a banded structure (Sec. 4.3), host code.
//
// Sec. 4.3 asks for P_c and P_r such that P_r A P_c is "as banded as possible", so that the
// banded QR of Sec. 4.4 applies to an input whose band is hidden by its numbering; it names no
// algorithm.  This takes reverse Cuthill-McKee on the column graph of A (columns adjacent when
// some row holds both: the graph of A^T A) for P_c, and orders the rows by their first and last
// column under P_c for P_r.  Exact rules (ties included), so that any two implementations agree
// to the index:
//   * while columns are unvisited, a breadth-first search starts at the unvisited column of
//     least degree (ties: lower index); a visited column's unvisited neighbours are queued in
//     order of (degree, index); the visit order, reversed, is the column order;
//   * rows sort by (first column, last column) under that order, ties by row index; an empty
//     row sorts last, with start = cols.
// Plan-time work on the host, like the rest of a structure plan.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.h"

extern "C" qrkit_status qrkit_band_order(int64_t rows, int64_t cols, const int64_t* row_ptr, const int32_t* col_idx,
                                         int32_t* col_perm, int64_t* row_perm, int32_t* row_start,
                                         int32_t* width) {
  if (rows < 0 || cols < 1 || cols > (int64_t)INT32_MAX || !row_ptr || !col_perm || !width) return QRKIT_EINVAL;
  if (rows > 0 && (!row_perm || !row_start)) return QRKIT_EINVAL;
  if (row_ptr[0] != 0) return QRKIT_EINVAL;
  for (int64_t i = 0; i < rows; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return QRKIT_EINVAL;
  const int64_t nnz = row_ptr[rows];
  if (nnz > 0 && !col_idx) return QRKIT_EINVAL;
  for (int64_t e = 0; e < nnz; ++e)
    if (col_idx[e] < 0 || col_idx[e] >= cols) return QRKIT_EINVAL;
  const int32_t N = (int32_t)cols;

  // rows of each column (CSC of the pattern, duplicates kept)
  std::vector<int64_t> cptr((size_t)N + 1, 0);
  for (int64_t e = 0; e < nnz; ++e) cptr[(size_t)col_idx[e] + 1] += 1;
  for (int32_t c = 0; c < N; ++c) cptr[(size_t)c + 1] += cptr[(size_t)c];
  std::vector<int64_t> crow((size_t)nnz);
  {
    std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
    for (int64_t i = 0; i < rows; ++i)
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) crow[(size_t)fill[(size_t)col_idx[e]]++] = i;
  }
  // column graph: distinct neighbours of every column
  std::vector<int64_t> aptr((size_t)N + 1, 0);
  std::vector<int32_t> adj;
  std::vector<int32_t> stamp((size_t)N, -1);
  for (int32_t c = 0; c < N; ++c) {
    stamp[(size_t)c] = c;
    for (int64_t k = cptr[(size_t)c]; k < cptr[(size_t)c + 1]; ++k) {
      const int64_t i = crow[(size_t)k];
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const int32_t b = col_idx[e];
        if (stamp[(size_t)b] != c) {
          stamp[(size_t)b] = c;
          adj.push_back(b);
        }
      }
    }
    aptr[(size_t)c + 1] = (int64_t)adj.size();
  }
  std::vector<int64_t> deg((size_t)N);
  for (int32_t c = 0; c < N; ++c) deg[(size_t)c] = aptr[(size_t)c + 1] - aptr[(size_t)c];
  auto before = [&](int32_t a, int32_t b) {
    return deg[(size_t)a] != deg[(size_t)b] ? deg[(size_t)a] < deg[(size_t)b] : a < b;
  };

  // Cuthill-McKee visit order, component by component
  std::vector<int32_t> by_degree((size_t)N);
  for (int32_t c = 0; c < N; ++c) by_degree[(size_t)c] = c;
  std::sort(by_degree.begin(), by_degree.end(), before);
  std::vector<char> visited((size_t)N, 0);
  std::vector<int32_t> order;
  order.reserve((size_t)N);
  std::vector<int32_t> nbrs;
  size_t next_start = 0;
  while ((int64_t)order.size() < N) {
    while (visited[(size_t)by_degree[next_start]]) ++next_start;
    const int32_t s = by_degree[next_start];
    visited[(size_t)s] = 1;
    size_t head = order.size();
    order.push_back(s);
    while (head < order.size()) {
      const int32_t c = order[head++];
      nbrs.clear();
      for (int64_t k = aptr[(size_t)c]; k < aptr[(size_t)c + 1]; ++k)
        if (!visited[(size_t)adj[(size_t)k]]) nbrs.push_back(adj[(size_t)k]);
      std::sort(nbrs.begin(), nbrs.end(), before);
      for (int32_t b : nbrs) {
        visited[(size_t)b] = 1;
        order.push_back(b);
      }
    }
  }
  // reversed: new position k holds column order[N - 1 - k]
  std::vector<int32_t> newpos((size_t)N);
  for (int32_t k = 0; k < N; ++k) {
    col_perm[k] = order[(size_t)(N - 1 - k)];
    newpos[(size_t)col_perm[k]] = k;
  }

  // rows by (first, last) under the new column order
  std::vector<int32_t> first((size_t)rows), last((size_t)rows);
  int32_t w = 0;
  for (int64_t i = 0; i < rows; ++i) {
    int32_t lo = N, hi = N - 1;
    if (row_ptr[i + 1] > row_ptr[i]) {
      lo = N;
      hi = -1;
      for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const int32_t p = newpos[(size_t)col_idx[e]];
        lo = std::min(lo, p);
        hi = std::max(hi, p);
      }
      w = std::max(w, hi - lo + 1);
    }
    first[(size_t)i] = lo;
    last[(size_t)i] = hi;
  }
  std::vector<int64_t> idx((size_t)rows);
  for (int64_t i = 0; i < rows; ++i) idx[(size_t)i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
    if (first[(size_t)a] != first[(size_t)b]) return first[(size_t)a] < first[(size_t)b];
    return last[(size_t)a] < last[(size_t)b];
  });
  for (int64_t k = 0; k < rows; ++k) {
    row_perm[k] = idx[(size_t)k];
    row_start[k] = first[(size_t)idx[(size_t)k]];
  }
  *width = w;
  return QRKIT_OK;
}
