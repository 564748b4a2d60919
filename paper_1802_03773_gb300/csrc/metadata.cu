// Structure metadata of a block-angular plan, on the host (no CUDA call): the offsets of the
// packed values, the row permutation P_r of [J; lambda^(1/2) D] (Sec. 4.5 row interleave,
// Sec. 5.2) and the structural pattern of R in natural column order (block columns, then the
// shared columns), by symbolic row merging of the rows in P_r order.  These are the integer
// arrays a caller needs to read the factor, and they are defined by the structure alone.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace {

qrkit_status structure_metadata(const qrkit_structure* s, qrkit_metadata* md) {
  if (!s || !md) return QRKIT_EINVAL;
  if (s->kind != QRKIT_STRUCT_BLOCKS) return QRKIT_EUNSUPPORTED;
  const int64_t K = s->num_blocks;
  if (K < 1 || !s->block_rows || !s->block_cols) return QRKIT_EINVAL;
  const int ck = s->coupled_kind;
  if (ck != QRKIT_COUPLED_NONE && ck != QRKIT_COUPLED_DENSE && ck != QRKIT_COUPLED_WINDOW) return QRKIT_EINVAL;
  const int64_t sc = ck == QRKIT_COUPLED_NONE ? 0 : s->shared_cols;
  if (sc < 0 || (ck != QRKIT_COUPLED_NONE && sc < 1)) return QRKIT_EINVAL;
  if (ck == QRKIT_COUPLED_WINDOW && (s->window < 1 || !s->window_start)) return QRKIT_EINVAL;
  std::vector<int64_t> vo(K + 1, 0), ro(K + 1, 0), co(K + 1, 0);
  for (int64_t i = 0; i < K; ++i) {
    const int n = s->block_rows[i], m = s->block_cols[i];
    if (n < 1 || m < 1) return QRKIT_EINVAL;
    vo[i + 1] = vo[i] + (int64_t)n * m;
    ro[i + 1] = ro[i] + n;
    co[i + 1] = co[i] + m;
  }
  const int64_t M = ro[K], nb = co[K], N = nb + sc;
  // segment end (exclusive shared column) of each block's window
  std::vector<int64_t> seg_end;
  if (ck == QRKIT_COUPLED_WINDOW) {
    seg_end.assign(K, sc);
    if (s->num_segments > 1) {
      if (!s->segment_cols || !s->segment_blocks) return QRKIT_EINVAL;
      int64_t c0 = 0, b0 = 0;
      for (int64_t g = 0; g < s->num_segments; ++g) {
        if (s->segment_cols[g] < 1 || s->segment_blocks[g] < 0) return QRKIT_EINVAL;
        for (int64_t i = b0; i < b0 + s->segment_blocks[g] && i < K; ++i) seg_end[i] = c0 + s->segment_cols[g];
        c0 += s->segment_cols[g];
        b0 += s->segment_blocks[g];
      }
      if (c0 != sc || b0 != K) return QRKIT_EINVAL;
    }
    for (int64_t i = 0; i < K; ++i)
      if (s->window_start[i] < 0 || s->window_start[i] >= seg_end[i]) return QRKIT_EINVAL;
  }
  const bool damped = md->damped != 0;
  const int64_t aug = M + (damped ? N : 0);
  md->num_blocks = K;
  md->rows = M;
  md->cols = N;
  md->values = vo[K];
  md->aug_rows = aug;
  if (md->val_off) std::copy(vo.begin(), vo.end(), md->val_off);
  if (md->row_off) std::copy(ro.begin(), ro.end(), md->row_off);
  if (md->col_off) std::copy(co.begin(), co.end(), md->col_off);
  // P_r: by leading column, J rows (lead = their block's first column) before the damping row
  // of that column, then by source index
  std::vector<int64_t> order;
  order.reserve((size_t)aug);
  {
    int64_t blk = 0;
    for (int64_t j = 0; j < N; ++j) {
      if (blk < K && co[blk] == j) {
        for (int64_t r = ro[blk]; r < ro[blk + 1]; ++r) order.push_back(r);
        ++blk;
      }
      if (damped) order.push_back(M + j);
    }
  }
  if (md->row_order) std::copy(order.begin(), order.end(), md->row_order);
  if (!md->r_row_ptr && !md->r_col_idx) {
    md->r_nnz = -1;
    return QRKIT_OK;
  }
  // symbolic row merge: R row c takes the union with every row merged into it; the row goes on
  // from its next column with that union
  std::vector<int64_t> blk_of(M);
  for (int64_t i = 0; i < K; ++i)
    for (int64_t r = ro[i]; r < ro[i + 1]; ++r) blk_of[r] = i;
  auto row_cols = [&](int64_t src, std::vector<int64_t>& out) {
    out.clear();
    if (src >= M) {
      out.push_back(src - M);
      return;
    }
    const int64_t i = blk_of[src];
    for (int64_t c = co[i]; c < co[i + 1]; ++c) out.push_back(c);
    if (ck == QRKIT_COUPLED_DENSE) {
      for (int64_t c = 0; c < sc; ++c) out.push_back(nb + c);
    } else if (ck == QRKIT_COUPLED_WINDOW) {
      const int64_t a = s->window_start[i], e = std::min<int64_t>(a + s->window, seg_end[i]);
      for (int64_t c = a; c < e; ++c) out.push_back(nb + c);
    }
  };
  std::vector<std::vector<int64_t>> R((size_t)N);
  std::vector<char> has((size_t)N, 0);
  std::vector<int64_t> cur, uni;
  for (const int64_t src : order) {
    row_cols(src, cur);
    while (!cur.empty()) {
      const int64_t c = cur.front();
      if (!has[(size_t)c]) {
        R[(size_t)c] = cur;
        has[(size_t)c] = 1;
        break;
      }
      uni.clear();
      std::set_union(R[(size_t)c].begin(), R[(size_t)c].end(), cur.begin(), cur.end(), std::back_inserter(uni));
      R[(size_t)c] = uni;
      cur.assign(uni.begin() + 1, uni.end());   // uni[0] == c
    }
  }
  int64_t nnz = 0;
  if (md->r_row_ptr) md->r_row_ptr[0] = 0;
  for (int64_t c = 0; c < N; ++c) {
    nnz += (int64_t)R[(size_t)c].size();
    if (md->r_row_ptr) md->r_row_ptr[c + 1] = nnz;
  }
  md->r_nnz = nnz;
  if (md->r_col_idx) {
    if (md->r_capacity < nnz) return QRKIT_EINVAL;
    int64_t k = 0;
    for (int64_t c = 0; c < N; ++c)
      for (const int64_t x : R[(size_t)c]) md->r_col_idx[k++] = (int32_t)x;
  }
  return QRKIT_OK;
}

}  // namespace

extern "C" qrkit_status qrkit_structure_metadata(const qrkit_structure* s, qrkit_metadata* md) {
  return structure_metadata(s, md);
}
