// Row permutation P_r of the reduced shared block of a windowed structure (Sec. 4.3): the
// reduced rows (the bottoms of Q_i^T [S_i; 0], one run per block) are sorted by their first
// shared column, ties kept in reduced-row order, so that every independent segment of S
// becomes one banded matrix whose rows appear in leading-column order (Sec. 4.4 input).
//
// Segmented stable counting sort, deterministic:
//   count   one warp per chunk of rows: per-chunk histogram over the segment's columns
//   scan    bin-major, chunk-minor exclusive offsets (in place), in three parallel passes: one
//           thread per (segment, bin) turns the bin's chunk counts into chunk-minor prefixes
//           and records the bin total; one CTA per segment scans its bin totals; one thread
//           per (segment, bin) adds the bin's base to its chunk entries
//   scatter one warp per chunk, its rows in order: rank among equal keys from
//           __match_any_sync, the chunk's running offsets advanced by the key's leader lane;
//           writes the sorted rows (values, starts) and both directions of the permutation.
// A start outside its segment is recorded as QRKIT_EINVAL and clamped into the segment so
// that every index stays in bounds.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace qrkit {
namespace {

constexpr int kScanThreads = 1024;

__device__ __forceinline__ void rs_record(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ int64_t clamp_key(int64_t start, int64_t col0, int64_t cols, int* status) {
  int64_t k = start - col0;
  if (k < 0 || k >= cols) {
    rs_record(status, QRKIT_EINVAL);
    k = k < 0 ? 0 : cols - 1;
  }
  return k;
}

__global__ void rsort_count_kernel(RowSortTables t, const int64_t* Xstart, int* hist, int* status) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= t.num_chunks) return;
  const int64_t row0 = t.chunk_row0[c], rows = t.chunk_rows[c];
  const int64_t col0 = t.chunk_col0[c], cols = t.chunk_cols[c];
  int* h = hist + t.chunk_hoff[c];
  for (int64_t r = lane; r < rows; r += 32) {
    const int64_t k = clamp_key(Xstart[row0 + r], col0, cols, status);
    atomicAdd(h + k, 1);
  }
}

constexpr int kBinThreads = 256;

// Pass 1 of the scan: bin b of segment blockIdx.x; chunk-minor exclusive prefixes in place,
// the bin's total to tot (indexed by global shared column).
__global__ void __launch_bounds__(kBinThreads) rsort_bin_prefix_kernel(RowSortTables t, int* hist, int* tot) {
  const int64_t seg = blockIdx.x;
  const int64_t c0 = t.seg_chunk0[seg], c1 = t.seg_chunk0[seg + 1];
  if (c0 == c1) return;
  const int64_t b = (int64_t)blockIdx.y * kBinThreads + threadIdx.x;
  if (b >= t.chunk_cols[c0]) return;
  int running = 0;
  for (int64_t c = c0; c < c1; ++c) {
    int* e = hist + t.chunk_hoff[c] + b;
    const int v = *e;
    *e = running;
    running += v;
  }
  tot[t.chunk_col0[c0] + b] = running;
}

// Pass 2: exclusive scan of a segment's bin totals (one CTA per segment), in place.
__global__ void __launch_bounds__(kScanThreads) rsort_bin_scan_kernel(RowSortTables t, int* tot) {
  __shared__ int warp_tot[kScanThreads / 32];
  __shared__ int carry_s;
  const int64_t seg = blockIdx.x;
  const int64_t c0 = t.seg_chunk0[seg], c1 = t.seg_chunk0[seg + 1];
  if (c0 == c1) return;
  const int64_t cols = t.chunk_cols[c0];
  int* tt = tot + t.chunk_col0[c0];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < cols; b0 += kScanThreads) {
    const int64_t b = b0 + threadIdx.x;
    const int v0 = b < cols ? tt[b] : 0;
    int incl = v0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int v = warp_tot[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
      }
      warp_tot[lane] = v;   // inclusive over warps
    }
    __syncthreads();
    const int carry = carry_s;
    if (b < cols) tt[b] = carry + (wid ? warp_tot[wid - 1] : 0) + incl - v0;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
  }
}

// Pass 3: the bin's base added to its chunk entries.
__global__ void __launch_bounds__(kBinThreads) rsort_bin_add_kernel(RowSortTables t, int* hist, const int* tot) {
  const int64_t seg = blockIdx.x;
  const int64_t c0 = t.seg_chunk0[seg], c1 = t.seg_chunk0[seg + 1];
  if (c0 == c1) return;
  const int64_t b = (int64_t)blockIdx.y * kBinThreads + threadIdx.x;
  if (b >= t.chunk_cols[c0]) return;
  const int base = tot[t.chunk_col0[c0] + b];
  for (int64_t c = c0; c < c1; ++c) hist[t.chunk_hoff[c] + b] += base;
}

template <typename T>
__global__ void rsort_scatter_kernel(RowSortTables t, const int64_t* Xstart, const T* Xw, int w,
                                     int* hist, int64_t* spos, int64_t* order, int64_t* Xstart_s,
                                     T* Xw_s) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= t.num_chunks) return;
  const int64_t row0 = t.chunk_row0[c], rows = t.chunk_rows[c];
  const int64_t col0 = t.chunk_col0[c], cols = t.chunk_cols[c];
  const int64_t out0 = t.chunk_out0[c];
  int* h = hist + t.chunk_hoff[c];
  for (int64_t r0 = 0; r0 < rows; r0 += 32) {
    const int64_t r = r0 + lane;
    const bool active = r < rows;
    const unsigned amask = __ballot_sync(0xffffffffu, active);
    if (active) {
      const int64_t st = Xstart[row0 + r];
      const int64_t k = clamp_key(st, col0, cols, nullptr);
      const unsigned peers = __match_any_sync(amask, (unsigned long long)k);
      const int leader = __ffs(peers) - 1;
      const int rank = __popc(peers & ((1u << lane) - 1u));
      int base = 0;
      if (lane == leader) {
        base = h[k];
        h[k] = base + __popc(peers);
      }
      base = __shfl_sync(amask, base, leader);
      const int64_t pos = out0 + base + rank;
      spos[row0 + r] = pos;
      order[pos] = row0 + r;
      Xstart_s[pos] = col0 + k;   // clamped: every start lies in its segment
      bool moved = false;
      if constexpr (sizeof(T) == 4) {
        if (w == 8) {   // a row of 8 floats: two 16-byte moves (rows are 32-byte aligned)
          const float4* src = reinterpret_cast<const float4*>(Xw + (row0 + r) * 8);
          float4* dst = reinterpret_cast<float4*>(Xw_s + pos * 8);
          const float4 v0 = src[0], v1 = src[1];
          dst[0] = v0;
          dst[1] = v1;
          moved = true;
        }
      }
      if (!moved)
        for (int q = 0; q < w; ++q) Xw_s[pos * w + q] = Xw[(row0 + r) * w + q];
    }
    __syncwarp();
  }
}

template <typename T>
__global__ void rsort_rhs_kernel(const int64_t* spos, const T* rhs, T* rhs_s, int64_t rows) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows) rhs_s[spos[r]] = rhs[r];
}

// Copy of caller-given window starts into the plan, each checked against its segment
// (block i belongs to segment k with seg_blk0[k] <= i < seg_blk0[k + 1]); a start outside
// is recorded as QRKIT_EINVAL and clamped.
__global__ void start_copy_kernel(const int32_t* in, int32_t* out, int64_t K, const int64_t* seg, int64_t nseg,
                                  int* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K) return;
  const int64_t* blk0 = seg;
  const int64_t* col0 = seg + nseg + 1;
  int64_t lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (blk0[mid] <= i) lo = mid; else hi = mid - 1;
  }
  int64_t v = in[i];
  if (v < col0[lo] || v >= col0[lo + 1]) {
    rs_record(status, QRKIT_EINVAL);
    v = v < col0[lo] ? col0[lo] : col0[lo + 1] - 1;
  }
  out[i] = (int32_t)v;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

qrkit_status window_start_copy(qrkit_ctx* ctx, const int32_t* in) {
  Plan& P = ctx->plan;
  const int64_t nseg = (int64_t)P.seg_cols.size();
  start_copy_kernel<<<nblk(P.K, 256), 256, 0, ctx->stream>>>(in, (int32_t*)P.d_start.ptr, P.K,
                                                              (const int64_t*)P.d_seg.ptr, nseg, ctx->d_status);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

qrkit_status reduced_row_sort(qrkit_ctx* ctx, const RowSortTables& t, int64_t nseg, int64_t hist_entries,
                              const int64_t* Xstart, const void* Xw, int w, int* hist, int64_t* spos,
                              int64_t* order, int64_t* Xstart_s, void* Xw_s) {
  cudaStream_t st = ctx->stream;
  if (t.num_chunks == 0) return QRKIT_OK;
  QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(hist, 0, (size_t)hist_entries * sizeof(int), st));
  rsort_count_kernel<<<nblk(t.num_chunks * 32, 128), 128, 0, st>>>(t, Xstart, hist, ctx->d_status);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  {
    // the three passes of the scan; bin totals after the histograms (indexed by shared column)
    int64_t maxcols = 1;
    for (const int64_t c : ctx->plan.seg_cols) maxcols = c > maxcols ? c : maxcols;
    int* tot = hist + hist_entries;
    const dim3 grid((unsigned)nseg, (unsigned)((maxcols + kBinThreads - 1) / kBinThreads));
    rsort_bin_prefix_kernel<<<grid, kBinThreads, 0, st>>>(t, hist, tot);
    rsort_bin_scan_kernel<<<(unsigned)nseg, kScanThreads, 0, st>>>(t, tot);
    rsort_bin_add_kernel<<<grid, kBinThreads, 0, st>>>(t, hist, tot);
    ctx->launches += 3;
    QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  }
  if (ctx->precision == QRKIT_FP64)
    rsort_scatter_kernel<double><<<nblk(t.num_chunks * 32, 128), 128, 0, st>>>(
        t, Xstart, (const double*)Xw, w, hist, spos, order, Xstart_s, (double*)Xw_s);
  else
    rsort_scatter_kernel<float><<<nblk(t.num_chunks * 32, 128), 128, 0, st>>>(
        t, Xstart, (const float*)Xw, w, hist, spos, order, Xstart_s, (float*)Xw_s);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

qrkit_status reduced_rhs_sort(qrkit_ctx* ctx, const int64_t* spos, const void* rhs, void* rhs_s, int64_t rows) {
  if (rows == 0) return QRKIT_OK;
  if (ctx->precision == QRKIT_FP64)
    rsort_rhs_kernel<double><<<nblk(rows, 256), 256, 0, ctx->stream>>>(spos, (const double*)rhs,
                                                                         (double*)rhs_s, rows);
  else
    rsort_rhs_kernel<float><<<nblk(rows, 256), 256, 0, ctx->stream>>>(spos, (const float*)rhs,
                                                                        (float*)rhs_s, rows);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

}  // namespace qrkit
