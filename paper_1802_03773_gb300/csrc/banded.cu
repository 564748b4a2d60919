// Block-banded QR of P_r [J; lambda^(1/2) D] (Sec. 4.4 "Block banded", Sec. 4.5 / Sec. 5.2
// row interleave of the damping rows) and the banded solve, for batches of independent
// banded instances.
//
// J row i of an instance touches columns floor(i / rows_per_col) .. + w - 1 (entries past the
// last column are ignored); values are stored row-major, w per row.  The damping row of
// column j has the single value lambda^(1/2) D_j at column j.
//
// Work mapping: one warp per instance, several instances per CTA.  The warp sweeps column
// groups [c0, c0 + 8): the front holds the rows carried from the previous group (at most
// w - 1, non-zero only from column c0 on) plus the J rows and damping rows whose first column
// lies in the group; rows are appended in batches to a shared-memory front and reduced by
// Householder reflections (Sec. 2) with lanes over columns, so the front never holds more
// than (group + w - 1) + batch rows however dense the rows are.  After the last batch the
// group's R rows are final (written as windows R[j, j .. j + w - 1]) and the next w - 1 rows
// are carried.  Every Householder vector is as long as its front, never as long as the
// matrix (Sec. 4.4).  Q is not kept: the right-hand side is reflected along with the front.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "device_util.cuh"
#include "internal.h"

namespace qrkit {
namespace {

constexpr int kBG = 8;          // columns per group
constexpr int kBW = 16;         // largest band window
constexpr int kBatch = 48;      // new rows appended per front reduction
constexpr int kFCols = kBG + kBW - 1 + 1;      // front columns incl. the rhs column
constexpr int kFStride = kFCols + 1;           // padded row stride (bank spread)
constexpr int kFRows = kBG + kBW - 1 + kBatch; // kept rows + one batch
constexpr int kWarps = 4;                      // instances per CTA (float)
template <typename T> constexpr int warps_for() { return sizeof(T) == sizeof(double) ? 2 : kWarps; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

__device__ __forceinline__ void brecord(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

template <typename T>
struct BandArgs {
  int64_t num_inst;
  const int64_t* inst_cols;   // columns per instance
  const int64_t* inst_col0;   // first global column of each instance
  const int64_t* inst_row0;   // first J row of each instance
  int rows_per_col;           // implicit row starts: row i starts at floor(i / rows_per_col)
  const int64_t* row_start;   // explicit row starts, global columns, non-decreasing per instance (null: implicit)
  const int64_t* inst_rows;   // rows per instance when row_start is given
  int w;                      // band window (<= kBW)
  const T* J;                 // rows x w, row-major
  const T* b;                 // rows
  const double* D;            // global columns (may be null when !damp)
  double lam;                 // lambda (damping rows present iff lam > 0)
  T* Rw;                      // global columns x w: R[j, j + t] at Rw[j * w + t]
  T* c;                       // global columns: top of Q^T [b; 0]
  T* x;                       // global columns: solution
  double* res2;               // per instance: squared norm of the rest of Q^T [b; 0]
  int refine_steps;
  int* status;
};

// One reduction of the front F (nr rows x fc columns + rhs column fc) by Householder
// reflections, column by column; lanes over columns for the dot products and updates.
template <typename T>
__device__ __forceinline__ void front_qr(T* F, int nr, int fc, int lane) {
  const int kmax = nr < fc ? nr : fc;
  for (int k = 0; k < kmax; ++k) {
    T s = 0;
    for (int r = k + 1 + lane; r < nr; r += 32) {
      const T a = F[r * kFStride + k];
      s += a * a;
    }
    s = warp_sum(s);
    const T alpha = F[k * kFStride + k];
    const T norm = sqrt(alpha * alpha + s);
    T beta = 0, tau = 0, scale = 0;
    if (norm != T(0)) {
      beta = alpha >= T(0) ? -norm : norm;
      tau = (beta - alpha) / beta;
      scale = T(1) / (alpha - beta);
    }
    for (int r = k + 1 + lane; r < nr; r += 32) F[r * kFStride + k] *= scale;
    __syncwarp();
    const int j = k + 1 + lane;   // one lane per trailing column (incl. the rhs column fc)
    if (j <= fc) {
      T wv = F[k * kFStride + j];
      for (int r = k + 1; r < nr; ++r) wv += F[r * kFStride + k] * F[r * kFStride + j];
      wv *= tau;
      F[k * kFStride + j] -= wv;
      for (int r = k + 1; r < nr; ++r) F[r * kFStride + j] -= wv * F[r * kFStride + k];
    }
    __syncwarp();
    if (lane == 0) F[k * kFStride + k] = beta;
    for (int r = k + 1 + lane; r < nr; r += 32) F[r * kFStride + k] = T(0);
    __syncwarp();
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * kWarps)
banded_factor_solve_kernel(BandArgs<T> A) {
  constexpr int NW = warps_for<T>();   // static shared memory stays under 48 KB
  __shared__ __align__(16) T sF[NW][kFRows * kFStride];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int64_t inst = (int64_t)blockIdx.x * NW + wid;
  if (inst >= A.num_inst) return;
  T* F = sF[wid];
  const int w = A.w;
  const int64_t N = A.inst_cols[inst];
  const int64_t col0 = A.inst_col0[inst];
  const int64_t row0 = A.inst_row0[inst];
  const int64_t nrows = A.row_start ? A.inst_rows[inst] : (int64_t)A.rows_per_col * N;
  const bool damp = A.lam > 0.0;
  const double lam_half = sqrt(A.lam);
  double res2 = 0.0;
  int carried = 0;   // rows 0 .. carried-1 of F hold the carried rows (columns from c0 on)
  int64_t jr_next = 0;   // explicit starts: first row not yet consumed
  for (int e = lane; e < kFRows * kFStride; e += 32) F[e] = T(0);
  __syncwarp();
  for (int64_t c0 = 0; c0 < N; c0 += kBG) {
    const int64_t c1 = c0 + kBG < N ? c0 + kBG : N;
    const int g = (int)(c1 - c0);
    const int64_t hi = c1 + w - 1 < N ? c1 + w - 1 : N;
    const int fc = (int)(hi - c0);            // front columns; the rhs sits in column fc
    // the rhs column index changes with fc: move the carried rows' rhs into place
    // (carried rows were written with the rhs at column kFCols - 1, see below)
    for (int r = lane; r < carried; r += 32) {
      const T rhs = F[r * kFStride + (kFCols - 1)];
      F[r * kFStride + (kFCols - 1)] = T(0);
      F[r * kFStride + fc] = rhs;
    }
    __syncwarp();
    int nr = carried;
    // stream of new rows: J rows starting in [c0, c1), then the damping rows of c0 .. c1-1
    int64_t jr, jr_end;
    if (A.row_start) {
      jr = jr_next;
      jr_end = jr;
      while (jr_end < nrows && A.row_start[row0 + jr_end] - col0 < c1) ++jr_end;
      jr_next = jr_end;
    } else {
      jr = (int64_t)A.rows_per_col * c0;
      jr_end = (int64_t)A.rows_per_col * c1 < nrows ? (int64_t)A.rows_per_col * c1 : nrows;
    }
    int64_t dr = damp ? c0 : c1;
    while (jr < jr_end || dr < c1) {
      const int room = kFRows - nr;
      const int64_t take_j = jr_end - jr < room ? jr_end - jr : room;
      const int64_t take_d = (c1 - dr) < (room - take_j) ? (c1 - dr) : (room - take_j);
      // append (lanes over new rows); each row is cleared first
      for (int t = lane; t < (int)(take_j + take_d); t += 32) {
        T* row = F + (nr + t) * kFStride;
        for (int q = 0; q < kFStride; ++q) row[q] = T(0);
        if (t < take_j) {
          const int64_t i = jr + t;
          const int64_t start = A.row_start ? A.row_start[row0 + i] - col0 : i / A.rows_per_col;
          const T* src = A.J + (row0 + i) * w;
          for (int q = 0; q < w; ++q) {
            const int64_t col = start + q;
            if (col >= c0 && col < N) row[col - c0] = src[q];
          }
          row[fc] = A.b[row0 + i];
        } else {
          const int64_t j = dr + (t - take_j);
          row[j - c0] = (T)(lam_half * A.D[col0 + j]);
        }
      }
      __syncwarp();
      nr += (int)(take_j + take_d);
      jr += take_j;
      dr += take_d;
      front_qr(F, nr, fc, lane);
      // rows beyond the triangle are now zero: their rhs is residual
      double part = 0.0;
      for (int r = fc + lane; r < nr; r += 32) {
        const double v = (double)F[r * kFStride + fc];
        part += v * v;
        F[r * kFStride + fc] = T(0);
      }
      res2 += warp_sum(part);
      nr = nr < fc ? nr : fc;
      __syncwarp();
    }
    if (nr < g) {
      brecord(A.status, QRKIT_ESINGULAR);   // fewer rows than columns in this group
    }
    // final R rows of the group
    for (int i = lane; i < g; i += 32) {
      const int64_t gj = col0 + c0 + i;
      for (int t = 0; t < w; ++t) {
        const int colf = i + t;
        A.Rw[gj * w + t] = (colf < fc && i < nr) ? F[i * kFStride + colf] : T(0);
      }
      A.c[gj] = i < nr ? F[i * kFStride + fc] : T(0);
    }
    __syncwarp();
    // carry rows g .. nr-1, shifted left by g columns; rhs parked in column kFCols - 1
    const int nc = nr - g > 0 ? nr - g : 0;
    if (c1 < N) {
      // ascending rows: the source row g + r is read before any later row overwrites it
      for (int r = 0; r < nc; ++r) {
        const T* src = F + (g + r) * kFStride;
        T v = T(0);
        if (lane < kFCols - 1 && lane + g < fc) v = src[lane + g];
        const T rhs = src[fc];
        __syncwarp();
        T* dst = F + r * kFStride;
        if (lane < kFCols - 1) dst[lane] = v;
        if (lane == 0) dst[kFCols - 1] = rhs;
        __syncwarp();
      }
      // clear the rows above the carried ones
      for (int e = nc * kFStride + lane; e < kFRows * kFStride; e += 32) F[e] = T(0);
      __syncwarp();
    }
    carried = nc;
  }
  if (lane == 0) A.res2[inst] = res2;
  // back-substitution R x = c on the banded R (one lane; the recurrence is sequential)
  if (lane == 0) {
    bool bad = false;
    for (int64_t j = N - 1; j >= 0; --j) {
      const int64_t gj = col0 + j;
      T s = A.c[gj];
      for (int t = 1; t < w && j + t < N; ++t) s -= A.Rw[gj * w + t] * A.x[gj + t];
      const T rjj = A.Rw[gj * w];
      if (rjj == T(0)) bad = true;
      A.x[gj] = s / rjj;
    }
    if (bad) brecord(A.status, QRKIT_ESINGULAR);
  }
}

// ---- refinement for float instances: r = b - J x in double (one lane per row), then
// g = J^T r - lambda D^2 x (one lane per column), then x += R^{-1} R^{-T} g by banded
// triangular solves; one warp per instance ----
__global__ void __launch_bounds__(32 * kWarps)
banded_refine_kernel(BandArgs<float> A, double* rbuf, double* gbuf, float* hbuf) {
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int64_t inst = (int64_t)blockIdx.x * kWarps + wid;
  if (inst >= A.num_inst) return;
  const int w = A.w;
  const int rpc = A.rows_per_col;
  const int64_t N = A.inst_cols[inst];
  const int64_t col0 = A.inst_col0[inst];
  const int64_t row0 = A.inst_row0[inst];
  const int64_t nrows = (int64_t)rpc * N;
  for (int64_t i = lane; i < nrows; i += 32) {
    const int64_t s = i / rpc;
    const float* row = A.J + (row0 + i) * w;
    double r = (double)A.b[row0 + i];
    for (int t = 0; t < w && s + t < N; ++t) r -= (double)row[t] * (double)A.x[col0 + s + t];
    rbuf[row0 + i] = r;
  }
  __syncwarp();
  for (int64_t j = lane; j < N; j += 32) {
    double acc = 0.0;
    const int64_t s_lo = j - w + 1 > 0 ? j - w + 1 : 0;
    for (int64_t s = s_lo; s <= j; ++s)
      for (int q = 0; q < rpc; ++q) {
        const int64_t i = s * rpc + q;
        if (i >= nrows) break;
        acc += (double)A.J[(row0 + i) * w + (j - s)] * rbuf[row0 + i];
      }
    if (A.lam > 0.0) {
      const double d = A.D[col0 + j];
      acc -= A.lam * d * d * (double)A.x[col0 + j];
    }
    gbuf[col0 + j] = acc;
  }
  __syncwarp();
  if (lane == 0) {
    // R^T h = g (forward): h_j = (g_j - sum_{t=1}^{w-1} R[j-t, j] h_{j-t}) / R[j, j]
    for (int64_t j = 0; j < N; ++j) {
      const int64_t gj = col0 + j;
      float s = (float)gbuf[gj];
      for (int t = 1; t < w && j - t >= 0; ++t) s -= A.Rw[(gj - t) * w + t] * hbuf[gj - t];
      hbuf[gj] = s / A.Rw[gj * w];
    }
    // R dx = h (backward), x += dx
    for (int64_t j = N - 1; j >= 0; --j) {
      const int64_t gj = col0 + j;
      float s = hbuf[gj];
      for (int t = 1; t < w && j + t < N; ++t) s -= A.Rw[gj * w + t] * hbuf[gj + t];
      hbuf[gj] = s / A.Rw[gj * w];
    }
    for (int64_t j = 0; j < N; ++j) A.x[col0 + j] += hbuf[col0 + j];
  }
}

// R^T h = g (transpose = 1: forward with R^T) or R x = h (backward) for the banded R of each
// instance (windows Rw by global column); one thread per instance, the recurrences are
// sequential.  In place on v (global columns).
template <typename T>
__global__ void band_tri_solve_kernel(int64_t num_inst, const int64_t* inst, const T* Rw, int w, T* v,
                                      int transpose) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= num_inst) return;
  const int64_t n = inst[k], c0 = inst[num_inst + k];
  const T* R = Rw + c0 * w;
  T* x = v + c0;
  if (transpose) {
    for (int64_t j = 0; j < n; ++j) {
      T s = x[j];
      for (int t = 1; t < w && j - t >= 0; ++t) s -= R[(j - t) * w + t] * x[j - t];
      x[j] = s / R[j * w];
    }
  } else {
    for (int64_t j = n - 1; j >= 0; --j) {
      T s = x[j];
      for (int t = 1; t < w && j + t < n; ++t) s -= R[j * w + t] * x[j + t];
      x[j] = s / R[j * w];
    }
  }
}

__global__ void band_colnorm_kernel(const float* Jf, const double* Jd, const int64_t* inst_cols,
                                    const int64_t* inst_col0, const int64_t* inst_row0,
                                    int64_t num_inst, int rpc, int w, double* D) {
  // one thread per global column: rows touching column j start in [j - w + 1, j]
  const int64_t total = inst_col0[num_inst - 1] + inst_cols[num_inst - 1];
  const int64_t gj = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gj >= total) return;
  int64_t lo = 0, hi = num_inst - 1;
  while (lo < hi) {   // instance of column gj
    const int64_t mid = (lo + hi + 1) / 2;
    if (inst_col0[mid] <= gj) lo = mid; else hi = mid - 1;
  }
  const int64_t inst = lo, j = gj - inst_col0[inst], N = inst_cols[inst];
  const int64_t nrows = (int64_t)rpc * N;
  double acc = 0.0;
  const int64_t s_lo = j - w + 1 > 0 ? j - w + 1 : 0;
  for (int64_t s = s_lo; s <= j; ++s)
    for (int q = 0; q < rpc; ++q) {
      const int64_t i = s * rpc + q;
      if (i >= nrows) break;
      const int64_t e = (inst_row0[inst] + i) * w + (j - s);
      const double v = Jf ? (double)Jf[e] : Jd[e];
      acc += v * v;
    }
  const double d = sqrt(acc);
  D[gj] = d == 0.0 ? 1.0 : d;
}

// Column norms for float J, in two phases per CTA of kColNormCols consecutive global columns.
// Rows come in groups of rows_per_col per column (group g = rows rpc g .. rpc g + rpc - 1,
// all starting at column g), so column j's entries are entry t of groups j - t, t < w.
// Phase 1: one thread per group sums the squares of its rpc rows per entry t (contiguous
// rpc x w floats, vector loads) into shared memory; phase 2: one thread per column adds its w
// diagonal partial sums (in double) from groups of its own instance.
constexpr int kColNormCols = 256;
__global__ void __launch_bounds__(kColNormCols) band_colnorm_f32_kernel(const float* J, int64_t total_cols,
                                                                        const int64_t* inst_col0, int64_t num_inst,
                                                                        int rpc, int w, int vec, double* D) {
  __shared__ float S[(kColNormCols + kBW - 1) * (kBW + 1)];
  const int stride = w + 1;   // odd row stride: consecutive columns hit different banks
  const int64_t j0 = (int64_t)blockIdx.x * kColNormCols;
  for (int gg = threadIdx.x; gg < kColNormCols + w - 1; gg += kColNormCols) {
    const int64_t g = j0 - (w - 1) + gg;
    float acc[kBW];
#pragma unroll
    for (int t = 0; t < kBW; ++t) acc[t] = 0.f;
    if (g >= 0 && g < total_cols) {
      const float* rows = J + g * rpc * w;
      if (vec) {   // rpc w a multiple of 4 and J 16-byte aligned
        const float4* r4 = reinterpret_cast<const float4*>(rows);
        for (int e = 0; e < rpc * w / 4; ++e) {
          const float4 v = r4[e];
          const int t0 = (4 * e) % w;   // w is a multiple of 4 or divides 4 here
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float x = u == 0 ? v.x : (u == 1 ? v.y : (u == 2 ? v.z : v.w));
            const int t = (t0 + u) % w;
#pragma unroll
            for (int tt = 0; tt < kBW; ++tt)
              if (tt == t) acc[tt] += x * x;
          }
        }
      } else {
        for (int q = 0; q < rpc; ++q)
#pragma unroll
          for (int t = 0; t < kBW; ++t)
            if (t < w) acc[t] += rows[q * w + t] * rows[q * w + t];
      }
    }
#pragma unroll
    for (int t = 0; t < kBW; ++t)
      if (t < w) S[gg * stride + t] = acc[t];
  }
  __syncthreads();
  const int64_t gj = j0 + threadIdx.x;
  if (gj >= total_cols) return;
  int64_t lo = 0, hi = num_inst - 1;
  while (lo < hi) {   // instance of column gj
    const int64_t mid = (lo + hi + 1) / 2;
    if (inst_col0[mid] <= gj) lo = mid; else hi = mid - 1;
  }
  const int64_t j = gj - inst_col0[lo];
  double sum = 0.0;
  for (int t = 0; t < w && t <= j; ++t) sum += (double)S[(threadIdx.x + w - 1 - t) * stride + t];
  const double d = sqrt(sum);
  D[gj] = d == 0.0 ? 1.0 : d;
}

// Refinement pieces of the parallel path for float J: the residual r = b - J x of each row as
// an unevaluated float pair (rh + rl, Dot2: error-free products and sums, the accuracy of a
// double residual without GB300's slow FP64 pipe), stored in place of a double r ...
__global__ void band_resid_f32_kernel(const float* J, const float* b, const float* x, const int64_t* inst_cols,
                                      const int64_t* inst_col0, const int64_t* inst_row0, int64_t num_inst,
                                      int64_t total_rows, int rpc, int w, float2* r) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= total_rows) return;
  int64_t lo = 0, hi = num_inst - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (inst_row0[mid] <= gi) lo = mid; else hi = mid - 1;
  }
  const int64_t i = gi - inst_row0[lo], N = inst_cols[lo], c0 = inst_col0[lo];
  const int64_t s = i / rpc;
  const float* row = J + gi * w;
  float sh = b[gi], sl = 0.f;
  for (int t = 0; t < w && s + t < N; ++t) {
    const float a = row[t], xj = -x[c0 + s + t];
    const float pr = __fmul_rn(a, xj);
    const float pe = __fmaf_rn(a, xj, -pr);
    float tt, e;
    dev::two_sum(sh, pr, tt, e);
    sh = tt;
    sl = __fadd_rn(sl, __fadd_rn(e, pe));
  }
  r[gi] = make_float2(sh, sl);
}

// ... and g = J^T r - lambda D^2 x per column, in the two phases of the column norms: per row
// group the Dot2 sums over its rows for each diagonal t (pairs in shared memory), then per
// column the compensated sum of its w diagonal pairs; g in double.
__global__ void __launch_bounds__(kColNormCols) band_g_f32_kernel(const float* J, const float* x, const float2* r,
                                                                  const double* D, double lam, int64_t total_cols,
                                                                  const int64_t* inst_col0, int64_t num_inst, int rpc,
                                                                  int w, double* g) {
  __shared__ float2 S[(kColNormCols + kBW - 1) * (kBW + 1)];
  const int stride = w + 1;
  const int64_t j0 = (int64_t)blockIdx.x * kColNormCols;
  for (int gg = threadIdx.x; gg < kColNormCols + w - 1; gg += kColNormCols) {
    const int64_t grp = j0 - (w - 1) + gg;
    float hs[kBW], hc[kBW];
#pragma unroll
    for (int t = 0; t < kBW; ++t) hs[t] = hc[t] = 0.f;
    if (grp >= 0 && grp < total_cols) {
      for (int q = 0; q < rpc; ++q) {
        const int64_t row = grp * rpc + q;
        const float2 rr = r[row];
        const float* jr = J + row * w;
#pragma unroll
        for (int t = 0; t < kBW; ++t) {
          if (t < w) {
            const float a = jr[t];
            const float pr = __fmul_rn(a, rr.x);
            float pe = __fmaf_rn(a, rr.x, -pr);
            pe = __fmaf_rn(a, rr.y, pe);
            float tt, e;
            dev::two_sum(hs[t], pr, tt, e);
            hs[t] = tt;
            hc[t] = __fadd_rn(hc[t], __fadd_rn(e, pe));
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < kBW; ++t)
      if (t < w) S[gg * stride + t] = make_float2(hs[t], hc[t]);
  }
  __syncthreads();
  const int64_t gj = j0 + threadIdx.x;
  if (gj >= total_cols) return;
  int64_t lo = 0, hi = num_inst - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (inst_col0[mid] <= gj) lo = mid; else hi = mid - 1;
  }
  const int64_t j = gj - inst_col0[lo];
  float s = 0.f, c = 0.f;
  for (int t = 0; t < w && t <= j; ++t) {
    const float2 v = S[(threadIdx.x + w - 1 - t) * stride + t];
    float tt, e;
    dev::two_sum(s, v.x, tt, e);
    s = tt;
    c = __fadd_rn(c, __fadd_rn(e, v.y));
  }
  double acc = (double)s + (double)c;
  if (lam > 0.0) acc -= lam * D[gj] * D[gj] * (double)x[gj];
  g[gj] = acc;
}

// Refinement pieces of the parallel path for double J (float J takes the Dot2 kernels
// above), one thread per row / per column: r = b - J x in double, then
// g_j = sum_i J_ij r_i - lambda D_j^2 x_j.
template <typename T>
__global__ void band_resid_kernel(const T* J, const T* b, const T* x, const int64_t* inst_cols,
                                  const int64_t* inst_col0, const int64_t* inst_row0, int64_t num_inst,
                                  int64_t total_rows, int rpc, int w, double* r) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= total_rows) return;
  int64_t lo = 0, hi = num_inst - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (inst_row0[mid] <= gi) lo = mid; else hi = mid - 1;
  }
  const int64_t i = gi - inst_row0[lo], N = inst_cols[lo], c0 = inst_col0[lo];
  const int64_t s = i / rpc;
  const T* row = J + gi * w;
  double acc = (double)b[gi];
  for (int t = 0; t < w && s + t < N; ++t) acc -= (double)row[t] * (double)x[c0 + s + t];
  r[gi] = acc;
}

template <typename T>
__global__ void band_g_kernel(const T* J, const T* x, const double* r, const double* D, double lam,
                              const int64_t* inst_cols, const int64_t* inst_col0, const int64_t* inst_row0,
                              int64_t num_inst, int64_t total_cols, int rpc, int w, double* g) {
  const int64_t gj = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gj >= total_cols) return;
  int64_t lo = 0, hi = num_inst - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (inst_col0[mid] <= gj) lo = mid; else hi = mid - 1;
  }
  const int64_t j = gj - inst_col0[lo], N = inst_cols[lo], r0 = inst_row0[lo];
  const int64_t nrows = (int64_t)rpc * N;
  double acc = 0.0;
  const int64_t s_lo = j - w + 1 > 0 ? j - w + 1 : 0;
  for (int64_t s = s_lo; s <= j; ++s)
    for (int q = 0; q < rpc; ++q) {
      const int64_t i = s * rpc + q;
      if (i >= nrows) break;
      acc += (double)J[(r0 + i) * w + (j - s)] * r[r0 + i];
    }
  if (lam > 0.0) acc -= lam * D[gj] * D[gj] * (double)x[gj];
  g[gj] = acc;
}

// Rows with explicit starts (global columns, non-decreasing within an instance): the rows of
// instance k are row0[k] .. row0[k] + rows[k] - 1, and column j is touched by the rows whose
// start lies in [j - w + 1, j], a contiguous run found by binary search.  inst: 4 x num_inst
// (cols, col0, row0, rows).
__device__ __forceinline__ int64_t inst_of_col(const int64_t* inst, int64_t num_inst, int64_t gj) {
  const int64_t* col0 = inst + num_inst;
  int64_t lo = 0, hi = num_inst - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (col0[mid] <= gj) lo = mid; else hi = mid - 1;
  }
  return lo;
}
// First row of [r0, r1) whose start is >= v (starts sorted in that range).
__device__ __forceinline__ int64_t first_row_at(const int64_t* start, int64_t r0, int64_t r1, int64_t v) {
  while (r0 < r1) {
    const int64_t mid = r0 + (r1 - r0) / 2;
    if (start[mid] < v) r0 = mid + 1; else r1 = mid;
  }
  return r0;
}

// D_j = || column j of J || (zero -> 1), one thread per global column, rows in order.
template <typename T>
__global__ void band_colnorm_explicit_kernel(const T* J, const int64_t* start, const int64_t* inst,
                                             int64_t num_inst, int64_t total_cols, int w, double* D) {
  const int64_t gj = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gj >= total_cols) return;
  const int64_t k = inst_of_col(inst, num_inst, gj);
  const int64_t r0 = inst[2 * num_inst + k], r1 = r0 + inst[3 * num_inst + k];
  double acc = 0.0;
  for (int64_t i = first_row_at(start, r0, r1, gj - w + 1); i < r1 && start[i] <= gj; ++i) {
    const double v = (double)J[i * w + (gj - start[i])];
    acc += v * v;
  }
  const double d = sqrt(acc);
  D[gj] = d == 0.0 ? 1.0 : d;
}

// r_i = b_i - sum_t J_it x_{start_i + t} in double (entries past the instance's last column are
// ignored), one thread per row.
template <typename T>
__global__ void band_resid_explicit_kernel(const T* J, const T* b, const T* x, const int64_t* start,
                                           const int64_t* inst, int64_t num_inst, int64_t total_rows, int w,
                                           double* r) {
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= total_rows) return;
  const int64_t* row0 = inst + 2 * num_inst;
  int64_t lo = 0, hi = num_inst - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (row0[mid] <= gi) lo = mid; else hi = mid - 1;
  }
  const int64_t end = inst[num_inst + lo] + inst[lo];   // one past the instance's last column
  double acc = (double)b[gi];
  for (int t = 0; t < w && start[gi] + t < end; ++t) acc -= (double)J[gi * w + t] * (double)x[start[gi] + t];
  r[gi] = acc;
}

// g_j = sum_i J_ij r_i - lambda D_j^2 x_j, one thread per global column, rows in order.
template <typename T>
__global__ void band_g_explicit_kernel(const T* J, const T* x, const double* r, const double* D, double lam,
                                       const int64_t* start, const int64_t* inst, int64_t num_inst,
                                       int64_t total_cols, int w, double* g) {
  const int64_t gj = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gj >= total_cols) return;
  const int64_t k = inst_of_col(inst, num_inst, gj);
  const int64_t r0 = inst[2 * num_inst + k], r1 = r0 + inst[3 * num_inst + k];
  double acc = 0.0;
  for (int64_t i = first_row_at(start, r0, r1, gj - w + 1); i < r1 && start[i] <= gj; ++i)
    acc += (double)J[i * w + (gj - start[i])] * r[i];
  if (lam > 0.0) acc -= lam * D[gj] * D[gj] * (double)x[gj];
  g[gj] = acc;
}

template <typename T>
__global__ void band_axpy_kernel(T* x, const T* d, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += d[i];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

qrkit_status banded_plan(qrkit_ctx* ctx, const qrkit_structure* s) {
  Plan& P = ctx->plan;
  if (s->rows_per_col < 1) return fail(ctx, QRKIT_EINVAL, "rows_per_col must be >= 1");
  if (s->band_window < 1 || s->band_window > kBW)
    return fail(ctx, QRKIT_EUNSUPPORTED, "band_window must be in [1, 16]");
  std::vector<int64_t> cols;
  if (s->num_blocks > 0 && s->instance_cols) {
    cols.assign(s->instance_cols, s->instance_cols + s->num_blocks);
  } else {
    if (s->cols < 1) return fail(ctx, QRKIT_EINVAL, "cols must be >= 1");
    cols.assign(1, s->cols);
  }
  for (size_t i = 0; i < cols.size(); ++i)
    if (cols[i] < 1) return fail(ctx, QRKIT_EINVAL, "instance " + std::to_string(i) + " has no columns");
  // rows per instance: rows_per_col * cols, or given with explicit row starts
  const bool expl = s->band_row_start != nullptr;
  std::vector<int64_t> nrows(cols.size());
  for (size_t i = 0; i < cols.size(); ++i) {
    if (!expl) {
      nrows[i] = cols[i] * s->rows_per_col;
    } else if (s->instance_rows) {
      nrows[i] = s->instance_rows[i];
    } else if (cols.size() == 1) {
      nrows[i] = s->rows;
    } else {
      return fail(ctx, QRKIT_EINVAL, "instance_rows is required with band_row_start and a batch of instances");
    }
    if (nrows[i] < 0) return fail(ctx, QRKIT_EINVAL, "instance " + std::to_string(i) + " has a negative row count");
  }
  std::vector<int64_t> c0(cols.size()), r0(cols.size());
  int64_t cc = 0, rr = 0;
  for (size_t i = 0; i < cols.size(); ++i) {
    c0[i] = cc;
    r0[i] = rr;
    cc += cols[i];
    rr += nrows[i];
  }
  std::vector<int64_t> gstart;
  if (expl) {
    gstart.resize((size_t)rr);
    for (size_t i = 0; i < cols.size(); ++i)
      for (int64_t k = 0; k < nrows[i]; ++k) {
        const int64_t v = s->band_row_start[r0[i] + k];
        if (v < 0 || v >= cols[i])
          return fail(ctx, QRKIT_EINVAL, "row " + std::to_string(r0[i] + k) + " starts outside its instance");
        if (k > 0 && v < s->band_row_start[r0[i] + k - 1])
          return fail(ctx, QRKIT_EINVAL, "row starts must not decrease within an instance (row " +
                                             std::to_string(r0[i] + k) + ")");
        gstart[(size_t)(r0[i] + k)] = c0[i] + v;
      }
  }
  Band& B = ctx->band;
  if (s->band_solver < QRKIT_BAND_AUTO || s->band_solver > QRKIT_BAND_PARALLEL)
    return fail(ctx, QRKIT_EINVAL, "unknown band_solver");
  if (s->band_solver == QRKIT_BAND_PARALLEL && s->band_window > 8)
    return fail(ctx, QRKIT_EUNSUPPORTED, "the parallel banded QR needs band_window <= 8");
  B.parallel = s->band_solver == QRKIT_BAND_PARALLEL || (s->band_solver == QRKIT_BAND_AUTO && s->band_window <= 8);
  B.num_inst = (int64_t)cols.size();
  B.total_cols = cc;
  B.total_rows = rr;
  B.rows_per_col = s->rows_per_col;
  B.w = s->band_window;
  B.explicit_starts = expl;
  qrkit_status st;
  auto up = [&](DevBuf& buf, const std::vector<int64_t>& v) -> qrkit_status {
    qrkit_status r = ensure(ctx, buf, v.size() * sizeof(int64_t), "band plan");
    if (r != QRKIT_OK) return r;
    QRKIT_CUDA_TRY(ctx, cudaMemcpy(buf.ptr, v.data(), v.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    return QRKIT_OK;
  };
  if ((st = up(B.d_cols, cols)) != QRKIT_OK) return st;
  if ((st = up(B.d_col0, c0)) != QRKIT_OK) return st;
  if ((st = up(B.d_row0, r0)) != QRKIT_OK) return st;
  if (expl) {
    std::vector<int64_t> inst(cols);
    inst.insert(inst.end(), c0.begin(), c0.end());
    inst.insert(inst.end(), r0.begin(), r0.end());
    inst.insert(inst.end(), nrows.begin(), nrows.end());
    if ((st = up(B.d_inst, inst)) != QRKIT_OK) return st;
    if ((st = up(B.d_rows, nrows)) != QRKIT_OK) return st;
    if (rr > 0 && (st = up(B.d_start, gstart)) != QRKIT_OK) return st;
  }
  const size_t es = elem_size(ctx);
  if ((st = ensure(ctx, B.Rw, (size_t)cc * B.w * es, "banded R")) != QRKIT_OK) return st;
  if ((st = ensure(ctx, B.c, (size_t)cc * es, "banded c")) != QRKIT_OK) return st;
  if ((st = ensure(ctx, B.D, (size_t)cc * sizeof(double), "banded D")) != QRKIT_OK) return st;
  if ((st = ensure(ctx, B.res2, (size_t)B.num_inst * sizeof(double), "banded residual")) != QRKIT_OK) return st;
  if (B.parallel) {
    if ((st = cr_build(ctx, B.cr, cols, c0, r0, nrows)) != QRKIT_OK) return st;
  }
  if (B.parallel || expl) {
    if ((st = ensure(ctx, B.g, (size_t)cc * sizeof(double), "banded g")) != QRKIT_OK) return st;
    if ((st = ensure(ctx, B.h, (size_t)cc * es, "banded h")) != QRKIT_OK) return st;
    if ((st = ensure(ctx, B.r, (size_t)std::max<int64_t>(rr, 1) * sizeof(double), "banded r")) != QRKIT_OK) return st;
  }
  P.s = *s;
  P.s.block_rows = nullptr;
  P.s.block_cols = nullptr;
  P.s.window_start = nullptr;
  P.s.instance_cols = nullptr;
  P.s.band_row_start = nullptr;
  P.s.instance_rows = nullptr;
  P.valid = true;
  return QRKIT_OK;
}

template <typename T>
__global__ void band_g_to_t_kernel(const double* g, T* h, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) h[i] = (T)g[i];
}

static qrkit_status widen_or_narrow_g(qrkit_ctx* ctx, const double* g, void* h, int64_t n) {
  if (ctx->precision == QRKIT_FP64)
    band_g_to_t_kernel<double><<<nblk(n, 256), 256, 0, ctx->stream>>>(g, (double*)h, n);
  else
    band_g_to_t_kernel<float><<<nblk(n, 256), 256, 0, ctx->stream>>>(g, (float*)h, n);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

template <typename T>
static qrkit_status banded_run(qrkit_ctx* ctx, const void* J, const void* b, const void* Dext,
                               double lambda, void* p, int refine_steps) {
  Band& B = ctx->band;
  cudaStream_t st = ctx->stream;
  const int64_t* dcols = (const int64_t*)B.d_cols.ptr;
  const int64_t* dc0 = (const int64_t*)B.d_col0.ptr;
  const int64_t* dr0 = (const int64_t*)B.d_row0.ptr;
  double* D = (double*)B.D.ptr;
  if (lambda > 0.0) {
    if (Dext) {
      if (sizeof(T) == sizeof(double)) {
        QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(D, Dext, (size_t)B.total_cols * sizeof(double),
                                            cudaMemcpyDeviceToDevice, st));
      } else {
        qrkit_status rc = widen_to_double(ctx, (const float*)Dext, D, B.total_cols);
        if (rc != QRKIT_OK) return rc;
      }
    } else if (B.explicit_starts) {
      band_colnorm_explicit_kernel<T><<<nblk(B.total_cols, 256), 256, 0, st>>>(
          (const T*)J, (const int64_t*)B.d_start.ptr, (const int64_t*)B.d_inst.ptr, B.num_inst, B.total_cols, B.w,
          D);
      ctx->launches += 1;
      QRKIT_CUDA_TRY(ctx, cudaGetLastError());
    } else {
      if (sizeof(T) == sizeof(float)) {
        const int rw = B.rows_per_col * B.w;
        const int vec = (rw % 4 == 0) && (B.w % 4 == 0 || 4 % B.w == 0) &&
                        (reinterpret_cast<uintptr_t>(J) & 15) == 0;
        band_colnorm_f32_kernel<<<nblk(B.total_cols, kColNormCols), kColNormCols, 0, st>>>(
            (const float*)J, B.total_cols, dc0, B.num_inst, B.rows_per_col, B.w, vec, D);
      } else {
        band_colnorm_kernel<<<nblk(B.total_cols, 256), 256, 0, st>>>(nullptr, (const double*)J, dcols, dc0, dr0,
                                                                    B.num_inst, B.rows_per_col, B.w, D);
      }
      ctx->launches += 1;
      QRKIT_CUDA_TRY(ctx, cudaGetLastError());
    }
  }
  if (B.explicit_starts) {
    // rows with explicit starts (e.g. the row and column permutations of Sec. 4.3 applied):
    // the parallel QR or the sweep, then refinement with a double residual
    const int64_t* gs = (const int64_t*)B.d_start.ptr;
    const int64_t* inst = (const int64_t*)B.d_inst.ptr;
    qrkit_status rc;
    if (B.parallel) {
      rc = cr_solve(ctx, *B.cr, gs, 1, B.w, J, b, D, lambda, p, (double*)B.res2.ptr);
    } else {
      rc = banded_explicit_solve(ctx, B.num_inst, inst, J, gs, b, B.w, D, lambda, B.Rw.ptr, B.c.ptr, p,
                                 (double*)B.res2.ptr);
    }
    if (rc != QRKIT_OK) return rc;
    for (int it = 0; it < refine_steps; ++it) {
      band_resid_explicit_kernel<T><<<nblk(std::max<int64_t>(B.total_rows, 1), 256), 256, 0, st>>>(
          (const T*)J, (const T*)b, (const T*)p, gs, inst, B.num_inst, B.total_rows, B.w, (double*)B.r.ptr);
      band_g_explicit_kernel<T><<<nblk(B.total_cols, 256), 256, 0, st>>>(
          (const T*)J, (const T*)p, (const double*)B.r.ptr, D, lambda, gs, inst, B.num_inst, B.total_cols, B.w,
          (double*)B.g.ptr);
      ctx->launches += 2;
      QRKIT_CUDA_TRY(ctx, cudaGetLastError());
      if (B.parallel) {
        if ((rc = cr_normal_solve(ctx, *B.cr, (const double*)B.g.ptr, B.h.ptr)) != QRKIT_OK) return rc;
      } else {
        if ((rc = widen_or_narrow_g(ctx, (const double*)B.g.ptr, B.h.ptr, B.total_cols)) != QRKIT_OK) return rc;
        if ((rc = banded_tri_solve(ctx, B.num_inst, inst, B.Rw.ptr, B.w, B.h.ptr, true)) != QRKIT_OK) return rc;
        if ((rc = banded_tri_solve(ctx, B.num_inst, inst, B.Rw.ptr, B.w, B.h.ptr, false)) != QRKIT_OK) return rc;
      }
      band_axpy_kernel<T><<<nblk(B.total_cols, 256), 256, 0, st>>>((T*)p, (const T*)B.h.ptr, B.total_cols);
      ctx->launches += 1;
      QRKIT_CUDA_TRY(ctx, cudaGetLastError());
    }
    return QRKIT_OK;
  }
  if (B.parallel) {
    qrkit_status rc = cr_solve(ctx, *B.cr, nullptr, B.rows_per_col, B.w, J, b, D, lambda, p,
                               (double*)B.res2.ptr);
    if (rc != QRKIT_OK) return rc;
    for (int it = 0; it < refine_steps; ++it) {
      if (sizeof(T) == sizeof(float)) {
        band_resid_f32_kernel<<<nblk(B.total_rows, 256), 256, 0, st>>>(
            (const float*)J, (const float*)b, (const float*)p, dcols, dc0, dr0, B.num_inst, B.total_rows,
            B.rows_per_col, B.w, (float2*)B.r.ptr);
        band_g_f32_kernel<<<nblk(B.total_cols, kColNormCols), kColNormCols, 0, st>>>(
            (const float*)J, (const float*)p, (const float2*)B.r.ptr, D, lambda, B.total_cols, dc0, B.num_inst,
            B.rows_per_col, B.w, (double*)B.g.ptr);
      } else {
        band_resid_kernel<T><<<nblk(B.total_rows, 256), 256, 0, st>>>(
            (const T*)J, (const T*)b, (const T*)p, dcols, dc0, dr0, B.num_inst, B.total_rows, B.rows_per_col, B.w,
            (double*)B.r.ptr);
        band_g_kernel<T><<<nblk(B.total_cols, 256), 256, 0, st>>>(
            (const T*)J, (const T*)p, (const double*)B.r.ptr, D, lambda, dcols, dc0, dr0, B.num_inst, B.total_cols,
            B.rows_per_col, B.w, (double*)B.g.ptr);
      }
      ctx->launches += 2;
      QRKIT_CUDA_TRY(ctx, cudaGetLastError());
      if ((rc = cr_normal_solve(ctx, *B.cr, (const double*)B.g.ptr, B.h.ptr)) != QRKIT_OK) return rc;
      band_axpy_kernel<T><<<nblk(B.total_cols, 256), 256, 0, st>>>((T*)p, (const T*)B.h.ptr, B.total_cols);
      ctx->launches += 1;
      QRKIT_CUDA_TRY(ctx, cudaGetLastError());
    }
    return QRKIT_OK;
  }
  BandArgs<T> A;
  A.num_inst = B.num_inst;
  A.inst_cols = dcols;
  A.inst_col0 = dc0;
  A.inst_row0 = dr0;
  A.rows_per_col = B.rows_per_col;
  A.row_start = nullptr;
  A.inst_rows = nullptr;
  A.w = B.w;
  A.J = (const T*)J;
  A.b = (const T*)b;
  A.D = D;
  A.lam = lambda;
  A.Rw = (T*)B.Rw.ptr;
  A.c = (T*)B.c.ptr;
  A.x = (T*)p;
  A.res2 = (double*)B.res2.ptr;
  A.refine_steps = refine_steps;
  A.status = ctx->d_status;
  banded_factor_solve_kernel<T><<<nblk(B.num_inst, warps_for<T>()), 32 * warps_for<T>(), 0, st>>>(A);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  if constexpr (sizeof(T) == sizeof(float)) {
    if (refine_steps > 0) {
      qrkit_status rc;
      if ((rc = ensure(ctx, B.g, (size_t)B.total_cols * sizeof(double), "banded g")) != QRKIT_OK) return rc;
      if ((rc = ensure(ctx, B.h, (size_t)B.total_cols * sizeof(float), "banded h")) != QRKIT_OK) return rc;
      if ((rc = ensure(ctx, B.r, (size_t)B.total_rows * sizeof(double), "banded r")) != QRKIT_OK) return rc;
      for (int it = 0; it < refine_steps; ++it) {
        banded_refine_kernel<<<nblk(B.num_inst, kWarps), 32 * kWarps, 0, st>>>(
            A, (double*)B.r.ptr, (double*)B.g.ptr, (float*)B.h.ptr);
        ctx->launches += 1;
        QRKIT_CUDA_TRY(ctx, cudaGetLastError());
      }
    }
  }
  return QRKIT_OK;
}

// Factor + solve banded instances whose rows carry explicit starts (the reduced blocks of a
// windowed block-angular structure, one instance per segment of S): rows x w values, damping
// rows lambda^(1/2) D_j (D in double, global columns) when lambda > 0.  Rw, c, x, D are
// indexed by global column (instance col0 + j); rows, starts and rhs by global row.
template <typename T>
static qrkit_status explicit_run(qrkit_ctx* ctx, int64_t num_inst, const int64_t* inst, const T* rows,
                                 const int64_t* starts, const T* rhs, int w, const double* D,
                                 double lambda, T* Rw, T* c, T* x, double* res2) {
  BandArgs<T> A;
  A.num_inst = num_inst;
  A.inst_cols = inst;
  A.inst_col0 = inst + num_inst;
  A.inst_row0 = inst + 2 * num_inst;
  A.inst_rows = inst + 3 * num_inst;
  A.rows_per_col = 1;
  A.row_start = starts;
  A.w = w;
  A.J = rows;
  A.b = rhs;
  A.D = D;
  A.lam = lambda;
  A.Rw = Rw;
  A.c = c;
  A.x = x;
  A.res2 = res2;
  A.refine_steps = 0;
  A.status = ctx->d_status;
  banded_factor_solve_kernel<T><<<nblk(num_inst, warps_for<T>()), 32 * warps_for<T>(), 0, ctx->stream>>>(A);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

qrkit_status banded_explicit_solve(qrkit_ctx* ctx, int64_t num_inst, const int64_t* inst,
                                   const void* rows, const int64_t* starts, const void* rhs, int w,
                                   const double* D, double lambda, void* Rw, void* c, void* x,
                                   double* res2) {
  if (w < 1 || w > kBW) return fail(ctx, QRKIT_EUNSUPPORTED, "reduced band window must be in [1, 16]");
  if (num_inst < 1) return QRKIT_OK;
  if (ctx->precision == QRKIT_FP64)
    return explicit_run<double>(ctx, num_inst, inst, (const double*)rows, starts, (const double*)rhs, w,
                                D, lambda, (double*)Rw, (double*)c, (double*)x, res2);
  return explicit_run<float>(ctx, num_inst, inst, (const float*)rows, starts, (const float*)rhs, w, D,
                             lambda, (float*)Rw, (float*)c, (float*)x, res2);
}

qrkit_status banded_tri_solve(qrkit_ctx* ctx, int64_t num_inst, const int64_t* inst, const void* Rw,
                              int w, void* v, bool transpose) {
  if (num_inst < 1) return QRKIT_OK;
  if (ctx->precision == QRKIT_FP64)
    band_tri_solve_kernel<double><<<nblk(num_inst, 64), 64, 0, ctx->stream>>>(
        num_inst, inst, (const double*)Rw, w, (double*)v, transpose ? 1 : 0);
  else
    band_tri_solve_kernel<float><<<nblk(num_inst, 64), 64, 0, ctx->stream>>>(
        num_inst, inst, (const float*)Rw, w, (float*)v, transpose ? 1 : 0);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

qrkit_status banded_factor_solve(qrkit_ctx* ctx, const void* J, const void* b, const void* D,
                                 double lambda, void* p, int refine_steps) {
  if (ctx->precision == QRKIT_FP64) return banded_run<double>(ctx, J, b, D, lambda, p, 0);
  const int steps = ctx->precision == QRKIT_FP32 ? 0 : refine_steps;
  return banded_run<float>(ctx, J, b, D, lambda, p, steps);
}

qrkit_status banded_get_factor(qrkit_ctx* ctx, void* Rw_out, void* c_out, double* res2_out) {
  Band& B = ctx->band;
  const size_t es = elem_size(ctx);
  if (B.parallel && (Rw_out || c_out))
    return fail(ctx, QRKIT_EUNSUPPORTED, "R windows and Q^T b exist only for the sweep algorithm");
  if (Rw_out)
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(Rw_out, B.Rw.ptr, (size_t)B.total_cols * B.w * es,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
  if (c_out)
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(c_out, B.c.ptr, (size_t)B.total_cols * es,
                                        cudaMemcpyDeviceToDevice, ctx->stream));
  if (res2_out)
    QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(res2_out, B.res2.ptr, (size_t)B.num_inst * sizeof(double),
                                        cudaMemcpyDeviceToHost, ctx->stream));
  return QRKIT_OK;
}

void release_band(Band& B) {
  release(B.d_cols); release(B.d_col0); release(B.d_row0); release(B.Rw); release(B.c);
  release(B.d_inst); release(B.d_rows); release(B.d_start);
  release(B.D); release(B.res2); release(B.g); release(B.h); release(B.r);
  release_cr(B.cr);
  B = Band();
}

}  // namespace qrkit
