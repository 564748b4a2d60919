// Normal equations by Cholesky, the comparison path of Sec. 1 / Sec. 6.1 ("QRkit+Chol"):
// (J^T J + lambda D^2) p = J^T b, Eq. (1), formed and solved in the context's precision
// (float for both float modes), whose error grows with cond(A)^2 where the QR path's grows
// with cond(A).
//
// Block-angular structure J = [blkdiag(J_i) | S]: the block unknowns are eliminated first
// (Schur complement onto the shared block):
//   G_i = J_i^T J_i + lambda D_i^2 = L_i L_i^T,  y_i = L_i^{-1} J_i^T b_i,  W_i = L_i^{-1} J_i^T S_i
//   A_S = sum_i (S_i^T S_i - W_i^T W_i) + lambda D_S^2,  r_S = sum_i (S_i^T b_i - W_i^T y_i)
//   A_S = U^T U (banded with half-bandwidth w - 1 for windows, one band per segment; dense
//   for a dense S),  p_S = U^{-1} U^{-T} r_S,  p_i = L_i^{-T} (y_i - W_i p_S[window]).
// The windowed sums are accumulated with atomics (order-dependent rounding); the dense sums
// are formed by one thread per entry in a fixed order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "internal.h"

namespace qrkit {
namespace {

constexpr int kNM = 8;    // largest block width
constexpr int kNW = 16;   // largest window

__device__ __forceinline__ void n_record(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

template <typename T>
struct NormalArgs {
  ComposedView<T> V;
  const T* b;
  const double* D;
  double lam;
  T* L;    // per block column c: row c of L_i (kNM values) at L[c * kNM]
  T* W;    // per block column c: row c of W_i (w values) at W[c * w]
  T* y;    // per block column
  T* As;   // WINDOW: A_S band, A_S(j, j + t) at As[j * w + t]; DENSE: s x s
  T* rs;   // s
  int* status;
};

// Per block: Cholesky of G_i, y_i, W_i and (windows) the Schur contributions.
template <typename T>
__global__ void normal_block_kernel(NormalArgs<T> A) {
  const ComposedView<T>& V = A.V;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.K) return;
  const int n = V.n[i], m = V.m[i];
  const int64_t c0 = V.col_off[i], r0 = V.row_off[i];
  const T* J = V.J + V.val_off[i];
  const T* b = A.b + r0;
  T L[kNM * kNM];
  T y[kNM];
  // G (lower) and J^T b
  for (int a = 0; a < m; ++a) {
    T r = 0;
    for (int q = 0; q < n; ++q) r += J[a * n + q] * b[q];
    y[a] = r;
    for (int c = 0; c <= a; ++c) {
      T g = 0;
      for (int q = 0; q < n; ++q) g += J[a * n + q] * J[c * n + q];
      if (a == c) g += (T)(A.lam * A.D[c0 + a] * A.D[c0 + a]);
      L[a * kNM + c] = g;
    }
  }
  // Cholesky (column algorithm) and y = L^{-1} J^T b
  bool bad = false;
  for (int j = 0; j < m; ++j) {
    T d = L[j * kNM + j];
    for (int k = 0; k < j; ++k) d -= L[j * kNM + k] * L[j * kNM + k];
    if (!(d > T(0))) {
      bad = true;
      d = T(1);
    }
    const T ljj = sqrt(d);
    L[j * kNM + j] = ljj;
    for (int a = j + 1; a < m; ++a) {
      T v = L[a * kNM + j];
      for (int k = 0; k < j; ++k) v -= L[a * kNM + k] * L[j * kNM + k];
      L[a * kNM + j] = v / ljj;
    }
  }
  if (bad) n_record(A.status, QRKIT_ESINGULAR);
  for (int a = 0; a < m; ++a) {
    T v = y[a];
    for (int k = 0; k < a; ++k) v -= L[a * kNM + k] * y[k];
    y[a] = v / L[a * kNM + a];
  }
  for (int a = 0; a < m; ++a) {
    for (int c = 0; c < kNM; ++c) A.L[(c0 + a) * kNM + c] = c <= a ? L[a * kNM + c] : T(0);
    A.y[c0 + a] = y[a];
  }
  if (V.coupled == QRKIT_COUPLED_NONE) return;
  const int w = V.w;
  if (V.coupled == QRKIT_COUPLED_DENSE) {
    // W_i = L^{-1} J_i^T S_i, one shared column at a time
    for (int c = 0; c < w; ++c) {
      T col[kNM];
      for (int a = 0; a < m; ++a) {
        T v = 0;
        for (int q = 0; q < n; ++q) v += J[a * n + q] * V.S[(int64_t)c * V.rows + r0 + q];
        for (int k = 0; k < a; ++k) v -= L[a * kNM + k] * col[k];
        col[a] = v / L[a * kNM + a];
        A.W[(c0 + a) * w + c] = col[a];
      }
    }
    return;
  }
  // windows: S_i is n x w column-major
  const T* S = V.S + r0 * w;
  const int64_t st = V.start[i];
  T Wl[kNM * kNW];
  for (int c = 0; c < w; ++c)
    for (int a = 0; a < m; ++a) {
      T v = 0;
      for (int q = 0; q < n; ++q) v += J[a * n + q] * S[c * n + q];
      for (int k = 0; k < a; ++k) v -= L[a * kNM + k] * Wl[k * kNW + c];
      Wl[a * kNW + c] = v / L[a * kNM + a];
      A.W[(c0 + a) * w + c] = Wl[a * kNW + c];
    }
  for (int c1 = 0; c1 < w; ++c1) {
    if (st + c1 >= V.s) break;
    T r = 0;
    for (int q = 0; q < n; ++q) r += S[c1 * n + q] * b[q];
    for (int a = 0; a < m; ++a) r -= Wl[a * kNW + c1] * y[a];
    if (r != T(0)) atomicAdd(A.rs + st + c1, r);
    for (int c2 = c1; c2 < w && st + c2 < V.s; ++c2) {
      T g = 0;
      for (int q = 0; q < n; ++q) g += S[c1 * n + q] * S[c2 * n + q];
      for (int a = 0; a < m; ++a) g -= Wl[a * kNW + c1] * Wl[a * kNW + c2];
      if (g != T(0)) atomicAdd(A.As + (st + c1) * w + (c2 - c1), g);
    }
  }
}

// Dense S: one thread per entry (c1 <= c2) of A_S and per entry of r_S, fixed summation order.
template <typename T>
__global__ void normal_dense_schur_kernel(NormalArgs<T> A) {
  const ComposedView<T>& V = A.V;
  const int s = V.s;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)s * s + s) return;
  if (e >= (int64_t)s * s) {
    const int c = (int)(e - (int64_t)s * s);
    T r = 0;
    for (int64_t q = 0; q < V.rows; ++q) r += V.S[(int64_t)c * V.rows + q] * A.b[q];
    for (int64_t a = 0; a < V.nb; ++a) r -= A.W[a * s + c] * A.y[a];
    A.rs[c] = r;
    return;
  }
  const int c1 = (int)(e / s), c2 = (int)(e % s);
  if (c2 < c1) return;
  T g = 0;
  for (int64_t q = 0; q < V.rows; ++q) g += V.S[(int64_t)c1 * V.rows + q] * V.S[(int64_t)c2 * V.rows + q];
  for (int64_t a = 0; a < V.nb; ++a) g -= A.W[a * s + c1] * A.W[a * s + c2];
  if (c1 == c2) g += (T)(A.lam * A.D[V.nb + c1] * A.D[V.nb + c1]);
  A.As[(int64_t)c1 * s + c2] = g;
  A.As[(int64_t)c2 * s + c1] = g;
}

// Banded A_S of each segment: add lambda D^2, factor A = U^T U in place (U(j, j + t) at
// As[j * w + t]), then U^T z = r, U p = z.  One warp per segment (lanes over the trailing
// update of a column); the recurrences run column by column.
template <typename T>
__global__ void normal_band_kernel(NormalArgs<T> A, const int64_t* seg, int64_t nseg, T* pS) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= nseg) return;
  const int64_t N = seg[k], c0 = seg[nseg + k];
  const int w = A.V.w;
  T* As = A.As + c0 * w;
  for (int64_t j = lane; j < N; j += 32)
    As[j * w] += (T)(A.lam * A.D[A.V.nb + c0 + j] * A.D[A.V.nb + c0 + j]);
  __syncwarp();
  bool bad = false;
  for (int64_t j = 0; j < N; ++j) {
    T d = As[j * w];
    if (!(d > T(0))) {
      bad = true;
      d = T(1);
    }
    const T u = sqrt(d);
    __syncwarp();
    if (lane == 0) As[j * w] = u;
    if (lane >= 1 && lane < w && j + lane < N) As[j * w + lane] /= u;
    __syncwarp();
    // trailing update: pairs (t1, t2), 1 <= t1 <= t2 < w
    for (int pr = lane; pr < w * w; pr += 32) {
      const int t1 = pr / w, t2 = pr % w;
      if (t1 >= 1 && t2 >= t1 && j + t2 < N) As[(j + t1) * w + (t2 - t1)] -= As[j * w + t1] * As[j * w + t2];
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (bad) n_record(A.status, QRKIT_ESINGULAR);
    T* x = pS + c0;
    const T* r = A.rs + c0;
    for (int64_t j = 0; j < N; ++j) {
      T v = r[j];
      for (int t = 1; t < w && j - t >= 0; ++t) v -= As[(j - t) * w + t] * x[j - t];
      x[j] = v / As[j * w];
    }
    for (int64_t j = N - 1; j >= 0; --j) {
      T v = x[j];
      for (int t = 1; t < w && j + t < N; ++t) v -= As[j * w + t] * x[j + t];
      x[j] = v / As[j * w];
    }
  }
}

// Dense A_S (s <= 64): one CTA, the column Cholesky in shared memory, then the two solves.
template <typename T>
__global__ void normal_dense_kernel(NormalArgs<T> A, T* pS) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* G = reinterpret_cast<T*>(smem_raw);
  const int s = A.V.s;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) G[e] = A.As[e];
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    if (threadIdx.x == 0) {
      T d = G[j * s + j];
      if (!(d > T(0))) {
        n_record(A.status, QRKIT_ESINGULAR);
        d = T(1);
      }
      G[j * s + j] = sqrt(d);
    }
    __syncthreads();
    const T u = G[j * s + j];
    for (int a = j + 1 + threadIdx.x; a < s; a += blockDim.x) G[a * s + j] /= u;
    __syncthreads();
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
      const int a = e / s, c = e % s;
      if (a > j && c > j && c <= a) G[a * s + c] -= G[a * s + j] * G[c * s + j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int a = 0; a < s; ++a) {
      T v = A.rs[a];
      for (int k = 0; k < a; ++k) v -= G[a * s + k] * pS[k];
      pS[a] = v / G[a * s + a];
    }
    for (int a = s - 1; a >= 0; --a) {
      T v = pS[a];
      for (int k = a + 1; k < s; ++k) v -= G[k * s + a] * pS[k];
      pS[a] = v / G[a * s + a];
    }
  }
}

// p_i = L_i^{-T} (y_i - W_i p_S[window]).
template <typename T>
__global__ void normal_backsub_kernel(NormalArgs<T> A, T* p) {
  const ComposedView<T>& V = A.V;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V.K) return;
  const int m = V.m[i];
  const int64_t c0 = V.col_off[i];
  T z[kNM];
  for (int a = 0; a < m; ++a) {
    T v = A.y[c0 + a];
    if (V.coupled != QRKIT_COUPLED_NONE) {
      const int64_t st = V.coupled == QRKIT_COUPLED_WINDOW ? V.start[i] : 0;
      const T* pS = p + V.nb;
      for (int c = 0; c < V.w; ++c)
        if (st + c < V.s) v -= A.W[(c0 + a) * V.w + c] * pS[st + c];
    }
    z[a] = v;
  }
  for (int a = m - 1; a >= 0; --a) {
    T v = z[a];
    for (int k = a + 1; k < m; ++k) v -= A.L[(c0 + k) * kNM + a] * z[k];
    z[a] = v / A.L[(c0 + a) * kNM + a];
  }
  for (int a = 0; a < m; ++a) p[c0 + a] = z[a];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T>
qrkit_status normal_typed(qrkit_ctx* ctx, const void* J, const void* S, const void* b, const void* Dext,
                          double lambda, void* p) {
  Plan& P = ctx->plan;
  Composed& C = ctx->comp;
  cudaStream_t st = ctx->stream;
  const int64_t N = P.cols + P.s.shared_cols;
  const int s = (int)P.s.shared_cols;
  const int w = P.s.coupled_kind == QRKIT_COUPLED_DENSE ? s : P.s.window;
  const size_t es = sizeof(T);
  qrkit_status rc;
  if ((rc = ensure(ctx, C.nrm_D, (size_t)N * sizeof(double), "normal D")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.nrm_L, (size_t)P.cols * kNM * es, "normal L")) != QRKIT_OK) return rc;
  if ((rc = ensure(ctx, C.nrm_y, (size_t)P.cols * es, "normal y")) != QRKIT_OK) return rc;
  if (P.s.coupled_kind != QRKIT_COUPLED_NONE) {
    if ((rc = ensure(ctx, C.nrm_W, (size_t)P.cols * w * es, "normal W")) != QRKIT_OK) return rc;
    const size_t as = P.s.coupled_kind == QRKIT_COUPLED_DENSE ? (size_t)s * s : (size_t)s * w;
    if ((rc = ensure(ctx, C.nrm_As, as * es, "normal A_S")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, C.nrm_rs, (size_t)s * es, "normal r_S")) != QRKIT_OK) return rc;
  }
  ComposedView<T> V = composed_view<T>(ctx, J, S);
  double* D = (double*)C.nrm_D.ptr;
  if (Dext) {
    if (sizeof(T) == sizeof(double)) {
      QRKIT_CUDA_TRY(ctx, cudaMemcpyAsync(D, Dext, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else if ((rc = widen_to_double(ctx, (const float*)Dext, D, N)) != QRKIT_OK) {
      return rc;
    }
  } else if ((rc = composed_column_norms(ctx, J, S, D)) != QRKIT_OK) {
    return rc;
  }
  NormalArgs<T> A;
  A.V = V;
  A.b = (const T*)b;
  A.D = D;
  A.lam = lambda;
  A.L = (T*)C.nrm_L.ptr;
  A.W = (T*)C.nrm_W.ptr;
  A.y = (T*)C.nrm_y.ptr;
  A.As = (T*)C.nrm_As.ptr;
  A.rs = (T*)C.nrm_rs.ptr;
  A.status = ctx->d_status;
  T* x = (T*)p;
  if (P.s.coupled_kind == QRKIT_COUPLED_WINDOW) {
    QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(A.As, 0, (size_t)s * w * es, st));
    QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(A.rs, 0, (size_t)s * es, st));
  }
  normal_block_kernel<T><<<nblk(P.K, 64), 64, 0, st>>>(A);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  if (P.s.coupled_kind == QRKIT_COUPLED_DENSE) {
    normal_dense_schur_kernel<T><<<nblk((int64_t)s * s + s, 128), 128, 0, st>>>(A);
    normal_dense_kernel<T><<<1, 256, (size_t)s * s * es, st>>>(A, x + P.cols);
    ctx->launches += 2;
    QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  } else if (P.s.coupled_kind == QRKIT_COUPLED_WINDOW) {
    const int64_t nseg = (int64_t)P.seg_cols.size();
    std::vector<int64_t> tab(P.seg_cols);
    tab.insert(tab.end(), P.seg_col0.begin(), P.seg_col0.end() - 1);
    if ((rc = ensure(ctx, C.nrm_seg, tab.size() * sizeof(int64_t), "normal segments")) != QRKIT_OK) return rc;
    QRKIT_CUDA_TRY(ctx, cudaMemcpy(C.nrm_seg.ptr, tab.data(), tab.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    normal_band_kernel<T><<<nblk(nseg * 32, 128), 128, 0, st>>>(A, (const int64_t*)C.nrm_seg.ptr, nseg, x + P.cols);
    ctx->launches += 1;
    QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  }
  normal_backsub_kernel<T><<<nblk(P.K, 64), 64, 0, st>>>(A, x);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

}  // namespace
}  // namespace qrkit

using namespace qrkit;

extern "C" qrkit_status qrkit_normal_solve(qrkit_ctx* ctx, const void* J, const void* S, const void* b,
                                           const void* D, double lambda, void* p) {
  if (!ctx) return QRKIT_EINVAL;
  const Plan& P = ctx->plan;
  if (!P.valid || P.s.kind != QRKIT_STRUCT_BLOCKS) return fail(ctx, QRKIT_ESTATE, "qrkit_normal_solve needs a block plan");
  if (!J || !b || !p) return fail(ctx, QRKIT_EINVAL, "J, b and p are required");
  if (P.s.coupled_kind != QRKIT_COUPLED_NONE && !S) return fail(ctx, QRKIT_EINVAL, "S is required");
  if (!(lambda >= 0.0)) return fail(ctx, QRKIT_EINVAL, "lambda must be >= 0");
  if (P.max_m > kNM) return fail(ctx, QRKIT_EUNSUPPORTED, "blocks wider than 8 columns");
  if (P.s.coupled_kind == QRKIT_COUPLED_DENSE && P.s.shared_cols > 64)
    return fail(ctx, QRKIT_EUNSUPPORTED, "dense shared block wider than 64 columns");
  if (P.s.coupled_kind == QRKIT_COUPLED_WINDOW && P.s.window > kNW)
    return fail(ctx, QRKIT_EUNSUPPORTED, "window wider than 16 columns");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (ctx->precision == QRKIT_FP64) return normal_typed<double>(ctx, J, S, b, D, lambda, p);
  return normal_typed<float>(ctx, J, S, b, D, lambda, p);
}
