// Device side of the batched block-diagonal QR solve by shape-uniform warp tasks
// (Sec. 4.1 "Block diagonal", Householder QR of Sec. 2, the compute / Q^T b / R solve
// interface of Sec. 5.1).
//
// Plan (host): the blocks are taken in supertiles of consecutive blocks; inside a supertile
// they are counting-sorted by shape key (row class c = (n - 1) / 4, column count m) and cut
// into warp tasks of P = floor(32 / G) blocks of one key, G = c + 1 lanes per block.  Lane q
// of a block's group holds rows 4q .. 4q + 3 of every column in registers (rows padded to 4G
// with zeros), so every loop of a warp has the same trip count: no divergence, and no
// CTA-wide barrier anywhere.  Supertiles keep the blocks that concurrent warps touch (and the
// neighbours sharing their 32-byte sectors) close in time, so partial sectors meet in L2.
//
// Kernels (device): persistent warps, each with its own shared memory, take tasks in a grid
// stride and run a software pipeline: while task i is computed, the copies of task i + 1's
// block data, task i + 2's entries and task i + 3's header are in flight.  The block data are
// the 16-byte-aligned supersets of each block's J and b, copied into the block's slots by the
// G lanes of its group with per-lane 16-byte cp.async copies (the blocks of a task are
// scattered, 20-500 bytes each: per-thread copies, not TMA, whose operands must be
// warp-uniform and would serialise one block after another).  The group factors the block with
// Householder reflectors H = I - tau v v^T (v[0] = 1, beta = -sign(x0)||x||; norms and dot
// products are shuffle reductions over the group), applies them to b (Q^T b) and
// back-substitutes.  The first kernel writes the factor and Q^T b back to the slots and sends
// them to HBM with 16-byte vector stores (unaligned head and tail elements by plain stores);
// with refinement it also estimates each block's float error a priori and lists the blocks
// that need refinement, one list per shape key.  The second kernel takes those lists in tasks
// of the same form, reads R (from the stored factor) and the float solution of the listed
// blocks, and refines them with a compensated float residual.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "device_util.cuh"
#include "internal.h"

namespace qrkit {
namespace tasks {

using namespace dev;

constexpr float kUnitRoundoff = 5.9604645e-8f;   // 2^-24
constexpr int kMaxCols = 8;
constexpr int kTaskMaxWarps = 8;   // the kernels are compiled for at most 256 threads per CTA
#ifndef QRKIT_TASK_CTAS
#define QRKIT_TASK_CTAS 2   // resident CTAs per SM the float task kernel is compiled for
#endif
#ifndef QRKIT_REFINE_CTAS
#define QRKIT_REFINE_CTAS 2   // the refinement kernel is compiled for 128 registers a thread
#endif
constexpr int kRefineWarps = 4;   // warps per CTA of the refinement kernel (its buffers are large)

__host__ __device__ constexpr int group_lanes(int key) { return (key >> 3) + 1; }
__host__ __device__ constexpr int task_blocks(int G) { return 32 / G; }
// Shared-memory slot of one block's J (or b) in a task: the 16-byte-aligned superset of
// len bytes starting anywhere spans at most round16(len) + 16 bytes.
__host__ __device__ constexpr int slot_j_bytes(int G, int M, int es) {
  return ((4 * G * M * es + 15) & ~15) + 16;
}
__host__ __device__ constexpr int slot_b_bytes(int G, int es) { return ((4 * G * es + 15) & ~15) + 16; }

// ---------------------------------------------------------------------------------------
// A block's lane group: G consecutive lanes starting at `base`; this lane is row group q.
// Reductions add in one fixed order, so every lane of a group holds the same bits.
template <int G>
struct Group {
  int base, q;
  __device__ __forceinline__ explicit Group(int lane) {
    base = (lane / G) * G;
    q = G == 1 ? 0 : lane - base;
  }
  template <typename T>
  __device__ __forceinline__ T sum(T v) const {
    if constexpr (G == 1) {
      return v;
    } else if constexpr (G == 2) {
      return v + __shfl_xor_sync(0xffffffffu, v, 1);
    } else if constexpr (G == 4) {
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      return v + __shfl_xor_sync(0xffffffffu, v, 2);
    } else {
      const T v0 = __shfl_sync(0xffffffffu, v, base);
      const T v1 = __shfl_sync(0xffffffffu, v, base + 1);
      const T v2 = __shfl_sync(0xffffffffu, v, base + 2);
      return (v0 + v1) + v2;
    }
  }
  // Sum of compensated pairs (s + c): TwoSum of the leading parts, errors added to c.
  __device__ __forceinline__ void sum2(float& s, float& c) const {
    if constexpr (G == 1) {
      return;
    } else if constexpr (G == 2 || G == 4) {
#pragma unroll
      for (int d = 1; d < G; d <<= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, d);
        const float c2 = __shfl_xor_sync(0xffffffffu, c, d);
        float t, e;
        two_sum(s, s2, t, e);
        s = t;
        c = __fadd_rn(__fadd_rn(c, c2), e);
      }
    } else {
      const float s0 = __shfl_sync(0xffffffffu, s, base), c0 = __shfl_sync(0xffffffffu, c, base);
      const float s1 = __shfl_sync(0xffffffffu, s, base + 1), c1 = __shfl_sync(0xffffffffu, c, base + 1);
      const float s2 = __shfl_sync(0xffffffffu, s, base + 2), c2 = __shfl_sync(0xffffffffu, c, base + 2);
      float t, e1, t2, e2;
      two_sum(s0, s1, t, e1);
      two_sum(t, s2, t2, e2);
      s = t2;
      c = __fadd_rn(__fadd_rn(__fadd_rn(c0, c1), c2), __fadd_rn(e1, e2));
    }
  }
  template <typename T>
  __device__ __forceinline__ T bcast(T v, int src_q) const {
    if constexpr (G == 1) return v;
    else return __shfl_sync(0xffffffffu, v, base + src_q);
  }
  __device__ __forceinline__ bool owns(int src_q) const {
    if constexpr (G == 1) return true;
    else return q == src_q;
  }
};

template <int G>
__host__ __device__ constexpr int kmax() { return 4 * G < kMaxCols ? 4 * G : kMaxCols; }

// Four consecutive values of a lane's rows (16-byte aligned).
__device__ __forceinline__ void store4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}

// The shape keys a task can have: row class 0 (G = 1) with m <= 4, classes 1-3 with m <= 8.
#define QRKIT_TASK_KEYS(X) \
  X(0) X(1) X(2) X(3) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) X(20) \
  X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31)

// Reciprocal and square root for the factorizations: the hardware approximations for float
// (rcp.approx / sqrt.approx: about one ulp, far below the rounding the factorization itself
// accumulates; zero maps to infinity and to zero), IEEE for double.
__device__ __forceinline__ float rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float root(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double root(double x) { return sqrt(x); }

// Registers of one lane: a[j][u] = row 4q + u of column j (zero below row n), c[u] = rhs.
template <typename T, int G>
__device__ __forceinline__ void load_regs(T (&a)[kMaxCols][4], T (&c)[4], const T* sJ, const T* sB,
                                          int n, int M, int q) {
#pragma unroll
  for (int j = 0; j < kmax<G>(); ++j) {
    if (j < M) {
      const T* col = sJ + j * n;
#pragma unroll
      for (int u = 0; u < 4; ++u) a[j][u] = 4 * q + u < n ? col[4 * q + u] : T(0);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) a[j][u] = T(0);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) c[u] = 4 * q + u < n ? sB[4 * q + u] : T(0);
}

template <typename T, int G>
__device__ __forceinline__ void store_regs(const T (&a)[kMaxCols][4], const T (&c)[4], T* sJ, T* sB,
                                           int n, int M, int q) {
#pragma unroll
  for (int j = 0; j < kmax<G>(); ++j) {
    if (j < M) {
      T* col = sJ + j * n;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (4 * q + u < n) col[4 * q + u] = a[j][u];
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (4 * q + u < n) sB[4 * q + u] = c[u];
}

// Householder QR of the group's block (Sec. 2) in registers, applied to the rhs on the way:
// afterwards a holds R on and above the diagonal and the reflectors' v below it (v[0] = 1
// implicit), c = Q^T b; the reflector coefficients go to tau[k * ts], k < M, as they are formed
// (lanes q = k mod G store tau_k; tau may be null).  M (warp-uniform) columns.
template <typename T, int G>
__device__ __forceinline__ void group_householder(T (&a)[kMaxCols][4], T (&c)[4], T* tau, int ts, int M,
                                                  const Group<G>& g) {
  const int q = g.q;
#pragma unroll
  for (int k = 0; k < kmax<G>(); ++k) {
    if (k < M) {
      // row k is row ku of lane kq: lanes q > kq hold rows below k only, lane kq the rows
      // ku + 1 .. 3 below it, lanes q < kq rows above it only
      const int kq = k >> 2, ku = k & 3;
      const bool gt = q > kq, ge = q >= kq, eq = q == kq;
      T full = T(0), tail = T(0);
#pragma unroll
      for (int u = 3; u >= 0; --u) {
        const T s2 = a[k][u] * a[k][u];
        if (u > ku) tail += s2;
        full += s2;
      }
      const T sq = g.sum(gt ? full : (eq ? tail : T(0)));
      const T alpha = g.bcast(a[k][ku], kq);
      const T nrm = root(alpha * alpha + sq);
      const T beta = alpha >= T(0) ? -nrm : nrm;
      const T d = alpha - beta;
      const bool live = nrm != T(0);
      const T scale = live ? rcp(d) : T(0);
      const T tk = live ? -d * rcp(beta) : T(0);
      const T f_ge = ge ? scale : T(0), f_gt = gt ? scale : T(0);
      T v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u > ku) {
          v[u] = a[k][u] * f_ge;
          a[k][u] = ge ? v[u] : a[k][u];
        } else if (u == ku) {
          v[u] = a[k][u] * f_gt + (eq ? T(1) : T(0));
          a[k][u] = gt ? v[u] : (eq ? beta : a[k][u]);
        } else {
          v[u] = a[k][u] * f_gt;
          a[k][u] = gt ? v[u] : a[k][u];
        }
      }
      if (tau && (k % G) == q) tau[k * ts] = tk;
#pragma unroll
      for (int j = k + 1; j < kmax<G>(); ++j) {
        if (j < M) {
          T w = T(0);
#pragma unroll
          for (int u = 0; u < 4; ++u) w += v[u] * a[j][u];
          w = g.sum(w) * tk;
#pragma unroll
          for (int u = 0; u < 4; ++u) a[j][u] -= v[u] * w;
        }
      }
      T w = T(0);
#pragma unroll
      for (int u = 0; u < 4; ++u) w += v[u] * c[u];
      w = g.sum(w) * tk;
#pragma unroll
      for (int u = 0; u < 4; ++u) c[u] -= v[u] * w;
    }
  }
}

// x = R^{-1} c[0..M): row k of R lives on lane k / 4 of the group, which computes x_k and
// broadcasts it.  Returns false on the lane that holds a zero pivot.
template <typename T, int G>
__device__ __forceinline__ bool group_backsub(const T (&a)[kMaxCols][4], const T (&c)[4], int M,
                                              const Group<G>& g, T (&x)[kMaxCols]) {
  bool ok = true;
#pragma unroll
  for (int k = kmax<G>() - 1; k >= 0; --k) {
    if (k < M) {
      T s = c[k & 3];
#pragma unroll
      for (int j = k + 1; j < kmax<G>(); ++j)
        if (j < M) s -= a[j][k & 3] * x[j];
      const T rkk = a[k][k & 3];
      if (g.owns(k >> 2) && rkk == T(0)) ok = false;
      x[k] = g.bcast(s * rcp(rkk), k >> 2);
    } else {
      x[k] = T(0);
    }
  }
  return ok;
}

// A-priori error estimate of the float least-squares solution.  Householder QR is backward
// stable, so the forward error is a small multiple of u (kappa + kappa^2 ||r|| / (||A|| ||x||))
// = u (||A|| ||A^+|| + ||A|| ||A^+||^2 ||r|| / ||x||) in 2-norms, ||A|| = ||R||, ||A^+|| = ||R^{-1}||.
// Both norms are replaced by upper bounds, so the estimate never falls below that expression:
// ||M||_2 <= min(||M||_F, (||M||_1 ||M||_inf)^(1/2)) (the Frobenius bound is tight for nearly
// rank-one M, the Hoelder one for well-conditioned M).  est = u (a y + a y^2 ||r|| / ||x||) with
// a, y those bounds for R and R^{-1}, u = 2^-24 and ||r|| = || rows M.. of Q^T b ||.  R^{-1} is
// formed column by column (the columns are independent back-substitutions).  True when the
// estimate exceeds `target` (or is NaN: a zero pivot, x = 0).  R: the upper triangle (R[i][k],
// i <= k); res2 = ||r||^2, x2 = ||x||^2; kappa receives the bound a y on the condition number.
template <int M>
__device__ __forceinline__ bool needs_refinement(const float (&R)[M][M], float res2, float x2, float target,
                                                 float& kappa) {
  float d[M];
  float rF2 = 0.f, r1 = 0.f, rI[M];
#pragma unroll
  for (int i = 0; i < M; ++i) rI[i] = 0.f;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    float cs = 0.f;
#pragma unroll
    for (int i = 0; i <= k; ++i) {
      rF2 += R[i][k] * R[i][k];
      cs += fabsf(R[i][k]);
      rI[i] += fabsf(R[i][k]);
    }
    r1 = fmaxf(r1, cs);
    d[k] = rcp(R[k][k]);
  }
  float yF2 = 0.f, y1 = 0.f, yI[M];
#pragma unroll
  for (int i = 0; i < M; ++i) yI[i] = 0.f;
#pragma unroll
  for (int j = 0; j < M; ++j) {   // column j of R^{-1}: y_j = 1 / R_jj, rows above by back-substitution
    float y[M];
    y[j] = d[j];
    float cs = fabsf(y[j]);
    yF2 += y[j] * y[j];
    yI[j] += fabsf(y[j]);
#pragma unroll
    for (int i = j - 1; i >= 0; --i) {
      float sm = 0.f;
#pragma unroll
      for (int l = i + 1; l <= j; ++l) sm += R[i][l] * y[l];
      y[i] = -sm * d[i];
      yF2 += y[i] * y[i];
      cs += fabsf(y[i]);
      yI[i] += fabsf(y[i]);
    }
    y1 = fmaxf(y1, cs);
  }
  float rInf = 0.f, yInf = 0.f;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    rInf = fmaxf(rInf, rI[i]);
    yInf = fmaxf(yInf, yI[i]);
  }
  const float an = fminf(sqrtf(rF2), sqrtf(r1 * rInf));
  const float yn = fminf(sqrtf(yF2), sqrtf(y1 * yInf));
  kappa = an * yn;
  const float est = kUnitRoundoff * (kappa + kappa * yn * sqrtf(res2 / x2));
  return !(est <= target);
}

// The upper triangle of the group's R (row i lives on lane i / 4) on every lane of the group;
// with LEAD only the group's lane 0 needs it, and rows 0..3 are its own.
template <typename T, int G, int M, bool LEAD = false>
__device__ __forceinline__ void group_gather_r(const T (&a)[kMaxCols][4], const Group<G>& g, float (&R)[M][M]) {
#pragma unroll
  for (int k = 0; k < M; ++k)
#pragma unroll
    for (int i = 0; i < M; ++i)
      R[i][k] = i > k ? 0.f : ((LEAD && i < 4) ? (float)a[k][i] : (float)g.bcast(a[k][i & 3], i >> 2));
}

// The refinement's two residuals of the augmented system [I J; J^T 0] [r; x] = [b; 0] in
// extended precision, rounded once to float: f = b - r - J x on the lane's rows and
// g = -J^T r (replicated over the group).  RES = 0: compensated float arithmetic (Dot2 of
// Ogita, Rump and Oishi: error-free products and sums, value = s + c); RES = 1: double.
// jq: the lane's row quad of J's column 0 (16-byte aligned, column stride 4G values, zero past
// n); bl: the lane's rows of b.
template <int G, int M, int RES>
__device__ __forceinline__ void group_aug_residuals(const float* jq, const float (&bl)[4],
                                                    const float (&x)[kMaxCols], const float (&r)[4], const Group<G>& g,
                                                    float (&f)[4], float (&gv)[kMaxCols]) {
  float jr[M][4];
#pragma unroll
  for (int j = 0; j < M; ++j) load4(jq + j * 4 * G, jr[j]);
  if constexpr (RES == 0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float sh, sl, t, e;
      two_sum(bl[u], -r[u], sh, sl);
#pragma unroll
      for (int j = 0; j < M; ++j) {
        const float p = __fmul_rn(jr[j][u], -x[j]);
        const float pe = __fmaf_rn(jr[j][u], -x[j], -p);
        two_sum(sh, p, t, e);
        sh = t;
        sl = __fadd_rn(sl, __fadd_rn(e, pe));
      }
      f[u] = __fadd_rn(sh, sl);
    }
#pragma unroll
    for (int j = 0; j < kMaxCols; ++j) gv[j] = 0.f;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      float sh = 0.f, sl = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float p = __fmul_rn(jr[j][u], r[u]);
        const float pe = __fmaf_rn(jr[j][u], r[u], -p);
        float t, e;
        two_sum(sh, p, t, e);
        sh = t;
        sl = __fadd_rn(sl, __fadd_rn(e, pe));
      }
      g.sum2(sh, sl);
      gv[j] = -__fadd_rn(sh, sl);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      double acc = (double)bl[u] - (double)r[u];
#pragma unroll
      for (int j = 0; j < M; ++j) acc = fma(-(double)jr[j][u], (double)x[j], acc);
      f[u] = (float)acc;
    }
#pragma unroll
    for (int j = 0; j < kMaxCols; ++j) gv[j] = 0.f;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      double acc = 0.0;
#pragma unroll
      for (int u = 0; u < 4; ++u) acc = fma((double)jr[j][u], (double)r[u], acc);
      gv[j] = (float)(-g.sum(acc));
    }
  }
}

// Refinement of the group's block by Bjorck's iterative refinement of the augmented system
// [I J; J^T 0] [r; x] = [b; 0] with the float factor J = Q [R; 0] (a: reflectors below the
// diagonal, R on and above it, tau).  Q_1 (the first M columns of Q) is formed explicitly in
// the lanes' rows by applying the reflectors to [I_M; 0], and R is copied to every lane of the
// group, so that a step needs no sequence of group reductions: only 2M independent ones.
// Start: x from the first solve and r = Q [0; c2] = b - Q_1 Q_1^T b (the residual the
// factorization itself gives).  One step, with the two residuals in extended precision:
// f = b - r - J x, g = -J^T r; h = R^{-T} g; d1 = Q_1^T f; t = d1 - h; dx = R^{-1} t;
// dr = Q [h; d2] = f - Q_1 t (d2 = Q_2^T f, so Q_2 d2 = f - Q_1 d1); x += dx, r += dr.  Its rate
// is about u kappa(J) (not u kappa^2 as for the seminormal equations), so it converges on
// every block with u kappa < 1.  A block stops, after at most `steps` steps, once a correction
// is at most tol relative to x (max norms), or once the next one is predicted to be: the
// error left after a step is about rate * (its correction) with rate <= c u kappa, so a step
// whose correction is below tol / (16 u kappa) relative to x ends the block (kappa: an upper
// bound of its condition number).  x is replicated over the group; jq points to the lane's row
// quad of J's column 0 (column stride 4G values, zero past n) and bl holds its rows of b.
// Returns the steps the block took.
template <int G, int M, int RES>
__device__ __forceinline__ int group_refine_aug(const float (&a)[kMaxCols][4], const float (&tau)[kMaxCols],
                                                float (&x)[kMaxCols], const float* jq, const float (&bl)[4],
                                                int n, float kappa, const Group<G>& g, int steps, float tol) {
  const float next_tol = tol / fmaxf(16.f * kUnitRoundoff * kappa, tol);
  const int q = g.q;
  // Q_1 = H_0 ... H_{M-1} [I_M; 0]: column j is changed by H_j .. H_0 only
  float qm[M][4];
#pragma unroll
  for (int j = 0; j < M; ++j)
#pragma unroll
    for (int u = 0; u < 4; ++u) qm[j][u] = 4 * q + u == j ? 1.f : 0.f;
#pragma unroll
  for (int k = M - 1; k >= 0; --k) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = 4 * q + u;
      v[u] = r > k ? a[k][u] : (r == k ? 1.f : 0.f);
    }
#pragma unroll
    for (int j = k; j < M; ++j) {
      float w = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) w += v[u] * qm[j][u];
      w = g.sum(w) * tau[k];
#pragma unroll
      for (int u = 0; u < 4; ++u) qm[j][u] -= v[u] * w;
    }
  }
  // R on every lane of the group (upper triangle) and 1 / diag
  float R[M][M], d[M];
  group_gather_r<float, G, M>(a, g, R);
#pragma unroll
  for (int i = 0; i < M; ++i) d[i] = rcp(R[i][i]);
  // r = b - Q_1 (Q_1^T b)
  float r[4];
  {
    float c1[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      float w = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) w += qm[j][u] * bl[u];
      c1[j] = g.sum(w);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float t = bl[u];
#pragma unroll
      for (int j = 0; j < M; ++j) t -= qm[j][u] * c1[j];
      r[u] = t;
    }
  }
  bool done = n == 0;
  int taken = 0;
  for (int step = 0; step < steps; ++step) {
    if (__all_sync(0xffffffffu, done)) break;
    taken += done ? 0 : 1;
    float f[4], gv[kMaxCols];
    group_aug_residuals<G, M, RES>(jq, bl, x, r, g, f, gv);
    // t = Q_1^T f - R^{-T} g
    float t[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      float w = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) w += qm[j][u] * f[u];
      t[j] = g.sum(w);
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
      float hk = gv[k];
#pragma unroll
      for (int i = 0; i < k; ++i) hk -= R[i][k] * (gv[i]);
      gv[k] = hk * d[k];   // gv becomes h = R^{-T} g in place
      t[k] -= gv[k];
    }
    // dx = R^{-1} t, dr = f - Q_1 t
    float dx[M];
#pragma unroll
    for (int k = M - 1; k >= 0; --k) {
      float sk = t[k];
#pragma unroll
      for (int l = k + 1; l < M; ++l) sk -= R[k][l] * dx[l];
      dx[k] = sk * d[k];
    }
    float dmax = 0.f, xmax = 0.f;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const float xn = x[k] + dx[k];
      dmax = fmaxf(dmax, fabsf(dx[k]));
      xmax = fmaxf(xmax, fabsf(xn));
      if (!done) x[k] = xn;
    }
    if (!done) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float dr = f[u];
#pragma unroll
        for (int j = 0; j < M; ++j) dr -= qm[j][u] * t[j];
        r[u] += dr;
      }
    }
    done = done || !(dmax > next_tol * xmax);
  }
  return taken;
}

// ---------------------------------------------------------------------------------------
// Software pipeline of a warp.  While task i is computed, the copies for task i + 1's block
// data, task i + 2's entries and task i + 3's header (all per-lane 16-byte cp.async copies)
// are in flight; they were issued as one commit group right after the warp waited for the
// previous group.  Shared memory of a warp: 4 header buffers, 3 entry buffers and 2 data
// buffers, each used by every 4th / 3rd / 2nd task.
constexpr int kHdrBufs = 4, kEntBufs = 3;
// Descriptor bytes of a warp: header buffers and entry buffers of up to 32 entries (entry
// size: 16 bytes in the factor kernel, 32 in the refinement kernel).
__host__ __device__ constexpr int warp_desc_bytes(int entry_bytes) {
  return kHdrBufs * (int)sizeof(TaskHdr) + kEntBufs * 32 * entry_bytes;
}

// Buffers of a warp, addressed by slot numbers (header slot i mod 4, entry slot i mod 3, data
// slot i mod 2 for the warp's i-th task; the loops keep the slot numbers as rotating counters).
struct WarpBufs {
  unsigned char* base;
  int data_bytes;
  int ent_bytes;   // one entry buffer
  __device__ __forceinline__ TaskHdr* hdr(int slot) const {
    return reinterpret_cast<TaskHdr*>(base + slot * (int)sizeof(TaskHdr));
  }
  __device__ __forceinline__ unsigned char* ent(int slot) const {
    return base + kHdrBufs * (int)sizeof(TaskHdr) + slot * ent_bytes;
  }
  __device__ __forceinline__ unsigned char* data(int slot) const {
    return base + kHdrBufs * (int)sizeof(TaskHdr) + kEntBufs * ent_bytes + slot * data_bytes;
  }
};
__device__ __forceinline__ int next3(int s) { return s == 2 ? 0 : s + 1; }

// lane / G and 32 / G for the run-time group sizes G = 1..4 (no integer division).
__device__ __forceinline__ int lane_group(int lane, int G) {
  return G == 1 ? lane : (G == 2 ? lane >> 1 : (G == 3 ? (lane * 11) >> 5 : lane >> 2));
}
__device__ __forceinline__ int blocks_per_task(int G) { return G == 1 ? 32 : (G == 2 ? 16 : (G == 3 ? 10 : 8)); }

// The slots of a block in a task's data buffer (group grp of a task of G lanes per block and
// M columns): J's superset at the J slot, b's after the P J slots; the values start at the
// global address's offset modulo 16.
template <typename T>
__device__ __forceinline__ void slot_ptrs(unsigned char* db, int G, int M, int grp, const T* gJ, const T* gB,
                                          unsigned char*& sJraw, unsigned char*& sBraw, T*& sJ, T*& sB) {
  const int P = task_blocks(G);
  const int JS = slot_j_bytes(G, M, (int)sizeof(T));
  const int BS = slot_b_bytes(G, (int)sizeof(T));
  sJraw = db + grp * JS;
  sBraw = db + P * JS + grp * BS;
  sJ = reinterpret_cast<T*>(sJraw + (reinterpret_cast<uintptr_t>(gJ) & 15));
  sB = reinterpret_cast<T*>(sBraw + (reinterpret_cast<uintptr_t>(gB) & 15));
}

// Copy of count values starting at g into a slot by the G lanes of a group: the
// 16-byte-aligned superset by 16-byte cp.async copies, or, where the superset would leave the
// buffer [lo, hi), the values themselves by plain loads (s = the slot's first value).
template <typename T>
__device__ __forceinline__ void issue_span(const T* g, int count, int G, int q, const T* lo, const T* hi,
                                           unsigned char* sraw, T* s) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(g);
  const uintptr_t l = a & ~(uintptr_t)15, h = (a + (uintptr_t)count * sizeof(T) + 15) & ~(uintptr_t)15;
  if (l >= reinterpret_cast<uintptr_t>(lo) && h <= reinterpret_cast<uintptr_t>(hi)) {
    const int nch = (int)((h - l) >> 4);
    for (int c = q; c < nch; c += G) cp_async16(sraw + 16 * c, reinterpret_cast<const void*>(l + 16 * (uintptr_t)c));
  } else {
    for (int k = q; k < count; k += G) s[k] = g[k];
  }
}

// Copies of one block's J (n x M values) and b (n values) into its slots.
template <typename T>
__device__ __forceinline__ void issue_block(const T* gJ, const T* gB, int n, int M, int G, int q, const T* J_lo,
                                            const T* J_hi, const T* b_lo, const T* b_hi, unsigned char* sJraw,
                                            unsigned char* sBraw, T* sJ, T* sB) {
  if (n <= 0) return;
  issue_span<T>(gJ, n * M, G, q, J_lo, J_hi, sJraw, sJ);
  issue_span<T>(gB, n, G, q, b_lo, b_hi, sBraw, sB);
}

// Copy of count elements from a slot to global memory: where both agree modulo 16 bytes the
// aligned interior goes as 16-byte vector stores, head and tail as plain stores; the group's
// lanes share the work.
template <typename T, int G>
__device__ __forceinline__ void send(T* dst, const T* src, int count, bool vec, int q) {
  if (!vec) {
    for (int k = q; k < count; k += G) dst[k] = src[k];
    return;
  }
  constexpr int VN = 16 / (int)sizeof(T);
  int h, ni;
  interior(dst, count, h, ni);
  const int nch = ni / VN;
  for (int c = q; c < nch; c += G)
    *reinterpret_cast<uint4*>(dst + h + c * VN) = *reinterpret_cast<const uint4*>(src + h + c * VN);
  for (int k = q; k < h; k += G) dst[k] = src[k];
  for (int k = h + ni + q; k < count; k += G) dst[k] = src[k];
}

// A block selected for refinement: its column offset (x), the offset of its first factor value
// in the task planes, its row count and the bound ||R||_F ||R^{-1}||_F on its condition number.
// Everything else the refinement reads is in the block's record (same list position).
struct RefEntry {
  int64_t c, f;
  int32_t n;
  float kappa;
  int64_t pad;
};
static_assert(sizeof(RefEntry) == 32, "refinement list layout");

// Refinement record of a block of shape key (G, M): its J in M columns of 4G rows (rows past n
// zero), b in 4G rows and the float solution x (8 values).
__host__ __device__ constexpr int record_values(int G, int M) { return 4 * G * (M + 1) + 8; }
__host__ __device__ constexpr int record_b(int G, int M) { return 4 * G * M; }
__host__ __device__ constexpr int record_tail(int G, int M) { return 4 * G * (M + 1); }

template <typename T>
struct TaskArgs {
  const TaskHdr* hdr;
  const TaskEntry* ent;
  int64_t num_tasks;
  const T* J;
  const T* b;
  const T* J_end;   // one past the last value (bounds of the copied supersets)
  const T* b_end;
  T* tF;            // factor in task planes (kPlaneValues per plane)
  T* tTau;          // tau in task planes (kTauPlane per plane)
  T* qtb;           // may be null
  T* x;
  int q_vec;        // qtb agrees with b modulo 16 bytes
  int warp_bytes;   // shared memory per warp (descriptor and data buffers)
  int data_bytes;   // one data buffer
  int* status;
  float select;             // selection: a-priori error estimate above which a block is refined
  RefEntry* rlist;          // selection: blocks to refine, one list per shape key
  int* rcount;              // kTaskKeys counts
  const int64_t* key_off;   // kTaskKeys + 1 list offsets (list capacity = blocks of the key)
  float* rec;               // refinement records, key k's at rec_off[k], in list order
  const int64_t* rec_off;
};

// Pipeline stages of the factor kernel: the header of task t, the entries of task t (its
// header is in shared memory), the block data of task t (header and entries are).
__device__ __forceinline__ void issue_hdr(const TaskHdr* g, int64_t t, int64_t T, TaskHdr* s, int lane) {
  if (t < T && lane < (int)sizeof(TaskHdr) / 16)
    cp_async16(reinterpret_cast<unsigned char*>(s) + 16 * lane, reinterpret_cast<const unsigned char*>(g + t) + 16 * lane);
}
__device__ __forceinline__ void issue_ent(const TaskEntry* g, int64_t t, int64_t T, const TaskHdr* sh,
                                          unsigned char* s, int lane) {
  if (t >= T) return;
  const int P = blocks_per_task(group_lanes(sh->key));
  if (lane < P) cp_async16(s + 16 * lane, g + sh->first + lane);
}
template <typename T>
__device__ __forceinline__ void issue_data(const TaskArgs<T>& A, int64_t t, const TaskHdr* sh, const unsigned char* se,
                                           unsigned char* db, int lane) {
  if (t >= A.num_tasks) return;
  const int key = sh->key;
  const int G = group_lanes(key), M = (key & 7) + 1, P = blocks_per_task(G);
  const int grp = lane_group(lane, G), q = lane - grp * G;
  if (grp >= P) return;
  const TaskEntry e = reinterpret_cast<const TaskEntry*>(se)[grp];
  const T* gJ = A.J + sh->v0 + e.v;
  const T* gB = A.b + sh->r0 + e.r;
  unsigned char *sJraw, *sBraw;
  T *sJ, *sB;
  slot_ptrs<T>(db, G, M, grp, gJ, gB, sJraw, sBraw, sJ, sB);
  issue_block<T>(gJ, gB, e.n, M, G, q, A.J, A.J_end, A.b, A.b_end, sJraw, sBraw, sJ, sB);
}

// One task of shape key (G, M), its data staged in db: M is a compile-time constant, so every
// loop bound and guard of the inlined helpers folds away.  The factor leaves the registers
// directly for the task's planes (one 16-byte store per lane and column), tau for its tau
// planes; J and b stay in the slots (a selected block's record is copied from there).
template <typename T, int G, int M, bool SEL>
__device__ __forceinline__ void run_task(const TaskArgs<T>& A, const TaskHdr& h, const unsigned char* se,
                                         unsigned char* db, int lane) {
  constexpr int P = task_blocks(G);
  const int grp = lane / G;
  const bool act = grp < P;
  const Group<G> g(lane);
  TaskEntry e{};
  if (act) e = reinterpret_cast<const TaskEntry*>(se)[grp];
  const int n = e.n;
  const T* gJ = A.J + h.v0 + e.v;
  const T* gB = A.b + h.r0 + e.r;
  unsigned char *sJraw, *sBraw;
  T *sJ, *sB;
  slot_ptrs<T>(db, G, M, act ? grp : 0, gJ, gB, sJraw, sBraw, sJ, sB);
  T a[kMaxCols][4], c[4], x[kMaxCols];
  load_regs<T, G>(a, c, sJ, sB, n, M, g.q);
  const int64_t plane = h.plane;
  group_householder<T, G>(a, c, n > 0 ? A.tTau + plane * kTauPlane + grp : nullptr, kTauPlane, M, g);
  if (!group_backsub<T, G>(a, c, M, g, x) && n > 0) record(A.status, QRKIT_ESINGULAR);
  T x2 = T(0);
  if (n > 0) {
    T* dx = A.x + h.c0 + e.c;
#pragma unroll
    for (int k = 0; k < kmax<G>(); ++k)
      if (k < M && (k % G) == g.q) dx[k] = x[k];
    T* f = A.tF + plane * kPlaneValues + grp * 4 * G + 4 * g.q;
#pragma unroll
    for (int j = 0; j < M; ++j) store4(f + j * kPlaneValues, a[j]);
  }
#pragma unroll
  for (int k = 0; k < kmax<G>(); ++k)
    if (k < M) x2 += x[k] * x[k];
  if constexpr (SEL) {
    float res2 = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = 4 * g.q + u;
      res2 += (r >= M && r < n) ? (float)(c[u] * c[u]) : 0.f;
    }
    res2 = g.sum(res2);
    float R[M][M];
    group_gather_r<T, G, M, true>(a, g, R);   // valid on the group's lane 0, which decides
    float kappa = 0.f;
    const bool need = n > 0 && needs_refinement<M>(R, res2, (float)x2, A.select, kappa);
    const bool sel = act && g.q == 0 && need;
    const unsigned mask = __ballot_sync(0xffffffffu, sel);
    if (mask) {
      int first = 0;
      if (lane == 0) first = atomicAdd(A.rcount + h.key, __popc(mask));
      first = __shfl_sync(0xffffffffu, first, 0);
      const int64_t pos = g.bcast((int64_t)first + __popc(mask & ((1u << lane) - 1u)), 0);
      const bool gsel = g.bcast(sel ? 1 : 0, 0) != 0;
      const int64_t cap = A.key_off[h.key + 1] - A.key_off[h.key];
      if (gsel && pos < cap) {
        // the record: J and b of the block from the slots (the lane's rows, zero past n) and x
        float* rec = A.rec + A.rec_off[h.key] + pos * record_values(G, M) + 4 * g.q;
#pragma unroll
        for (int j = 0; j < M; ++j) {
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = 4 * g.q + u < n ? (float)sJ[j * n + 4 * g.q + u] : 0.f;
          store4(rec + j * 4 * G, v);
        }
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = 4 * g.q + u < n ? (float)sB[4 * g.q + u] : 0.f;
        store4(rec + record_b(G, M), v);
        if (g.q == 0) {
          float* tail = rec + record_tail(G, M);   // rec includes the lane offset 4q = 0 here
          float xv[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) xv[k] = k < M ? (float)x[k] : 0.f;
          store4(tail, *reinterpret_cast<const float(*)[4]>(xv));
          store4(tail + 4, *reinterpret_cast<const float(*)[4]>(xv + 4));
          RefEntry re;
          re.c = h.c0 + e.c;
          re.f = plane * kPlaneValues + grp * 4 * G;
          re.n = n;
          re.kappa = kappa;
          re.pad = 0;
          A.rlist[A.key_off[h.key] + pos] = re;
        }
      }
    }
  }
  if (A.qtb) {   // Q^T b through the b slot to HBM
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (4 * g.q + u < n) sB[4 * g.q + u] = c[u];
    __syncwarp();
    if (n > 0) send<T, G>(A.qtb + h.r0 + e.r, sB, n, A.q_vec != 0, g.q);
  }
}

// Key classes of the factor kernel: 0 every key; for float, 1 the keys of blocks with at most
// 4 columns (compiled for 3 resident CTAs per SM: more warps to hide latency, and their
// register needs fit) and 2 the wider ones (2 CTAs per SM).
__host__ __device__ constexpr bool key_in_class(int key, int cls) {
  return cls == 0 || ((key & 7) < 4) == (cls == 1);
}
template <typename T, int CLS>
constexpr int task_ctas() {
  return sizeof(T) == 4 ? (CLS == 1 ? 3 : QRKIT_TASK_CTAS) : 2;
}

template <typename T, bool SEL, int CLS = 0>
__global__ void __launch_bounds__(32 * kTaskMaxWarps, task_ctas<T, CLS>()) block_task_kernel(TaskArgs<T> A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  const WarpBufs W{smem_raw + (size_t)wid * A.warp_bytes, A.data_bytes, 32 * (int)sizeof(TaskEntry)};
  const int64_t NT = A.num_tasks;
  const int64_t t0 = (int64_t)blockIdx.x * wpc + wid, stride = (int64_t)gridDim.x * wpc;
  if (t0 >= NT) return;
  // prologue: header 0; header 1 and entries 0; header 2, entries 1 and data 0
  issue_hdr(A.hdr, t0, NT, W.hdr(0), lane);
  cp_async_commit();
  cp_async_wait_all();
  __syncwarp();
  issue_hdr(A.hdr, t0 + stride, NT, W.hdr(1), lane);
  issue_ent(A.ent, t0, NT, W.hdr(0), W.ent(0), lane);
  cp_async_commit();
  cp_async_wait_all();
  __syncwarp();
  issue_hdr(A.hdr, t0 + 2 * stride, NT, W.hdr(2), lane);
  issue_ent(A.ent, t0 + stride, NT, W.hdr(1), W.ent(1), lane);
  issue_data<T>(A, t0, W.hdr(0), W.ent(0), W.data(0), lane);
  cp_async_commit();
  int sh = 0, se = 0, sd = 0;   // slots of task i
  for (int64_t t = t0; t < NT; t += stride) {
    cp_async_wait_all();
    __syncwarp();   // task i's data, task i + 1's entries and task i + 2's header have landed
    const int sh1 = (sh + 1) & 3, sh2 = (sh + 2) & 3, sh3 = (sh + 3) & 3;
    const int se1 = next3(se), se2 = next3(se1);
    issue_hdr(A.hdr, t + 3 * stride, NT, W.hdr(sh3), lane);
    issue_ent(A.ent, t + 2 * stride, NT, W.hdr(sh2), W.ent(se2), lane);
    issue_data<T>(A, t + stride, W.hdr(sh1), W.ent(se1), W.data(sd ^ 1), lane);
    cp_async_commit();
    const TaskHdr h = *W.hdr(sh);
    switch (h.key) {
#define QRKIT_TASK_CASE(k)                                                                       \
  case k:                                                                                        \
    if constexpr (key_in_class(k, CLS)) run_task<T, ((k) >> 3) + 1, ((k) & 7) + 1, SEL>(A, h, W.ent(se), W.data(sd), lane); \
    break;
      QRKIT_TASK_KEYS(QRKIT_TASK_CASE)
#undef QRKIT_TASK_CASE
      default: if (lane == 0) record(A.status, QRKIT_EINVAL); break;
    }
    __syncwarp();   // every lane is done with task i's buffers before they are refilled
    sh = sh1;
    se = se1;
    sd ^= 1;
  }
  cp_async_wait_all();
}

// ---------------------------------------------------------------------------------------
// Refinement of the listed blocks (float).  A task is P listed blocks of one shape key; each
// group reads its block's record (J, b and the float solution, contiguous) and its factor rows
// from the task planes, by 16-byte loads of whole row quads, and refines it.  The factor and
// the solution come from the first kernel, so the blocks are not factored again.
struct RefineTaskArgs {
  const float* tF;     // factor planes of the first kernel
  const float* rec;    // records
  const int64_t* rec_off;
  float* x;            // in: the first kernel's solution; out: refined
  const RefEntry* rlist;
  const int* rcount;
  const int64_t* key_off;
  int steps;
  float tol;
  int* steps_max;      // the most steps any block took (atomic maximum)
  int* status;
};

// Refinement tasks: per shape key, ceil(selected / P) tasks of P listed blocks; a task index
// maps to its key through the keys' prefix sums (lane k holds key k's first task).
struct RefineTasks {
  int64_t start, total;
  __device__ __forceinline__ void key_of(int64_t t, int& key, int64_t& local) const {
    key = 31 - __clz(__ballot_sync(0xffffffffu, start <= t));
    local = t - __shfl_sync(0xffffffffu, start, key);
  }
};

__device__ __forceinline__ int64_t ref_count(const RefineTaskArgs& A, int key) {
  const int64_t cap = A.key_off[key + 1] - A.key_off[key];
  return (int64_t)A.rcount[key] < cap ? (int64_t)A.rcount[key] : cap;
}

template <int G, int M, int RES>
__device__ __forceinline__ void refine_task(const RefineTaskArgs& A, int key, int64_t local, int lane) {
  constexpr int P = task_blocks(G);
  const int grp = lane / G;
  const Group<G> g(lane);
  const int64_t idx = local * P + grp;
  const bool have = grp < P && idx < ref_count(A, key);
  RefEntry e{};
  if (have) e = A.rlist[A.key_off[key] + idx];
  const int n = have ? e.n : 0;
  const float* rec = A.rec + A.rec_off[key] + (have ? idx : 0) * record_values(G, M);
  float bl[4], a[kMaxCols][4], tau[kMaxCols], x[kMaxCols];
#pragma unroll
  for (int j = 0; j < kMaxCols; ++j) {
#pragma unroll
    for (int u = 0; u < 4; ++u) a[j][u] = 0.f;
    tau[j] = 0.f;
    x[j] = 0.f;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) bl[u] = 0.f;
  if (n > 0) {
    const float* f = A.tF + e.f + 4 * g.q;
#pragma unroll
    for (int j = 0; j < M; ++j) load4(f + j * kPlaneValues, a[j]);
    load4(rec + record_b(G, M) + 4 * g.q, bl);
#pragma unroll
    for (int k = 0; k < M; ++k) x[k] = rec[record_tail(G, M) + k];
  }
  // tau_k = 2 / v^T v of the stored reflector (v_k = 1), equal in exact arithmetic to the
  // (beta - alpha) / beta the factorization formed
#pragma unroll
  for (int k = 0; k < M; ++k) {
    float w = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) w += 4 * g.q + u > k ? a[k][u] * a[k][u] : 0.f;
    w = g.sum(w);   // every lane takes part in the group reduction
    tau[k] = n > 0 ? 2.f / (1.f + w) : 0.f;
  }
  const int taken = group_refine_aug<G, M, RES>(a, tau, x, rec + 4 * g.q, bl, n, e.kappa, g, A.steps, A.tol);
  const int most = __reduce_max_sync(0xffffffffu, n > 0 ? taken : 0);
  if (lane == 0 && most > 0) atomicMax(A.steps_max, most);
  if (n > 0) {
    float* dx = A.x + e.c;
#pragma unroll
    for (int k = 0; k < kmax<G>(); ++k)
      if (k < M && (k % G) == g.q) dx[k] = x[k];
  }
}

template <int RES>
__global__ void __launch_bounds__(32 * kTaskMaxWarps, QRKIT_REFINE_CTAS) block_task_refine_kernel(RefineTaskArgs A) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpc = blockDim.x >> 5;
  // tasks per shape key (lane k: key k), their exclusive prefix sums over the keys
  RefineTasks RT;
  {
    const int64_t cnt = ref_count(A, lane);
    const int64_t per = task_blocks(group_lanes(lane));
    const int64_t tk = (cnt + per - 1) / per;
    int64_t inc = tk;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t o = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += o;
    }
    RT.start = inc - tk;
    RT.total = __shfl_sync(0xffffffffu, inc, 31);
  }
  const int64_t stride = (int64_t)gridDim.x * wpc;
  for (int64_t t = (int64_t)blockIdx.x * wpc + wid; t < RT.total; t += stride) {
    int key;
    int64_t local;
    RT.key_of(t, key, local);
    switch (key) {
#define QRKIT_REFINE_CASE(k) \
  case k: refine_task<((k) >> 3) + 1, ((k) & 7) + 1, RES>(A, key, local, lane); break;
      QRKIT_TASK_KEYS(QRKIT_REFINE_CASE)
#undef QRKIT_REFINE_CASE
      default: break;
    }
  }
}

// The factor of the task planes copied into J's packing (reflectors below the diagonal, R on
// and above it) and tau into column order: one warp per task, lanes as in the factor kernel.
template <typename T>
__global__ void __launch_bounds__(256) unpack_factor_kernel(const TaskHdr* hdr, const TaskEntry* ent,
                                                             int64_t num_tasks, const T* tF, const T* tTau, T* F,
                                                             T* tau) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = w0; t < num_tasks; t += stride) {
    const TaskHdr h = hdr[t];
    const int G = group_lanes(h.key), M = (h.key & 7) + 1, P = blocks_per_task(G);
    const int grp = lane_group(lane, G), q = lane - grp * G;
    if (grp >= P) continue;
    const TaskEntry e = ent[h.first + grp];
    const int n = e.n;
    if (n == 0) continue;
    const int64_t plane = h.plane;
    for (int j = 0; j < M; ++j)
      for (int u = 0; u < 4; ++u) {
        const int r = 4 * q + u;
        if (F && r < n) F[h.v0 + e.v + (int64_t)j * n + r] = tF[(plane + j) * kPlaneValues + grp * 4 * G + r];
      }
    if (tau && q == 0)
      for (int k = 0; k < M; ++k) tau[h.c0 + e.c + k] = tTau[(plane + k) * kTauPlane + grp];
  }
}

// Host-side entry points of the kernels; each is defined by the translation unit that
// instantiates its kernel (block_tasks_<kind>.cu), so the variants compile in parallel.
template <typename T, bool SEL, int CLS>
cudaError_t kernel_setup(size_t smem, int threads, int* per_sm);
template <typename T, bool SEL, int CLS>
cudaError_t kernel_launch(const TaskArgs<T>& A, unsigned grid, int threads, size_t smem, cudaStream_t st);

// The definitions an instantiating translation unit expands for its (T, SEL, CLS).
#define QRKIT_TASK_KERNEL_ENTRIES(T, SEL, CLS)                                                            \
  template <>                                                                                             \
  cudaError_t kernel_setup<T, SEL, CLS>(size_t smem, int threads, int* per_sm) {                          \
    auto k = block_task_kernel<T, SEL, CLS>;                                                              \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
    if (e != cudaSuccess) return e;                                                                       \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem);                      \
  }                                                                                                       \
  template <>                                                                                             \
  cudaError_t kernel_launch<T, SEL, CLS>(const TaskArgs<T>& A, unsigned grid, int threads, size_t smem,   \
                                         cudaStream_t st) {                                               \
    block_task_kernel<T, SEL, CLS><<<grid, threads, smem, st>>>(A);                                       \
    return cudaGetLastError();                                                                            \
  }
// RES: the refinement's residual precision (0: compensated float, 1: double).
template <int RES>
cudaError_t refine_setup(size_t smem, int threads, int* per_sm);
template <int RES>
cudaError_t refine_launch(const RefineTaskArgs& A, unsigned grid, int threads, size_t smem, cudaStream_t st);

}  // namespace tasks
}  // namespace qrkit
