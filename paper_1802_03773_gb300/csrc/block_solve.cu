// Batched block-diagonal QR solve (Sec. 4.1 "Block diagonal", Sec. 5.1 solver interface),
// fused: factor + Q^T b + back-substitution + refinement in one pass over HBM.
//
// Work mapping (GB300): one persistent launch; each CTA walks tiles of consecutive blocks
// (cut by the plan so a tile fits the shared-memory budget).  A tile's J values and b are
// staged in shared memory with 16-byte vector loads, every block is factored by a group of
// 4 lanes (lane q holds rows q, q+4, q+8, q+12 in registers), Householder norms and dot
// products are 4-lane shuffle reductions, and the results go back to HBM with vector
// stores.  Blocks of a warp share the warp's largest column count as loop bound.
//
// Reflector convention (Sec. 2): H = I - tau v v^T, v[0] = 1, beta = -sign(x0) ||x||.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace qrkit {
namespace {

constexpr int kG = 4;          // lanes per block
constexpr int kRPL = 4;        // rows per lane -> at most 16 rows per block
constexpr int kMaxC = 8;       // at most 8 columns per block
constexpr int kThreads = 256;  // threads per CTA

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

// ---------------------------------------------------------------------------------------
// Extended-precision residual arithmetic.
// For float factors the residual r = b - J x and g = J^T r are accumulated in double-float
// (an unevaluated sum hi + lo of two floats) built from the error-free transformations
// TwoSum (Knuth) and TwoProduct via FMA (Dekker / Ogita-Rump-Oishi).  Every operation uses
// the _rn intrinsics so the compiler cannot contract or reassociate them.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  DF r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}
// x + a * b with the product taken exactly.
__device__ __forceinline__ DF df_add_prod(DF x, float a, float b) {
  float p = __fmul_rn(a, b);
  float pe = __fmaf_rn(a, b, -p);
  float s, e;
  two_sum(x.hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, pe));
  DF r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}
// x + a * (y.hi + y.lo)
__device__ __forceinline__ DF df_add_prod_df(DF x, float a, DF y) {
  float p = __fmul_rn(a, y.hi);
  float pe = __fmaf_rn(a, y.hi, -p);
  pe = __fmaf_rn(a, y.lo, pe);
  float s, e;
  two_sum(x.hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, pe));
  DF r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

// Accumulator policies: Hi<T, kind>::acc is the residual type.
//   kind 0: plain double (used for T = double, and selectable for float)
//   kind 1: double-float (float factors only)
template <typename T, int KIND> struct Hi;
template <typename T> struct Hi<T, 0> {
  using acc = double;
  static __device__ __forceinline__ acc from(T a) { return (double)a; }
  static __device__ __forceinline__ acc sub_prod(acc x, T a, T b) {
    return fma(-(double)a, (double)b, x);
  }
  static __device__ __forceinline__ acc add_prod_acc(acc x, T a, acc y) {
    return fma((double)a, y, x);
  }
  static __device__ __forceinline__ acc add(acc x, acc y) { return x + y; }
  static __device__ __forceinline__ acc zero() { return 0.0; }
  static __device__ __forceinline__ acc shfl_xor(acc x, int m) {
    return __shfl_xor_sync(0xffffffffu, x, m);
  }
  static __device__ __forceinline__ T round(acc x) { return (T)x; }
};
template <> struct Hi<float, 1> {
  using acc = DF;
  static __device__ __forceinline__ acc from(float a) { return DF{a, 0.f}; }
  static __device__ __forceinline__ acc sub_prod(acc x, float a, float b) {
    return df_add_prod(x, -a, b);
  }
  static __device__ __forceinline__ acc add_prod_acc(acc x, float a, acc y) {
    return df_add_prod_df(x, a, y);
  }
  static __device__ __forceinline__ acc add(acc x, acc y) { return df_add(x, y); }
  static __device__ __forceinline__ acc zero() { return DF{0.f, 0.f}; }
  static __device__ __forceinline__ acc shfl_xor(acc x, int m) {
    DF r;
    r.hi = __shfl_xor_sync(0xffffffffu, x.hi, m);
    r.lo = __shfl_xor_sync(0xffffffffu, x.lo, m);
    return r;
  }
  static __device__ __forceinline__ float round(acc x) { return __fadd_rn(x.hi, x.lo); }
};

template <typename T>
__device__ __forceinline__ T group_sum(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

__device__ __forceinline__ void record(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

template <typename T>
__device__ __forceinline__ bool finite_val(T v) {
  return isfinite(v);
}

// Copy count elements global -> shared.  dst[k] <-> src[k]; dst must be laid out so that
// (dst + k) and (src + k) share their offset modulo 16 bytes (the caller offsets dst).
template <typename T>
__device__ __forceinline__ void copy_in(T* dst, const T* __restrict__ src, int64_t count) {
  using V = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::n;
  const uintptr_t a = reinterpret_cast<uintptr_t>(src);
  if (((a ^ reinterpret_cast<uintptr_t>(dst)) & 15) != 0) {
    for (int64_t k = threadIdx.x; k < count; k += blockDim.x) dst[k] = src[k];
    return;
  }
  int head = (int)(((16 - (a & 15)) & 15) / sizeof(T));
  if (head > count) head = (int)count;
  for (int k = threadIdx.x; k < head; k += blockDim.x) dst[k] = src[k];
  const int64_t nvec = (count - head) / VN;
  const V* vs = reinterpret_cast<const V*>(src + head);
  V* vd = reinterpret_cast<V*>(dst + head);
  for (int64_t k = threadIdx.x; k < nvec; k += blockDim.x) vd[k] = __ldcs(vs + k);
  for (int64_t k = head + nvec * VN + threadIdx.x; k < count; k += blockDim.x) dst[k] = src[k];
}

// Copy count elements shared -> global with the same alignment rule; never writes outside
// [dst, dst + count).
template <typename T>
__device__ __forceinline__ void copy_out(T* __restrict__ dst, const T* src, int64_t count) {
  using V = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::n;
  const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
  if (((a ^ reinterpret_cast<uintptr_t>(src)) & 15) != 0) {
    for (int64_t k = threadIdx.x; k < count; k += blockDim.x) dst[k] = src[k];
    return;
  }
  int head = (int)(((16 - (a & 15)) & 15) / sizeof(T));
  if (head > count) head = (int)count;
  for (int k = threadIdx.x; k < head; k += blockDim.x) dst[k] = src[k];
  const int64_t nvec = (count - head) / VN;
  V* vd = reinterpret_cast<V*>(dst + head);
  const V* vs = reinterpret_cast<const V*>(src + head);
  for (int64_t k = threadIdx.x; k < nvec; k += blockDim.x) __stcs(vd + k, vs[k]);
  for (int64_t k = head + nvec * VN + threadIdx.x; k < count; k += blockDim.x) dst[k] = src[k];
}

// Exclusive scan of three per-block quantities over a tile (nb <= kThreads).
__device__ __forceinline__ void tile_scan3(int nb, const uint8_t* sN, const uint8_t* sM,
                                           int* sVo, int* sRo, int* sCo, int* warp_tot) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int nn = tid < nb ? sN[tid] : 0;
  int mm = tid < nb ? sM[tid] : 0;
  int v = nn * mm, r = nn, c = mm;
  int iv = v, ir = r, ic = c;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int tv = __shfl_up_sync(0xffffffffu, iv, d);
    int tr = __shfl_up_sync(0xffffffffu, ir, d);
    int tc = __shfl_up_sync(0xffffffffu, ic, d);
    if (lane >= d) { iv += tv; ir += tr; ic += tc; }
  }
  if (lane == 31) {
    warp_tot[wid * 3 + 0] = iv;
    warp_tot[wid * 3 + 1] = ir;
    warp_tot[wid * 3 + 2] = ic;
  }
  __syncthreads();
  int bv = 0, br = 0, bc = 0;
  for (int w = 0; w < wid; ++w) {
    bv += warp_tot[w * 3 + 0];
    br += warp_tot[w * 3 + 1];
    bc += warp_tot[w * 3 + 2];
  }
  if (tid < nb) {
    sVo[tid] = bv + iv - v;
    sRo[tid] = br + ir - r;
    sCo[tid] = bc + ic - c;
  }
  __syncthreads();
}

template <typename T>
struct BlockSolveArgs {
  const uint8_t* n;
  const uint8_t* m;
  const int64_t* tile_block;
  const int64_t* tile_val;
  const int64_t* tile_row;
  const int64_t* tile_col;
  int64_t num_tiles;
  const T* J;
  const T* b;
  T* F;        // factor, J packing
  T* tau;      // sum m
  T* qtb;      // sum n (may be null)
  T* x;        // sum m
  int refine_steps;
  int* status;
  int vb, rb, cb, bb;  // tile budgets
};

template <typename T>
struct Smem {
  T* J;
  T* b;
  T* tau;
  T* x;
  uint8_t* n;
  uint8_t* m;
  int* vo;
  int* ro;
  int* co;
  int* wtot;
};

template <typename T>
__host__ __device__ inline size_t smem_bytes(int vb, int rb, int cb, int bb) {
  const int VN = 16 / (int)sizeof(T);
  size_t off = 0;
  off += (size_t)(vb + VN) * sizeof(T);
  off += (size_t)(rb + VN) * sizeof(T);
  off += (size_t)(cb + VN) * sizeof(T) * 2;
  off += (size_t)((bb + 15) / 16 * 16) * 2;
  off += (size_t)(bb + 1) * sizeof(int) * 3;
  off += (size_t)(kThreads / 32) * 3 * sizeof(int);
  return (off + 15) / 16 * 16;
}

// One group (4 lanes) factors and solves one block held in registers.
//   a[r][j] = B[q + 4 r][j] (row-major per lane), bb[r] = b[q + 4 r]
template <typename T, int HK>
__device__ __forceinline__ void factor_solve_group(
    int q, int gbase, int nn, int mm, int mw, bool valid, T (&a)[kRPL][kMaxC], T (&bb)[kRPL],
    T (&taus)[kMaxC], T (&xs)[kMaxC], const T* sJb, const T* sBb, int refine_steps,
    int* status) {
  // ---- Householder QR, one reflector per column (Sec. 2) ----
#pragma unroll
  for (int k = 0; k < kMaxC; ++k) {
    if (k < mw) {
      T sq = 0;
#pragma unroll
      for (int r = 0; r < kRPL; ++r) {
        const int i = q + kG * r;
        if (i > k && i < nn) sq += a[r][k] * a[r][k];
      }
      sq = group_sum(sq);
      const T alpha = __shfl_sync(0xffffffffu, a[k / kG][k], gbase + (k % kG));
      const T norm = sqrt(alpha * alpha + sq);
      T beta, tau, scale;
      if (norm == T(0)) {
        beta = 0; tau = 0; scale = 0;
      } else {
        beta = alpha >= T(0) ? -norm : norm;
        tau = (beta - alpha) / beta;
        scale = T(1) / (alpha - beta);
      }
      // v_i = a_ik * scale below the diagonal, v_k = 1
      T v[kRPL];
#pragma unroll
      for (int r = 0; r < kRPL; ++r) {
        const int i = q + kG * r;
        v[r] = (i == k) ? T(1) : ((i > k && i < nn) ? a[r][k] * scale : T(0));
      }
      // apply H_k to the trailing columns and the rhs
#pragma unroll
      for (int j = k + 1; j < kMaxC; ++j) {
        if (j < mw) {
          T w = 0;
#pragma unroll
          for (int r = 0; r < kRPL; ++r) w += v[r] * a[r][j];
          w = group_sum(w) * tau;
#pragma unroll
          for (int r = 0; r < kRPL; ++r) a[r][j] -= v[r] * w;
        }
      }
      {
        T w = 0;
#pragma unroll
        for (int r = 0; r < kRPL; ++r) w += v[r] * bb[r];
        w = group_sum(w) * tau;
#pragma unroll
        for (int r = 0; r < kRPL; ++r) bb[r] -= v[r] * w;
      }
      // store v below the diagonal and beta on it
#pragma unroll
      for (int r = 0; r < kRPL; ++r) {
        const int i = q + kG * r;
        if (i == k) a[r][k] = beta;
        else if (i > k) a[r][k] = v[r];
      }
      taus[k] = tau;
    }
  }
  // ---- back-substitution R x = c (Sec. 5.1, matrixR().solve) ----
  bool bad = false;
#pragma unroll
  for (int k = kMaxC - 1; k >= 0; --k) {
    if (k < mw) {
      T s = bb[k / kG];
#pragma unroll
      for (int j = k + 1; j < kMaxC; ++j)
        if (j < mw) s -= a[k / kG][j] * xs[j];
      T xk = s / a[k / kG][k];
      xk = __shfl_sync(0xffffffffu, xk, gbase + (k % kG));
      xs[k] = (k < mm) ? xk : T(0);
      if (valid && k < mm && !finite_val(xk)) bad = true;
    }
  }
  // ---- refinement: x += R^{-1} R^{-T} (J^T (b - J x)), residual in extended precision ----
  using H = Hi<T, HK>;
  for (int step = 0; step < refine_steps; ++step) {
    typename H::acc res[kRPL];
#pragma unroll
    for (int r = 0; r < kRPL; ++r) {
      const int i = q + kG * r;
      typename H::acc acc = H::zero();
      if (valid && i < nn) {
        acc = H::from(sBb[i]);
#pragma unroll
        for (int j = 0; j < kMaxC; ++j)
          if (j < mm) acc = H::sub_prod(acc, sJb[j * nn + i], xs[j]);
      }
      res[r] = acc;
    }
    T g[kMaxC];
#pragma unroll
    for (int j = 0; j < kMaxC; ++j) {
      g[j] = 0;
      if (j < mw) {
        typename H::acc acc = H::zero();
#pragma unroll
        for (int r = 0; r < kRPL; ++r) {
          const int i = q + kG * r;
          if (valid && j < mm && i < nn) acc = H::add_prod_acc(acc, sJb[j * nn + i], res[r]);
        }
        acc = H::add(acc, H::shfl_xor(acc, 1));
        acc = H::add(acc, H::shfl_xor(acc, 2));
        g[j] = H::round(acc);
      }
    }
    // h = R^{-T} g (forward substitution; h_i of the lane's own rows kept in hl)
    T hl[kRPL];
#pragma unroll
    for (int r = 0; r < kRPL; ++r) hl[r] = 0;
#pragma unroll
    for (int k = 0; k < kMaxC; ++k) {
      if (k < mw) {
        T part = 0;
#pragma unroll
        for (int r = 0; r < kRPL; ++r) {
          const int i = q + kG * r;
          if (i < k) part += a[r][k] * hl[r];
        }
        part = group_sum(part);
        const T rkk = __shfl_sync(0xffffffffu, a[k / kG][k], gbase + (k % kG));
        T hk = (k < mm) ? (g[k] - part) / rkk : T(0);
        if (q == (k % kG)) hl[k / kG] = hk;
      }
    }
    // dx = R^{-1} h (back-substitution with h in place of c)
    T dx[kMaxC];
#pragma unroll
    for (int k = kMaxC - 1; k >= 0; --k) {
      dx[k] = 0;
      if (k < mw) {
        T s = hl[k / kG];
#pragma unroll
        for (int j = k + 1; j < kMaxC; ++j)
          if (j < mw) s -= a[k / kG][j] * dx[j];
        T d = s / a[k / kG][k];
        d = __shfl_sync(0xffffffffu, d, gbase + (k % kG));
        dx[k] = (k < mm) ? d : T(0);
      }
    }
#pragma unroll
    for (int k = 0; k < kMaxC; ++k) xs[k] += dx[k];
  }
  if (bad) record(status, QRKIT_ESINGULAR);
}

template <typename T, int HK>
__global__ void __launch_bounds__(kThreads)
block_solve_kernel(BlockSolveArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int VN = Vec16<T>::n;
  Smem<T> S;
  {
    size_t off = 0;
    S.J = reinterpret_cast<T*>(smem_raw + off);
    off += (size_t)(A.vb + VN) * sizeof(T);
    S.b = reinterpret_cast<T*>(smem_raw + off);
    off += (size_t)(A.rb + VN) * sizeof(T);
    S.tau = reinterpret_cast<T*>(smem_raw + off);
    off += (size_t)(A.cb + VN) * sizeof(T);
    S.x = reinterpret_cast<T*>(smem_raw + off);
    off += (size_t)(A.cb + VN) * sizeof(T);
    S.n = smem_raw + off;
    off += (size_t)((A.bb + 15) / 16 * 16);
    S.m = smem_raw + off;
    off += (size_t)((A.bb + 15) / 16 * 16);
    S.vo = reinterpret_cast<int*>(smem_raw + off);
    off += (size_t)(A.bb + 1) * sizeof(int);
    S.ro = reinterpret_cast<int*>(smem_raw + off);
    off += (size_t)(A.bb + 1) * sizeof(int);
    S.co = reinterpret_cast<int*>(smem_raw + off);
    off += (size_t)(A.bb + 1) * sizeof(int);
    S.wtot = reinterpret_cast<int*>(smem_raw + off);
  }
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int q = lane & (kG - 1);
  const int gbase = lane & ~(kG - 1);
  const int gid = tid / kG;
  constexpr int kGroups = kThreads / kG;

  for (int64_t t = blockIdx.x; t < A.num_tiles; t += gridDim.x) {
    const int64_t b0 = A.tile_block[t];
    const int nb = (int)(A.tile_block[t + 1] - b0);
    const int64_t v0 = A.tile_val[t], r0 = A.tile_row[t], c0 = A.tile_col[t];
    const int64_t nv = A.tile_val[t + 1] - v0, nr = A.tile_row[t + 1] - r0,
                  nc = A.tile_col[t + 1] - c0;
    for (int i = tid; i < nb; i += kThreads) {
      S.n[i] = A.n[b0 + i];
      S.m[i] = A.m[b0 + i];
    }
    __syncthreads();
    tile_scan3(nb, S.n, S.m, S.vo, S.ro, S.co, S.wtot);
    // offset the staging buffers so global and shared addresses agree modulo 16 bytes
    T* sJ = S.J + ((reinterpret_cast<uintptr_t>(A.J + v0) & 15) / sizeof(T));
    T* sB = S.b + ((reinterpret_cast<uintptr_t>(A.b + r0) & 15) / sizeof(T));
    T* sTau = S.tau + ((reinterpret_cast<uintptr_t>(A.tau + c0) & 15) / sizeof(T));
    T* sX = S.x + ((reinterpret_cast<uintptr_t>(A.x + c0) & 15) / sizeof(T));
    copy_in(sJ, A.J + v0, nv);
    copy_in(sB, A.b + r0, nr);
    __syncthreads();

    for (int base = 0; base < nb; base += kGroups) {
      const int bi = base + gid;
      const bool valid = bi < nb;
      const int nn = valid ? S.n[bi] : 0;
      const int mm = valid ? S.m[bi] : 0;
      int mw = mm;
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) mw = max(mw, __shfl_xor_sync(0xffffffffu, mw, d));
      const int vo = valid ? S.vo[bi] : 0;
      const int ro = valid ? S.ro[bi] : 0;
      const int co = valid ? S.co[bi] : 0;
      const T* sJb = sJ + vo;
      const T* sBb = sB + ro;
      T a[kRPL][kMaxC];
      T bb[kRPL];
#pragma unroll
      for (int r = 0; r < kRPL; ++r) {
        const int i = q + kG * r;
        bb[r] = (i < nn) ? sBb[i] : T(0);
#pragma unroll
        for (int j = 0; j < kMaxC; ++j) a[r][j] = (j < mm && i < nn) ? sJb[j * nn + i] : T(0);
      }
      T taus[kMaxC], xs[kMaxC];
#pragma unroll
      for (int j = 0; j < kMaxC; ++j) { taus[j] = 0; xs[j] = 0; }
      factor_solve_group<T, HK>(q, gbase, nn, mm, mw, valid, a, bb, taus, xs, sJb, sBb,
                                A.refine_steps, A.status);
      // results back to the staging buffers: factor in place of J, Q^T b in place of b
      if (valid) {
#pragma unroll
        for (int r = 0; r < kRPL; ++r) {
          const int i = q + kG * r;
          if (i < nn) {
            T* col = const_cast<T*>(sJb);
#pragma unroll
            for (int j = 0; j < kMaxC; ++j)
              if (j < mm) col[j * nn + i] = a[r][j];
            const_cast<T*>(sBb)[i] = bb[r];
          }
        }
        if (q == 0) {
#pragma unroll
          for (int j = 0; j < kMaxC; ++j)
            if (j < mm) {
              sTau[co + j] = taus[j];
              sX[co + j] = xs[j];
            }
        }
      }
    }
    __syncthreads();
    copy_out(A.F + v0, sJ, nv);
    if (A.qtb) copy_out(A.qtb + r0, sB, nr);
    copy_out(A.tau + c0, sTau, nc);
    copy_out(A.x + c0, sX, nc);
    __syncthreads();
  }
}

template <typename T, int HK>
qrkit_status launch_typed(qrkit_ctx* ctx, const void* J, const void* b, void* p, void* qtb,
                          int refine_steps) {
  Plan& P = ctx->plan;
  BlockSolveArgs<T> A;
  A.n = (const uint8_t*)P.d_n.ptr;
  A.m = (const uint8_t*)P.d_m.ptr;
  A.tile_block = (const int64_t*)P.d_tile_block.ptr;
  A.tile_val = (const int64_t*)P.d_tile_val.ptr;
  A.tile_row = (const int64_t*)P.d_tile_row.ptr;
  A.tile_col = (const int64_t*)P.d_tile_col.ptr;
  A.num_tiles = P.num_tiles;
  A.J = (const T*)J;
  A.b = (const T*)b;
  A.F = (T*)ctx->ws.factor.ptr;
  A.tau = (T*)ctx->ws.tau.ptr;
  A.qtb = (T*)qtb;
  A.x = (T*)p;
  A.refine_steps = refine_steps;
  A.status = ctx->d_status;
  A.vb = P.budget.values;
  A.rb = P.budget.rows;
  A.cb = P.budget.cols;
  A.bb = P.budget.blocks;
  const size_t smem = smem_bytes<T>(A.vb, A.rb, A.cb, A.bb);
  auto kern = block_solve_kernel<T, HK>;
  QRKIT_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
  int per_sm = 0;
  QRKIT_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)ctx->num_sms * per_sm;
  if (grid > P.num_tiles) grid = P.num_tiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kThreads, smem, ctx->stream>>>(A);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  return QRKIT_OK;
}

}  // namespace

TileBudget block_solve_budget(size_t elem) {
  TileBudget b;
  b.blocks = kThreads;
  if (elem == sizeof(float)) {
    b.values = 8192; b.rows = 4096; b.cols = 2048;
  } else {
    b.values = 4096; b.rows = 2048; b.cols = 1024;
  }
  return b;
}

int block_solve_max_rows() { return kG * kRPL; }
int block_solve_max_cols() { return kMaxC; }

qrkit_status launch_block_solve(qrkit_ctx* ctx, const void* J, const void* b, const void* D,
                                void* p, void* qtb, int refine_steps) {
  (void)D;
  if (ctx->precision == QRKIT_FP64) return launch_typed<double, 0>(ctx, J, b, p, qtb, refine_steps);
  const int steps = ctx->precision == QRKIT_FP32 ? 0 : refine_steps;
  return launch_typed<float, 1>(ctx, J, b, p, qtb, steps);
}

}  // namespace qrkit
