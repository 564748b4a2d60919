// Batched block-diagonal QR solve (Sec. 4.1 "Block diagonal", Sec. 5.1 solver interface),
// fused: factor + Q^T b + back-substitution + refinement in one pass over HBM.
//
// Work mapping (GB300): one launch; each CTA factors one tile of consecutive blocks (cut by
// the plan so a tile fits the shared-memory budget) and several CTAs share an SM, so the
// load, sort, factor and store phases of different tiles overlap.  A tile's J values and b
// are staged in shared memory by TMA bulk copies (cp.async.bulk + mbarrier) while the
// block shapes are scanned and sorted; results leave with coalesced vector stores.  Inside a tile the blocks are counting-sorted by (row
// class, column count) so that each warp works on blocks of one shape class: blocks of
// <= 4 rows get one lane, <= 8 rows two lanes, <= 16 rows four lanes; lane q of a group
// holds rows 4q .. 4q+3 of the column being processed, the columns stay in shared memory
// and are swept by runtime loops (compact code), and Householder norms and dot products
// are shuffle reductions over the group.
//
// Reflector convention (Sec. 2): H = I - tau v v^T, v[0] = 1, beta = -sign(x0) ||x||.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>
#include <type_traits>

#include "device_util.cuh"
#include "internal.h"

namespace qrkit {
namespace {

using namespace dev;

constexpr int kMaxRows = 16;   // rows per block (one lane, padded to 4, 8, 12 or 16)
constexpr int kMaxCols = 8;    // columns per block
constexpr int kThreads = 256;  // threads per CTA
constexpr float kUnitRoundoff = 5.9604645e-8f;   // 2^-24
constexpr float kRefineTarget = 1e-6f;           // blocks estimated above this are refined
constexpr int kKeys = 36;      // sort keys: 4 row classes x (m = 0..8)
constexpr long long kDrainPolls = 1LL << 26;   // polls of the wait for a CTA's own copies after a timeout
static_assert(kKeys <= 64, "the bin scan handles at most 64 keys");

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

// Row class of an n-row block: its rows are padded to R = 4 (class + 1) in the working area.
__host__ __device__ inline int row_class(int n) { return (n - 1) >> 2; }
__host__ __device__ inline int padded_rows(int n) { return 4 * (row_class(n) + 1); }

// Exclusive scans over a tile (nb <= kThreads) of the per-block value, row, column and
// padded-working-area counts.
__device__ __forceinline__ void tile_scan4(int nb, const uint8_t* sN, const uint8_t* sM,
                                           int* sVo, int* sRo, int* sCo, int* sPo, int* warp_tot) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nn = tid < nb ? sN[tid] : 0;
  const int mm = tid < nb ? sM[tid] : 0;
  const int v = nn * mm, r = nn, c = mm, pp = tid < nb ? padded_rows(nn) * mm : 0;
  int iv = v, ir = r, ic = c, ip = pp;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int tv = __shfl_up_sync(0xffffffffu, iv, d);
    const int tr = __shfl_up_sync(0xffffffffu, ir, d);
    const int tc = __shfl_up_sync(0xffffffffu, ic, d);
    const int tp = __shfl_up_sync(0xffffffffu, ip, d);
    if (lane >= d) { iv += tv; ir += tr; ic += tc; ip += tp; }
  }
  if (lane == 31) {
    warp_tot[wid * 4 + 0] = iv;
    warp_tot[wid * 4 + 1] = ir;
    warp_tot[wid * 4 + 2] = ic;
    warp_tot[wid * 4 + 3] = ip;
  }
  __syncthreads();
  int bv = 0, br = 0, bc = 0, bp = 0;
  for (int w = 0; w < wid; ++w) {
    bv += warp_tot[w * 4 + 0];
    br += warp_tot[w * 4 + 1];
    bc += warp_tot[w * 4 + 2];
    bp += warp_tot[w * 4 + 3];
  }
  if (tid < nb) {
    sVo[tid] = bv + iv - v;
    sRo[tid] = br + ir - r;
    sCo[tid] = bc + ic - c;
    sPo[tid] = bp + ip - pp;
  }
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
  int refine_steps;      // at most this many refinement steps per block
  float refine_tol;      // stop when max|dx| <= refine_tol * max|x|
  int* status;
  int vb, rb, cb, bb, pb;  // tile budgets (pb: padded working area)
  long long wait_limit;  // polls of an mbarrier before giving up
  int* rlist;            // selection mode: blocks to refine, 4 row-class lists of rcap entries
  int* rcount;           // their lengths (4)
  int64_t rcap;
};

// Shared-memory layout (identical on host and device).  Each block is factored in a padded
// working area W (column stride = rows covered by its lane group, 16-byte aligned), then
// written back in packed form over the J buffer, which stages the factor for the store.
// Without refinement Q^T b is formed in place in the b buffer.
struct Layout {
  size_t J, b, n, m, W, Cw, rs, c, tau, x, g, vo, ro, co, po, qo, wtot, perm, hist, sel, bar, total;
};
__host__ __device__ inline size_t round16(size_t v) { return (v + 15) / 16 * 16; }
template <typename T>
__host__ __device__ inline Layout make_layout(int vb, int rb, int cb, int bb, int pb, bool refine,
                                             bool select = false) {
  const int VN = 16 / (int)sizeof(T);
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += round16(bytes); return o; };
  L.J = take((size_t)(vb + 2 * VN) * sizeof(T));
  L.b = take((size_t)(rb + 2 * VN) * sizeof(T));
  L.n = take((size_t)bb);
  L.m = take((size_t)bb);
  L.W = take((size_t)pb * sizeof(T));
  L.Cw = 0;
  L.rs = refine ? take((size_t)2 * (rb + 3 * bb) * sizeof(T)) : 0;   // residual scratch
  L.c = refine ? take((size_t)(rb + 2 * VN) * sizeof(T)) : 0;
  L.tau = take((size_t)(cb + 2 * VN) * sizeof(T));
  L.x = take((size_t)(cb + 2 * VN) * sizeof(T));
  L.g = refine ? take((size_t)(cb + 2 * VN) * sizeof(T)) : 0;
  L.vo = take((size_t)(bb + 1) * sizeof(int));
  L.ro = take((size_t)(bb + 1) * sizeof(int));
  L.co = take((size_t)(bb + 1) * sizeof(int));
  L.po = take((size_t)(bb + 1) * sizeof(int));
  L.qo = take((size_t)(bb + 1) * sizeof(int));
  L.wtot = take((size_t)(32 + kThreads / 32) * sizeof(int));
  L.perm = take((size_t)bb * sizeof(int));
  L.hist = take((size_t)(2 * kKeys + 8) * sizeof(int));
  L.sel = select ? take((size_t)(bb + 16) * sizeof(int)) : 0;   // selected blocks + counters
  L.bar = take(sizeof(uint64_t));
  L.total = off;
  return L;
}

// Four consecutive rows of one column (the rows one lane owns), moved with one 16-byte
// (float) or two 16-byte (double) shared-memory accesses.
template <typename T>
struct Row4 {
  T v[4];
};
__device__ __forceinline__ Row4<float> ld4(const float* p) {
  const float4 f = *reinterpret_cast<const float4*>(p);
  return Row4<float>{{f.x, f.y, f.z, f.w}};
}
__device__ __forceinline__ Row4<double> ld4(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  return Row4<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, const Row4<float>& r) {
  *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
}
__device__ __forceinline__ void st4(double* p, const Row4<double>& r) {
  reinterpret_cast<double2*>(p)[0] = make_double2(r.v[0], r.v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(r.v[2], r.v[3]);
}

// x = R^{-1} c (R on and above the diagonal of the factor F, column stride cs); one lane.
template <typename T>
__device__ __forceinline__ bool back_substitute(const T* F, int cs, int mm, const T* c, T* x) {
  bool ok = true;
  for (int k = mm - 1; k >= 0; --k) {
    T s = c[k];
    for (int j = k + 1; j < mm; ++j) s -= F[j * cs + k] * x[j];
    const T rkk = F[k * cs + k];
    ok = ok && rkk != T(0);
    x[k] = s * frcp(rkk);
  }
  return ok;
}

// One lane factors one n x m block (Sec. 2) held in the padded working area W: column j at
// W + j * R (R = rows padded to a multiple of 4, zeros below row n), factored in place (V
// below the diagonal, R on and above).  The lane's rhs rows live in registers while the
// reflectors are applied (Q^T b).  Pivots are read as scalars from shared memory, so every
// register array is indexed by compile-time constants.  One instantiation per row class.
template <typename T, int R>
__device__ __forceinline__ void lane_householder(T* W, int mm, T (&bb)[R], T* tau_out) {
  for (int k = 0; k < mm; ++k) {
    T* colk = W + k * R;
    T c[R];
#pragma unroll
    for (int r = 0; r < R; r += 4) {
      const Row4<T> x = ld4(colk + r);
      c[r] = x.v[0]; c[r + 1] = x.v[1]; c[r + 2] = x.v[2]; c[r + 3] = x.v[3];
    }
    T sq = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) sq += (r > k) ? c[r] * c[r] : T(0);
    const T alpha = colk[k];
    const T norm = fsqrt(alpha * alpha + sq);
    T beta = 0, tau = 0, scale = 0;
    if (norm != T(0)) {
      beta = alpha >= T(0) ? -norm : norm;
      const T d = alpha - beta;
      scale = frcp(d);
      tau = -d * frcp(beta);
    }
    T v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = (r == k) ? T(1) : ((r > k) ? c[r] * scale : T(0));
#pragma unroll
    for (int r = 0; r < R; r += 4) {
      Row4<T> o;
#pragma unroll
      for (int u = 0; u < 4; ++u) o.v[u] = (r + u > k) ? v[r + u] : c[r + u];
      st4(colk + r, o);
    }
    colk[k] = beta;
    tau_out[k] = tau;
    for (int j = k + 1; j < mm; ++j) {
      T* colj = W + j * R;
      T d[R];
#pragma unroll
      for (int r = 0; r < R; r += 4) {
        const Row4<T> x = ld4(colj + r);
        d[r] = x.v[0]; d[r + 1] = x.v[1]; d[r + 2] = x.v[2]; d[r + 3] = x.v[3];
      }
      T w = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) w += v[r] * d[r];
      w *= tau;
#pragma unroll
      for (int r = 0; r < R; r += 4) {
        Row4<T> o;
#pragma unroll
        for (int u = 0; u < 4; ++u) o.v[u] = d[r + u] - v[r + u] * w;
        st4(colj + r, o);
      }
    }
    T w = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) w += v[r] * bb[r];
    w *= tau;
#pragma unroll
    for (int r = 0; r < R; ++r) bb[r] -= v[r] * w;
  }
}

// Refinement of a float block by one lane: g = J^T (b - J x) with the residual in
// compensated float arithmetic (Dot2 of Ogita, Rump and Oishi: error-free products and
// sums, value = s + c), then dx = R^{-1} R^{-T} g and x += dx.  With the residual taken
// exactly this is the first step of Bjorck's augmented-system refinement from (x, b - J x).
// Rp: padded row stride of F; rs: scratch of 2 * Rp floats for the residual.  Only the
// ceil(n / 4) row groups that hold rows are touched (nothing at all for n = 0).
// Returns max |dx| / max |x|.
__device__ __noinline__ float lane_refine(int nn, int Rp, int mm, const float* J,
                                             const float* b, const float* F, float* x,
                                             float* g, float* rs) {
  const int ng = (nn + 3) >> 2;
  // residual rows, four at a time
  for (int q = 0; q < ng; ++q) {
    float sh[4], sl[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      sh[u] = (4 * q + u < nn) ? b[4 * q + u] : 0.f;
      sl[u] = 0.f;
    }
    for (int j = 0; j < mm; ++j) {
      const float xj = -x[j];
      const float* Jj = J + j * nn;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (4 * q + u < nn) {
          const float a = Jj[4 * q + u];
          const float p = __fmul_rn(a, xj);
          const float pe = __fmaf_rn(a, xj, -p);
          float t, e;
          two_sum(sh[u], p, t, e);
          sh[u] = t;
          sl[u] = __fadd_rn(sl[u], __fadd_rn(e, pe));
        }
      }
    }
    st4(rs + 4 * q, Row4<float>{{sh[0], sh[1], sh[2], sh[3]}});
    st4(rs + Rp + 4 * q, Row4<float>{{sl[0], sl[1], sl[2], sl[3]}});
  }
  // g_j = sum_i J_ij r_i
  for (int j = 0; j < mm; ++j) {
    const float* Jj = J + j * nn;
    float s = 0.f, c = 0.f;
    for (int q = 0; q < ng; ++q) {
      const Row4<float> rh = ld4(rs + 4 * q);
      const Row4<float> rl = ld4(rs + Rp + 4 * q);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (4 * q + u < nn) {
          const float a = Jj[4 * q + u];
          const float p = __fmul_rn(a, rh.v[u]);
          float pe = __fmaf_rn(a, rh.v[u], -p);
          pe = __fmaf_rn(a, rl.v[u], pe);
          float t, e;
          two_sum(s, p, t, e);
          s = t;
          c = __fadd_rn(c, __fadd_rn(e, pe));
        }
      }
    }
    g[j] = __fadd_rn(s, c);
  }
  for (int k = 0; k < mm; ++k) {          // h = R^{-T} g, in place
    float s = g[k];
    for (int i = 0; i < k; ++i) s -= F[k * Rp + i] * g[i];
    g[k] = s * frcp(F[k * Rp + k]);
  }
  for (int k = mm - 1; k >= 0; --k) {     // dx = R^{-1} h, in place
    float s = g[k];
    for (int j = k + 1; j < mm; ++j) s -= F[j * Rp + k] * g[j];
    g[k] = s * frcp(F[k * Rp + k]);
  }
  float dmax = 0.f, xmax = 0.f;
  for (int k = 0; k < mm; ++k) {
    const float xn = x[k] + g[k];
    x[k] = xn;
    dmax = fmaxf(dmax, fabsf(g[k]));
    xmax = fmaxf(xmax, fabsf(xn));
  }
  return xmax > 0.f ? dmax / xmax : 0.f;
}

// A-priori error estimate of a block's float least-squares solution (Householder QR is
// backward stable: relative error ~ u (kappa + kappa^2 ||r|| / (||A|| ||x||))), with
// ||A|| ~ ||R||_F, ||R^{-1}||_2^2 from two power steps v <- R^{-1} R^{-T} v (from below) and
// ||r|| = || rows m.. of Q^T b ||; true when the estimate exceeds kRefineTarget.  W: the
// factor (R on and above the diagonal, column stride R), c: Q^T b.  Register-resident: the
// loops run to the 8-column bound with predicates.
template <int R>
__device__ __forceinline__ bool needs_refinement(int nn, int mm, const float* W, const float (&c)[R],
                                                 const float* x) {
  if (mm <= 0) return false;
  float rF2 = 0.f, x2 = 0.f, res2 = 0.f;
  float d[kMaxCols], v[kMaxCols];
#pragma unroll
  for (int k = 0; k < kMaxCols; ++k) {
    const bool on = k < mm;
    d[k] = on ? frcp(W[k * R + k]) : 0.f;
    v[k] = on ? 1.f : 0.f;
    if (on) x2 += x[k] * x[k];
#pragma unroll
    for (int i = 0; i <= k; ++i)
      if (on) rF2 += W[k * R + i] * W[k * R + i];
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r >= mm && r < nn) res2 += c[r] * c[r];
  float vn2 = (float)mm, inv2 = 0.f;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float sc = rsqrtf(vn2);
#pragma unroll
    for (int k = 0; k < kMaxCols; ++k) {   // R^T w = v / ||v||
      float t = v[k] * sc;
#pragma unroll
      for (int i = 0; i < k; ++i) t -= W[k * R + i] * v[i];
      v[k] = k < mm ? t * d[k] : 0.f;
    }
#pragma unroll
    for (int k = kMaxCols - 1; k >= 0; --k) {   // R v' = w
      float t = v[k];
#pragma unroll
      for (int j = k + 1; j < kMaxCols; ++j) t -= (j < mm ? W[j * R + k] : 0.f) * v[j];
      v[k] = k < mm ? t * d[k] : 0.f;
    }
    vn2 = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxCols; ++k) vn2 += v[k] * v[k];
    inv2 = sqrtf(vn2);
  }
  const float rF = sqrtf(rF2);
  const float est = kUnitRoundoff * (rF * sqrtf(inv2) + rF * inv2 * sqrtf(res2 / x2));
  return !(est <= kRefineTarget);   // NaN (x = 0, zero pivot) refines
}

// Everything one lane does for one block: padded copy in, factor, Q^T b, back-substitution,
// adaptive refinement (until the correction is below refine_tol relative to x, at most
// max_steps), packed copy of the factor out (Fout, may alias J: written last).  All 32
// lanes of the warp call it (lanes without a block pass nn = mm = 0) and every phase ends in
// __syncwarp(), so lanes whose loops ran for different lengths reconverge.  The refinement
// is one shared (not inlined) routine for every row class, which keeps the code that warps
// loop back into small.  rs: scratch of 2 * R floats for the residual.
template <typename T, bool REF, int R, bool SEL = false>
__device__ __forceinline__ bool lane_block(int nn, int mm, const T* J, const T* b, T* W, T* C,
                                           T* tau, T* x, T* g, T* rs, T* Fout, int max_steps,
                                           float refine_tol, int* status) {
  for (int j = 0; j < mm; ++j) {
#pragma unroll
    for (int r = 0; r < R; r += 4) {
      Row4<T> o;
#pragma unroll
      for (int u = 0; u < 4; ++u) o.v[u] = (r + u < nn) ? J[j * nn + r + u] : T(0);
      st4(W + j * R + r, o);
    }
  }
  T bb[R];
#pragma unroll
  for (int r = 0; r < R; ++r) bb[r] = (r < nn) ? b[r] : T(0);
  lane_householder<T, R>(W, mm, bb, tau);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r < nn) C[r] = bb[r];
  if (!back_substitute(W, R, mm, C, x)) record(status, QRKIT_ESINGULAR);
  __syncwarp();
  bool need = false;
  if constexpr (SEL) need = needs_refinement<R>(nn, mm, W, bb, x);
  if constexpr (REF) {
    for (int step = 0; step < max_steps; ++step) {
      const float rel = lane_refine(nn, R, mm, J, b, W, x, g, rs);
      if (!(rel > refine_tol)) break;
    }
    __syncwarp();
  }
  if (Fout) {
    for (int j = 0; j < mm; ++j)
      for (int r = 0; r < nn; ++r) Fout[j * nn + r] = W[j * R + r];
  }
  __syncwarp();
  return need;
}

// Per-tile geometry shared by the issue, compute and store phases.
template <typename T>
struct TileGeo {
  int64_t b0, v0, r0, c0;
  int nb, nv, nr, nc;
  int offJ, offB;   // shared-memory element offsets (alignment to global)
};

template <typename T>
__device__ __forceinline__ TileGeo<T> tile_geo(const BlockSolveArgs<T>& A, int64_t t) {
  TileGeo<T> g;
  g.b0 = A.tile_block[t];
  g.nb = (int)(A.tile_block[t + 1] - g.b0);
  g.v0 = A.tile_val[t];
  g.r0 = A.tile_row[t];
  g.c0 = A.tile_col[t];
  g.nv = (int)(A.tile_val[t + 1] - g.v0);
  g.nr = (int)(A.tile_row[t + 1] - g.r0);
  g.nc = (int)(A.tile_col[t + 1] - g.c0);
  g.offJ = align_off(A.J + g.v0);
  g.offB = align_off(A.b + g.r0);
  return g;
}

// Thread 0: start the bulk loads of a tile's J and b interiors.
template <typename T>
__device__ __forceinline__ void issue_tile_load(const BlockSolveArgs<T>& A, const TileGeo<T>& g,
                                                T* sJ, T* sB, uint64_t* bar) {
  int hJ, nJ, hB, nB;
  interior(A.J + g.v0, g.nv, hJ, nJ);
  interior(A.b + g.r0, g.nr, hB, nB);
  const uint32_t bytes = (uint32_t)(nJ + nB) * sizeof(T);
  fence_proxy_async();
  mbar_expect_tx(bar, bytes);
  if (nJ) bulk_g2s(sJ + g.offJ + hJ, A.J + g.v0 + hJ, (uint32_t)nJ * sizeof(T), bar);
  if (nB) bulk_g2s(sB + g.offB + hB, A.b + g.r0 + hB, (uint32_t)nB * sizeof(T), bar);
}

// All threads: plain loads of what the bulk copies leave out (unaligned head and tail
// elements) and of the tile's block shapes.
template <typename T>
__device__ __forceinline__ void load_tile_edges(const BlockSolveArgs<T>& A, const TileGeo<T>& g,
                                                T* sJ, T* sB, uint8_t* sN, uint8_t* sM) {
  int hJ, nJ, hB, nB;
  interior(A.J + g.v0, g.nv, hJ, nJ);
  interior(A.b + g.r0, g.nr, hB, nB);
  const int tid = threadIdx.x;
  const int tJ = g.nv - (hJ + nJ);
  for (int k = tid; k < hJ + tJ; k += kThreads) {
    const int e = k < hJ ? k : hJ + nJ + (k - hJ);
    sJ[g.offJ + e] = A.J[g.v0 + e];
  }
  const int tB = g.nr - (hB + nB);
  for (int k = tid; k < hB + tB; k += kThreads) {
    const int e = k < hB ? k : hB + nB + (k - hB);
    sB[g.offB + e] = A.b[g.r0 + e];
  }
  for (int k = tid; k < g.nb; k += kThreads) {
    sN[k] = A.n[g.b0 + k];
    sM[k] = A.m[g.b0 + k];
  }
}

// Coalesced copy shared -> global; vector stores when both sides agree modulo 16 bytes.
template <typename T>
__device__ __forceinline__ void store_out(T* __restrict__ dst, const T* src, int count) {
  using V = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::n;
  const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
  if (((a ^ reinterpret_cast<uintptr_t>(src)) & 15) != 0) {
    for (int k = threadIdx.x; k < count; k += kThreads) dst[k] = src[k];
    return;
  }
  int head = (int)(((16 - (a & 15)) & 15) / sizeof(T));
  if (head > count) head = count;
  for (int k = threadIdx.x; k < head; k += kThreads) dst[k] = src[k];
  const int nvec = (count - head) / VN;
  V* vd = reinterpret_cast<V*>(dst + head);
  const V* vs = reinterpret_cast<const V*>(src + head);
  for (int k = threadIdx.x; k < nvec; k += kThreads) __stcs(vd + k, vs[k]);
  for (int k = head + nvec * VN + threadIdx.x; k < count; k += kThreads) dst[k] = src[k];
}

template <typename T, bool REF, bool SEL = false>
__global__ void __launch_bounds__(kThreads, 3)
block_solve_kernel(BlockSolveArgs<T> A) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Layout L = make_layout<T>(A.vb, A.rb, A.cb, A.bb, A.pb, REF, SEL);
  int* sVo = reinterpret_cast<int*>(smem_raw + L.vo);
  int* sRo = reinterpret_cast<int*>(smem_raw + L.ro);
  int* sCo = reinterpret_cast<int*>(smem_raw + L.co);
  int* sPo = reinterpret_cast<int*>(smem_raw + L.po);
  int* sQo = reinterpret_cast<int*>(smem_raw + L.qo);
  T* sRs = reinterpret_cast<T*>(smem_raw + L.rs);
  int* sW = reinterpret_cast<int*>(smem_raw + L.wtot);
  int* sPerm = reinterpret_cast<int*>(smem_raw + L.perm);
  int* sHist = reinterpret_cast<int*>(smem_raw + L.hist);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + L.bar);
  uint8_t* sNs = smem_raw + L.n;
  uint8_t* sMs = smem_raw + L.m;
  T* sWork = reinterpret_cast<T*>(smem_raw + L.W);

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp_id = tid >> 5;
  const int64_t t = blockIdx.x;   // one tile per CTA; several CTAs per SM overlap their phases
  if (t >= A.num_tiles) return;
  const TileGeo<T> g = tile_geo(A, t);
  T* sJ = reinterpret_cast<T*>(smem_raw + L.J) + g.offJ;
  T* sB = reinterpret_cast<T*>(smem_raw + L.b) + g.offB;
  // (A) bulk loads of the J and b interiors (TMA), plain loads of the edges and shapes
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    issue_tile_load(A, g, reinterpret_cast<T*>(smem_raw + L.J), reinterpret_cast<T*>(smem_raw + L.b), bar);
  }
  load_tile_edges(A, g, reinterpret_cast<T*>(smem_raw + L.J), reinterpret_cast<T*>(smem_raw + L.b), sNs, sMs);
  for (int k = tid; k < 2 * kKeys; k += kThreads) sHist[k] = 0;
  __syncthreads();
  // (B) per-block offsets and the counting sort by (row class, m) while the copy lands
  tile_scan4(g.nb, sNs, sMs, sVo, sRo, sCo, sPo, sW);
  __syncthreads();
  // padded-row offsets (rows rounded up to 4): a second scan over the tile
  {
    const int lane_ = tid & 31, wid = tid >> 5;
    const int pr = tid < g.nb ? padded_rows(sNs[tid]) : 0;
    int inc = pr;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane_ >= d) inc += o;
    }
    if (lane_ == 31) sW[32 + wid] = inc;
    __syncthreads();
    int base = 0;
    for (int w = 0; w < wid; ++w) base += sW[32 + w];
    if (tid < g.nb) sQo[tid] = base + inc - pr;
  }
  int myrank = 0, mykey = 0;
  if (tid < g.nb) {
    const int nn = sNs[tid], mm = sMs[tid];
    mykey = row_class(nn) * 9 + mm;
    myrank = atomicAdd(&sHist[mykey], 1);
  }
  __syncthreads();
  if (tid < 32) {
    // exclusive scan of the kKeys (<= 64) bins: two bins per lane
    const int v0 = 2 * tid < kKeys ? sHist[2 * tid] : 0;
    const int v1 = 2 * tid + 1 < kKeys ? sHist[2 * tid + 1] : 0;
    int inc = v0 + v1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, inc, d);
      if (tid >= d) inc += o;
    }
    const int excl = inc - v0 - v1;
    if (2 * tid < kKeys) sHist[kKeys + 2 * tid] = excl;
    if (2 * tid + 1 < kKeys) sHist[kKeys + 2 * tid + 1] = excl + v0;
  }
  __syncthreads();
  if (tid < g.nb) sPerm[sHist[kKeys + mykey] + myrank] = tid;
  // (C) wait for the bulk loads (bounded)
  bool ok = false;
  for (long long polls = 0; polls < A.wait_limit; ++polls) {
    if (mbar_try_wait(bar, 0u)) { ok = true; break; }
  }
  if (__syncthreads_or(!ok)) {
    if (tid == 0) record(A.status, QRKIT_ETIMEOUT);
    // the bulk loads may still be in flight: wait for them once more, with a limit of its own
    // (the first limit may be as small as zero), before the CTA's shared memory is given up
    for (long long polls = 0; polls < kDrainPolls; ++polls)
      if (mbar_try_wait(bar, 0u)) break;
    return;
  }
  // staging of the results: the factor goes back over J (packed), Q^T b over b unless the
  // refinement still needs b
  const int offF = align_off(A.F + g.v0);
  T* sF = reinterpret_cast<T*>(smem_raw + L.J) + offF;
  const bool f_alias = offF == g.offJ;   // same alignment: factor written in place of J
  const int offC = A.qtb ? align_off(A.qtb + g.r0) : g.offB;
  T* sC = REF ? reinterpret_cast<T*>(smem_raw + L.c) + offC : sB;
  T* sT = reinterpret_cast<T*>(smem_raw + L.tau) + align_off(A.tau + g.c0);
  T* sX = reinterpret_cast<T*>(smem_raw + L.x) + align_off(A.x + g.c0);
  T* sG = REF ? reinterpret_cast<T*>(smem_raw + L.g) : nullptr;
  if (REF) {
    for (int k = tid; k < g.nr; k += kThreads) sC[k] = sB[k];
    __syncthreads();
  }
  // (D) factor + solve (+ refine): one lane per block, a warp takes 32 consecutive sorted
  // blocks of one row class (padded rows R = 4, 8, 12, 16)
  int cstart[4], ccount[4], nch[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    cstart[c] = sHist[kKeys + 9 * c];
    ccount[c] = (c < 3 ? sHist[kKeys + 9 * (c + 1)] : g.nb) - cstart[c];
    nch[c] = (ccount[c] + 31) >> 5;
  }
  const int total_chunks = nch[0] + nch[1] + nch[2] + nch[3];
  T* Fstage = f_alias ? sF : nullptr;
  int* sSel = SEL ? reinterpret_cast<int*>(smem_raw + L.sel) : nullptr;   // [0..15] counters
  if (SEL && tid < 16) sSel[tid] = 0;
  if (SEL) __syncthreads();
  for (int ch = warp_id; ch < total_chunks; ch += kThreads / 32) {
    int c = 0, first = ch;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      if (c == cc && first >= nch[cc]) { first -= nch[cc]; c = cc + 1; }
    const int cst = c == 0 ? cstart[0] : (c == 1 ? cstart[1] : (c == 2 ? cstart[2] : cstart[3]));
    const int ccn = c == 0 ? ccount[0] : (c == 1 ? ccount[1] : (c == 2 ? ccount[2] : ccount[3]));
    const int pos = first * 32 + lane;
    int bi = pos < ccn ? sPerm[cst + pos] : -1;
    if (pos < ccn && (bi < 0 || bi >= g.nb)) {   // cannot happen with a consistent sort
      record(A.status, QRKIT_EINVAL);
      bi = -1;
    }
    {
      // every lane takes part (lanes without a block: nn = mm = 0, nothing is touched)
      const bool has = bi >= 0;
      const int nn = has ? sNs[bi] : 0, mm = has ? sMs[bi] : 0;
      const int vo = has ? sVo[bi] : 0, ro = has ? sRo[bi] : 0, co = has ? sCo[bi] : 0;
      const int qo = has ? sQo[bi] : 0;
      T* Wb = sWork + (has ? sPo[bi] : 0);
      T* Fo = (Fstage && has) ? Fstage + vo : nullptr;
      T* gb = REF ? sG + co : nullptr;
      T* rsb = REF ? sRs + 2 * qo : nullptr;
      bool need;
      switch (c) {
        case 0: need = lane_block<T, REF, 4, SEL>(nn, mm, sJ + vo, sB + ro, Wb, sC + ro, sT + co, sX + co, gb, rsb, Fo, A.refine_steps, A.refine_tol, A.status); break;
        case 1: need = lane_block<T, REF, 8, SEL>(nn, mm, sJ + vo, sB + ro, Wb, sC + ro, sT + co, sX + co, gb, rsb, Fo, A.refine_steps, A.refine_tol, A.status); break;
        case 2: need = lane_block<T, REF, 12, SEL>(nn, mm, sJ + vo, sB + ro, Wb, sC + ro, sT + co, sX + co, gb, rsb, Fo, A.refine_steps, A.refine_tol, A.status); break;
        default: need = lane_block<T, REF, 16, SEL>(nn, mm, sJ + vo, sB + ro, Wb, sC + ro, sT + co, sX + co, gb, rsb, Fo, A.refine_steps, A.refine_tol, A.status); break;
      }
      if (SEL && has && need) sSel[16 + atomicAdd(&sSel[0], 1)] = (c << 28) | bi;
    }
  }
  __syncthreads();
  if constexpr (SEL) {
    // the selected blocks go to the global row-class lists: one atomic per class per tile
    const int total = sSel[0];
    for (int k = tid; k < total; k += kThreads) atomicAdd(&sSel[1 + (sSel[16 + k] >> 28)], 1);
    __syncthreads();
    if (tid < 4) sSel[5 + tid] = sSel[1 + tid] ? atomicAdd(&A.rcount[tid], sSel[1 + tid]) : 0;
    if (tid < 4) sSel[9 + tid] = 0;
    __syncthreads();
    for (int k = tid; k < total; k += kThreads) {
      const int e = sSel[16 + k], c = e >> 28, bi = e & 0x0FFFFFFF;
      const int64_t pos = (int64_t)sSel[5 + c] + atomicAdd(&sSel[9 + c], 1);
      if (pos < A.rcap) A.rlist[c * A.rcap + pos] = (int)(g.b0 + bi);
    }
  }
  if (!f_alias) {
    // the factor's staging cannot share J's alignment: write it from the working area
    for (int bi = tid; bi < g.nb; bi += kThreads) {
      const int nn = sNs[bi], mm = sMs[bi], R = padded_rows(nn);
      const T* Wb = sWork + sPo[bi];
      for (int j = 0; j < mm; ++j)
        for (int i = 0; i < nn; ++i) A.F[g.v0 + sVo[bi] + j * nn + i] = Wb[j * R + i];
    }
  }
  // (E) results to HBM with coalesced stores
  if (f_alias) store_out(A.F + g.v0, sF, g.nv);
  if (A.qtb) store_out(A.qtb + g.r0, sC, g.nr);
  store_out(A.tau + g.c0, sT, g.nc);
  store_out(A.x + g.c0, sX, g.nc);
}

// Refinement of the blocks the selection listed (one thread per block, grid-stride over the
// four row-class lists so that a warp's blocks share a row class): each step forms the
// residual r = b - J x and g = J^T r in compensated float arithmetic (TwoProduct by FMA,
// TwoSum), then x += R^{-1} R^{-T} g with the stored R; a block stops once its correction is
// below tol relative to x (max norms), after at most `steps` steps.
struct RefineArgs {
  const uint8_t* n;
  const uint8_t* m;
  const int64_t* val_off;
  const int64_t* row_off;
  const int64_t* col_off;
  const float* J;
  const float* b;
  const float* F;   // factor in J's packing: R on and above the diagonal
  float* x;
  const int* rlist;
  const int* rcount;
  int64_t rcap;
  int steps;
  float tol;
};

__global__ void __launch_bounds__(128) block_refine_kernel(RefineArgs A) {
  int64_t cnt[4], total = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    cnt[c] = A.rcount[c] < A.rcap ? A.rcount[c] : A.rcap;
    total += cnt[c];
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c = 0;
    int64_t pos = i;
    while (c < 3 && pos >= cnt[c]) {
      pos -= cnt[c];
      ++c;
    }
    const int64_t blk = A.rlist[c * A.rcap + pos];
    const int nn = A.n[blk], mm = A.m[blk];
    if (nn > kMaxRows || mm > kMaxCols || mm < 1) continue;
    const float* J = A.J + A.val_off[blk];
    const float* F = A.F + A.val_off[blk];
    const float* b = A.b + A.row_off[blk];
    float* xo = A.x + A.col_off[blk];
    float x[kMaxCols], rh[kMaxRows], rl[kMaxRows], h[kMaxCols];
    for (int j = 0; j < mm; ++j) x[j] = xo[j];
    for (int step = 0; step < A.steps; ++step) {
      for (int r = 0; r < nn; ++r) {
        float sh = b[r], sl = 0.f;
        for (int j = 0; j < mm; ++j) {
          const float a = J[j * nn + r], xj = -x[j];
          const float pr = __fmul_rn(a, xj);
          const float pe = __fmaf_rn(a, xj, -pr);
          float t, e;
          two_sum(sh, pr, t, e);
          sh = t;
          sl = __fadd_rn(sl, __fadd_rn(e, pe));
        }
        rh[r] = sh;
        rl[r] = sl;
      }
      for (int j = 0; j < mm; ++j) {
        float sj = 0.f, cj = 0.f;
        for (int r = 0; r < nn; ++r) {
          const float a = J[j * nn + r];
          const float pr = __fmul_rn(a, rh[r]);
          float pe = __fmaf_rn(a, rh[r], -pr);
          pe = __fmaf_rn(a, rl[r], pe);
          float t, e;
          two_sum(sj, pr, t, e);
          sj = t;
          cj = __fadd_rn(cj, __fadd_rn(e, pe));
        }
        h[j] = __fadd_rn(sj, cj);
      }
      for (int k = 0; k < mm; ++k) {   // R^T h = g
        float v = h[k];
        for (int i = 0; i < k; ++i) v -= F[k * nn + i] * h[i];
        h[k] = v / F[k * nn + k];
      }
      for (int k = mm - 1; k >= 0; --k) {   // R dx = h
        float v = h[k];
        for (int j = k + 1; j < mm; ++j) v -= F[j * nn + k] * h[j];
        h[k] = v / F[k * nn + k];
      }
      float dmax = 0.f, xmax = 0.f;
      for (int k = 0; k < mm; ++k) {
        x[k] += h[k];
        dmax = fmaxf(dmax, fabsf(h[k]));
        xmax = fmaxf(xmax, fabsf(x[k]));
      }
      if (!(dmax > A.tol * xmax)) break;
    }
    for (int j = 0; j < mm; ++j) xo[j] = x[j];
  }
}

// Launch with fully formed arguments (opting the kernel in to its dynamic shared memory).
template <typename T, bool REF>
cudaError_t launch_block_kernel(const BlockSolveArgs<T>& A, cudaStream_t st) {
  const size_t smem = make_layout<T>(A.vb, A.rb, A.cb, A.bb, A.pb, REF).total;
  auto kern = block_solve_kernel<T, REF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)A.num_tiles, kThreads, smem, st>>>(A);
  return cudaGetLastError();
}

template <typename T, bool REF, bool SEL = false>
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
  A.refine_tol = 1e-6f;
  A.status = ctx->d_status;
  A.vb = P.budget.values;
  A.rb = P.budget.rows;
  A.cb = P.budget.cols;
  A.bb = P.budget.blocks;
  A.pb = P.budget.padded;
  A.wait_limit = ctx->wait_limit;
  A.rlist = nullptr;
  A.rcount = nullptr;
  A.rcap = 0;
  if (SEL) {
    qrkit_status rc;
    if ((rc = ensure(ctx, ctx->ws.rlist, (size_t)4 * P.K * sizeof(int), "refinement lists")) != QRKIT_OK) return rc;
    if ((rc = ensure(ctx, ctx->ws.rcount, 4 * sizeof(int), "refinement counts")) != QRKIT_OK) return rc;
    QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->ws.rcount.ptr, 0, 4 * sizeof(int), ctx->stream));
    A.rlist = (int*)ctx->ws.rlist.ptr;
    A.rcount = (int*)ctx->ws.rcount.ptr;
    A.rcap = P.K;
  }
  const size_t smem = make_layout<T>(A.vb, A.rb, A.cb, A.bb, A.pb, REF, SEL).total;
  auto kern = block_solve_kernel<T, REF, SEL>;
  const int variant = (sizeof(T) == sizeof(double) ? 2 : 0) + (REF ? 1 : 0) + (SEL ? 4 : 0);
  if (ctx->smem_attr[variant] < smem) {
    QRKIT_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
    ctx->smem_attr[variant] = smem;
  }
  kern<<<(unsigned)P.num_tiles, kThreads, smem, ctx->stream>>>(A);
  ctx->launches += 1;
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  if constexpr (SEL && sizeof(T) == sizeof(float)) {
    RefineArgs R;
    R.n = A.n;
    R.m = A.m;
    R.val_off = (const int64_t*)P.d_val_off.ptr;
    R.row_off = (const int64_t*)P.d_row_off.ptr;
    R.col_off = (const int64_t*)P.d_col_off.ptr;
    R.J = (const float*)J;
    R.b = (const float*)b;
    R.F = (const float*)A.F;
    R.x = (float*)p;
    R.rlist = A.rlist;
    R.rcount = A.rcount;
    R.rcap = A.rcap;
    R.steps = refine_steps;
    R.tol = A.refine_tol;
    const int64_t want = (P.K + 127) / 128;
    const unsigned grid = (unsigned)(want < (int64_t)ctx->num_sms * 8 ? want : (int64_t)ctx->num_sms * 8);
    block_refine_kernel<<<grid > 0 ? grid : 1, 128, 0, ctx->stream>>>(R);
    ctx->launches += 1;
    QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  }
  return QRKIT_OK;
}

}  // namespace

TileBudget block_solve_budget(size_t elem) {
  TileBudget b;
  b.blocks = kThreads;
  if (elem == sizeof(float)) {
    b.values = 3072; b.rows = 1024; b.cols = 512; b.padded = 4096;
  } else {
    b.values = 1536; b.rows = 512; b.cols = 256; b.padded = 2048;
  }
  return b;
}

int block_solve_max_rows() { return kMaxRows; }
int block_solve_max_cols() { return kMaxCols; }

qrkit_status launch_block_solve(qrkit_ctx* ctx, const void* J, const void* b, const void* D,
                                void* p, void* qtb, int refine_steps) {
  (void)D;
  if (ctx->plan.mapping == 0 && ctx->plan.num_tasks > 0) return launch_block_tasks(ctx, J, b, p, qtb, refine_steps);
  if (ctx->precision == QRKIT_FP64) return launch_typed<double, false>(ctx, J, b, p, qtb, 0);
  const int steps = ctx->precision == QRKIT_FP32 ? 0 : refine_steps;
  if (steps > 0) return launch_typed<float, false, true>(ctx, J, b, p, qtb, steps);
  return launch_typed<float, false>(ctx, J, b, p, qtb, 0);
}

}  // namespace qrkit

// ---------------------------------------------------------------------------------------
// Allocation-free variant of the batched block solve.
//
// Some callers cannot call cudaMalloc at all: code that runs under a framework owning every
// byte of device memory through its own pool, or a process whose memory budget is fixed
// once at start-up.  For them qrkit_block_solve_noalloc solves the same problem as
// qrkit_factor_solve, without a context and without allocating, by the tile kernel
// (block_solve_kernel over tiles of consecutive blocks, refinement inside the kernel; the
// context path's default is the warp-task kernels): every intermediate it needs (block
// shapes, tile schedule, factor values, tau, status word) lives in the file-scope array
// below.  The array is part of the library image, so every process that loads the
// library holds it on each device it uses until the process exits.
namespace qrkit {
namespace {

constexpr size_t kNoallocScratchBytes = (size_t)QRKIT_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device with that device current.
// A host-side reference to g_noalloc_scratch is only a host stand-in, never a device address.
unsigned char* g_noalloc_ptr[64] = {nullptr};
std::mutex g_noalloc_mutex;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Makes `device` current for the lifetime of the guard and gives the caller's thread its
// previous current device back on every return path.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = prev == device || cudaSetDevice(device) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (ok && prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

}  // namespace qrkit

extern "C" qrkit_status qrkit_block_solve_noalloc(int device, void* stream, int precision,
                                                  int64_t num_blocks, const uint8_t* block_rows,
                                                  const uint8_t* block_cols, const void* J,
                                                  const void* b, void* p, int refine_steps) {
  using namespace qrkit;
  if (device < 0 || device >= 64) return QRKIT_EINVAL;
  if (precision < QRKIT_FP64 || precision > QRKIT_FP32) return QRKIT_EINVAL;
  if (num_blocks < 1 || !block_rows || !block_cols || !J || !b || !p) return QRKIT_EINVAL;
  if (refine_steps < 0 || refine_steps > 8) return QRKIT_EINVAL;
  // host-side plan: the same tile schedule as qrkit_plan builds
  Plan P;
  P.K = num_blocks;
  P.n.assign(block_rows, block_rows + num_blocks);
  P.m.assign(block_cols, block_cols + num_blocks);
  for (int64_t i = 0; i < P.K; ++i) {
    const int n = P.n[i], m = P.m[i];
    if (n < 1 || m < 1 || n < m) return QRKIT_EINVAL;
    if (n > kMaxRows || m > kMaxCols) return QRKIT_EUNSUPPORTED;
    P.rows += n;
    P.cols += m;
    P.values += (int64_t)n * m;
    P.max_m = P.max_m > m ? P.max_m : m;
  }
  const size_t elem = precision == QRKIT_FP64 ? sizeof(double) : sizeof(float);
  P.budget = block_solve_budget(elem);
  cut_tiles_for(P);
  // scratch layout; reject problems that do not fit
  const size_t tb = (size_t)(P.num_tiles + 1) * sizeof(int64_t);
  size_t off = 0;
  const size_t o_status = off; off = align256(off + sizeof(int));
  const size_t o_n = off; off = align256(off + (size_t)P.K);
  const size_t o_m = off; off = align256(off + (size_t)P.K);
  const size_t o_tb = off; off = align256(off + tb);
  const size_t o_tv = off; off = align256(off + tb);
  const size_t o_tr = off; off = align256(off + tb);
  const size_t o_tc = off; off = align256(off + tb);
  const size_t o_F = off; off = align256(off + (size_t)P.values * elem);
  const size_t o_tau = off; off = align256(off + (size_t)P.cols * elem);
  if (off > kNoallocScratchBytes) return QRKIT_EUNSUPPORTED;
  DeviceGuard guard(device);
  if (!guard.ok) return QRKIT_ECUDA;
  cudaError_t e = cudaSuccess;
  cudaStream_t st = (cudaStream_t)stream;
  if (st) {   // a stream of another device would run the kernel against the wrong array
    int sdev = -1;
    if ((e = cudaStreamGetDevice(st, &sdev)) != cudaSuccess) return QRKIT_ECUDA;
    if (sdev != device) return QRKIT_EINVAL;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return QRKIT_ECUDA;
      g_noalloc_ptr[device] = static_cast<unsigned char*>(ptr);
    }
    base = g_noalloc_ptr[device];
  }
  // the array keeps the previous call's contents: the status word must start at zero;
  // every other region used here is written in full before it is read
  if ((e = cudaMemsetAsync(base + o_status, 0, sizeof(int), st)) != cudaSuccess) return QRKIT_ECUDA;
  struct Up { size_t off; const void* src; size_t bytes; } ups[] = {
      {o_n, P.n.data(), (size_t)P.K}, {o_m, P.m.data(), (size_t)P.K},
      {o_tb, P.tile_block.data(), tb}, {o_tv, P.tile_val.data(), tb},
      {o_tr, P.tile_row.data(), tb}, {o_tc, P.tile_col.data(), tb}};
  for (const Up& u : ups)
    if ((e = cudaMemcpyAsync(base + u.off, u.src, u.bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return QRKIT_ECUDA;
  int* status = reinterpret_cast<int*>(base + o_status);
  auto fill = [&](auto* tag) {
    using T = std::remove_pointer_t<decltype(tag)>;
    BlockSolveArgs<T> A{};
    A.rlist = nullptr;
    A.rcount = nullptr;
    A.rcap = 0;
    A.n = base + o_n;
    A.m = base + o_m;
    A.tile_block = reinterpret_cast<const int64_t*>(base + o_tb);
    A.tile_val = reinterpret_cast<const int64_t*>(base + o_tv);
    A.tile_row = reinterpret_cast<const int64_t*>(base + o_tr);
    A.tile_col = reinterpret_cast<const int64_t*>(base + o_tc);
    A.num_tiles = P.num_tiles;
    A.J = static_cast<const T*>(J);
    A.b = static_cast<const T*>(b);
    A.F = reinterpret_cast<T*>(base + o_F);
    A.tau = reinterpret_cast<T*>(base + o_tau);
    A.qtb = nullptr;
    A.x = static_cast<T*>(p);
    A.refine_tol = 1e-6f;
    A.status = status;
    A.vb = P.budget.values;
    A.rb = P.budget.rows;
    A.cb = P.budget.cols;
    A.bb = P.budget.blocks;
    A.pb = P.budget.padded;
    A.wait_limit = 1LL << 26;
    return A;
  };
  if (precision == QRKIT_FP64) {
    BlockSolveArgs<double> A = fill((double*)nullptr);
    A.refine_steps = 0;
    e = launch_block_kernel<double, false>(A, st);
  } else if (precision == QRKIT_FP32 || refine_steps == 0) {
    BlockSolveArgs<float> A = fill((float*)nullptr);
    A.refine_steps = 0;
    e = launch_block_kernel<float, false>(A, st);
  } else {
    BlockSolveArgs<float> A = fill((float*)nullptr);
    A.refine_steps = refine_steps;
    e = launch_block_kernel<float, true>(A, st);
  }
  if (e != cudaSuccess) return QRKIT_ECUDA;
  // the call returns only after the solve: read the device status word back (no allocation)
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return QRKIT_ECUDA;
  int h = 0;
  if ((e = cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return QRKIT_ECUDA;
  return (qrkit_status)h;
}
