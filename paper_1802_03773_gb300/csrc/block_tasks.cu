// Batched block-diagonal QR solve by shape-uniform warp tasks, host side: the task lists of
// a plan (supertiles of consecutive blocks counting-sorted by shape key and cut into warp
// tasks), and the launches of the factor kernel and of the refinement kernel.  The kernels
// are in block_tasks.cuh, instantiated by block_tasks_{f32,f32sel,f64,refine}.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "block_tasks.cuh"

namespace qrkit {
namespace tasks {
namespace {

// One data buffer of a warp: the block slots of the largest task among the keys present in
// the plan.
int warp_slot_bytes(const Plan& P, int es) {
  int best = 0;
  for (int k = 0; k < kTaskKeys; ++k) {
    if (P.key_off[k + 1] == P.key_off[k]) continue;
    const int G = group_lanes(k), M = (k & 7) + 1;
    best = std::max(best, task_blocks(G) * (slot_j_bytes(G, M, es) + slot_b_bytes(G, es)));
  }
  return (best + 127) / 128 * 128;
}

// Resident CTAs per SM of a kernel at this shared-memory size; the kernel's shared-memory
// limit is raised and its occupancy queried once per (kernel, size) and cached.
template <typename F>
qrkit_status resident(qrkit_ctx* ctx, F setup, int threads, size_t smem, int slot, int& per_sm) {
  if (ctx->smem_attr[slot] != smem || ctx->occ_threads[slot] != threads) {
    int r = 0;
    QRKIT_CUDA_TRY(ctx, setup(smem, threads, &r));
    if (r < 1) return fail(ctx, QRKIT_EUNSUPPORTED, "block task kernel does not fit on an SM");
    ctx->smem_attr[slot] = smem;
    ctx->occ_threads[slot] = threads;
    ctx->occ_per_sm[slot] = r;
  }
  per_sm = ctx->occ_per_sm[slot];
  return QRKIT_OK;
}

template <typename T, bool SEL>
qrkit_status launch_tasks_typed(qrkit_ctx* ctx, const void* J, const void* b, void* p, void* qtb,
                                int refine_steps) {
  Plan& P = ctx->plan;
  const int es = (int)sizeof(T);
  const int wpc = P.task_warps;
  static_assert(sizeof(TaskHdr) % 16 == 0 && sizeof(RefEntry) % 16 == 0, "16-byte copies");
  const int threads = 32 * wpc;
  TaskArgs<T> A;
  A.hdr = (const TaskHdr*)P.d_task_hdr.ptr;
  A.ent = (const TaskEntry*)P.d_task_ent.ptr;
  A.num_tasks = P.num_tasks;
  A.J = (const T*)J;
  A.b = (const T*)b;
  A.J_end = A.J + P.values;
  A.b_end = A.b + P.rows;
  A.F = (T*)ctx->ws.factor.ptr;
  A.tau = (T*)ctx->ws.tau.ptr;
  A.qtb = (T*)qtb;
  A.x = (T*)p;
  A.f_vec = ((reinterpret_cast<uintptr_t>(A.F) ^ reinterpret_cast<uintptr_t>(J)) & 15) == 0;
  A.q_vec = qtb && ((reinterpret_cast<uintptr_t>(qtb) ^ reinterpret_cast<uintptr_t>(b)) & 15) == 0;
  A.data_bytes = warp_slot_bytes(P, es);
  A.warp_bytes = (warp_desc_bytes((int)sizeof(TaskEntry)) + 2 * A.data_bytes + 127) / 128 * 128;
  A.status = ctx->d_status;
  A.rlist = nullptr;
  A.rcount = nullptr;
  A.key_off = (const int64_t*)P.d_key_off.ptr;
  qrkit_status st;
  if (SEL) {
    if ((st = ensure(ctx, ctx->ws.tlist, (size_t)std::max<int64_t>(P.K, 1) * sizeof(RefEntry), "refinement lists")) !=
        QRKIT_OK)
      return st;
    if ((st = ensure(ctx, ctx->ws.tcount, kTaskKeys * sizeof(int), "refinement counts")) != QRKIT_OK) return st;
    QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->ws.tcount.ptr, 0, kTaskKeys * sizeof(int), ctx->stream));
    A.rlist = (RefEntry*)ctx->ws.tlist.ptr;
    A.rcount = (int*)ctx->ws.tcount.ptr;
  }
  const size_t smem = (size_t)wpc * A.warp_bytes;
  int per_sm = 0;
  if ((st = resident(ctx, kernel_setup<T, SEL>, threads, smem, sizeof(T) == 8 ? 10 : (SEL ? 9 : 8), per_sm)) != QRKIT_OK)
    return st;
  const int64_t want = (P.num_tasks + wpc - 1) / wpc;
  const int64_t full = (int64_t)ctx->num_sms * per_sm;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min(want, full));
  QRKIT_CUDA_TRY(ctx, (kernel_launch<T, SEL>(A, grid, threads, smem, ctx->stream)));
  ctx->launches += 1;
  if constexpr (SEL && sizeof(T) == sizeof(float)) {
    RefineTaskArgs R;
    R.J = (const float*)J;
    R.b = (const float*)b;
    R.J_end = R.J + P.values;
    R.b_end = R.b + P.rows;
    R.F = (const float*)A.F;
    R.x = (float*)p;
    R.rlist = A.rlist;
    R.rcount = A.rcount;
    R.key_off = A.key_off;
    R.steps = refine_steps;
    R.tol = 1e-6f;
    R.data_bytes = A.data_bytes;
    R.warp_bytes = (warp_desc_bytes((int)sizeof(RefEntry)) + 2 * R.data_bytes + 127) / 128 * 128;
    const size_t smem2 = (size_t)wpc * R.warp_bytes;
    R.status = A.status;
    int per_sm2 = 0;
    if ((st = resident(ctx, refine_setup, threads, smem2, 11, per_sm2)) != QRKIT_OK) return st;
    const int64_t want2 = (P.max_refine_tasks + wpc - 1) / wpc;
    const int64_t full2 = (int64_t)ctx->num_sms * per_sm2;
    const unsigned grid2 = (unsigned)std::max<int64_t>(1, std::min(want2, full2));
    QRKIT_CUDA_TRY(ctx, refine_launch(R, grid2, threads, smem2, ctx->stream));
    ctx->launches += 1;
  }
  return QRKIT_OK;
}

}  // namespace
}  // namespace tasks

using namespace tasks;

void release_block_tasks(Plan& P) {
  release(P.d_task_hdr);
  release(P.d_task_ent);
  release(P.d_key_off);
  P.num_tasks = 0;
  P.max_refine_tasks = 0;
  P.key_off.clear();
}

qrkit_status build_block_tasks(qrkit_ctx* ctx, int64_t supertile, int warps, bool key_major) {
  Plan& P = ctx->plan;
  if (supertile < 32 || supertile > 65536) return fail(ctx, QRKIT_EINVAL, "supertile must be in [32, 65536]");
  if (warps < 1 || warps > kTaskMaxWarps) return fail(ctx, QRKIT_EINVAL, "warps per CTA must be in [1, 8]");
  if (P.K > (int64_t)INT32_MAX) return fail(ctx, QRKIT_EUNSUPPORTED, "more than 2^31 - 1 blocks");
  std::vector<TaskHdr> hdr;
  std::vector<TaskEntry> ent;
  hdr.reserve((size_t)(P.K / 8 + kTaskKeys));
  ent.reserve((size_t)(P.K + P.K / 16 + 32 * kTaskKeys));
  std::vector<int64_t> key_count(kTaskKeys, 0);
  std::vector<int64_t> cnt(kTaskKeys), pos(kTaskKeys);
  std::vector<int32_t> order;
  auto key_of = [&](int64_t i) { return ((P.n[i] - 1) >> 2) * 8 + (P.m[i] - 1); };
  for (int64_t s0 = 0; s0 < P.K; s0 += supertile) {
    const int64_t s1 = std::min(P.K, s0 + supertile);
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t i = s0; i < s1; ++i) cnt[key_of(i)] += 1;
    int64_t acc = 0;
    for (int k = 0; k < kTaskKeys; ++k) {
      pos[k] = acc;
      acc += cnt[k];
    }
    order.resize((size_t)(s1 - s0));
    for (int64_t i = s0; i < s1; ++i) order[pos[key_of(i)]++] = (int32_t)(i - s0);
    int64_t at = 0;
    for (int k = 0; k < kTaskKeys; ++k) {
      const int per = task_blocks(group_lanes(k));
      for (int64_t c0 = 0; c0 < cnt[k]; c0 += per) {
        TaskHdr h{};
        h.v0 = P.val_off[s0];
        h.r0 = P.row_off[s0];
        h.c0 = P.col_off[s0];
        h.b0 = s0;
        h.first = (int64_t)ent.size();
        h.key = k;
        hdr.push_back(h);
        for (int l = 0; l < per; ++l) {
          TaskEntry e{};
          if (c0 + l < cnt[k]) {
            const int64_t i = s0 + order[(size_t)(at + c0 + l)];
            e.v = (uint32_t)(P.val_off[i] - h.v0);
            e.r = (uint32_t)(P.row_off[i] - h.r0);
            e.c = (uint32_t)(P.col_off[i] - h.c0);
            e.blk = (uint16_t)(i - s0);
            e.n = P.n[i];
            e.m = P.m[i];
          }
          ent.push_back(e);
        }
      }
      at += cnt[k];
      key_count[k] += cnt[k];
    }
  }
  if (key_major)   // all tasks of a shape key together (supertiles in order within a key)
    std::stable_sort(hdr.begin(), hdr.end(), [](const TaskHdr& x, const TaskHdr& y) { return x.key < y.key; });
  P.key_off.assign(kTaskKeys + 1, 0);
  P.max_refine_tasks = 0;
  for (int k = 0; k < kTaskKeys; ++k) {
    P.key_off[k + 1] = P.key_off[k] + key_count[k];
    const int per = task_blocks(group_lanes(k));
    P.max_refine_tasks += (key_count[k] + per - 1) / per;
  }
  qrkit_status st;
  auto up = [&](DevBuf& d, const void* src, size_t bytes, const char* what) -> qrkit_status {
    qrkit_status r = ensure(ctx, d, bytes, what);
    if (r != QRKIT_OK) return r;
    QRKIT_CUDA_TRY(ctx, cudaMemcpy(d.ptr, src, bytes, cudaMemcpyHostToDevice));
    return QRKIT_OK;
  };
  if ((st = up(P.d_task_hdr, hdr.data(), hdr.size() * sizeof(TaskHdr), "task headers")) != QRKIT_OK) return st;
  if ((st = up(P.d_task_ent, ent.data(), ent.size() * sizeof(TaskEntry), "task entries")) != QRKIT_OK) return st;
  if ((st = up(P.d_key_off, P.key_off.data(), P.key_off.size() * sizeof(int64_t), "task key offsets")) != QRKIT_OK)
    return st;
  P.num_tasks = (int64_t)hdr.size();
  P.supertile = supertile;
  P.task_warps = warps;
  P.key_major = key_major;
  return QRKIT_OK;
}

qrkit_status launch_block_tasks(qrkit_ctx* ctx, const void* J, const void* b, void* p, void* qtb,
                                int refine_steps) {
  if (ctx->plan.num_tasks < 1) return fail(ctx, QRKIT_ESTATE, "the plan has no warp tasks");
  if (ctx->precision == QRKIT_FP64) return launch_tasks_typed<double, false>(ctx, J, b, p, qtb, 0);
  const int steps = ctx->precision == QRKIT_FP32 ? 0 : refine_steps;
  if (steps > 0) return launch_tasks_typed<float, true>(ctx, J, b, p, qtb, steps);
  return launch_tasks_typed<float, false>(ctx, J, b, p, qtb, 0);
}

}  // namespace qrkit
