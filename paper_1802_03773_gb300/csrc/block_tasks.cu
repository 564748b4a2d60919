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

// One data buffer of a warp: the block slots of the largest task among the keys of class cls
// present in the plan.
int warp_slot_bytes(const Plan& P, int es, int cls) {
  int best = 0;
  for (int k = 0; k < kTaskKeys; ++k) {
    if (P.key_off[k + 1] == P.key_off[k] || !key_in_class(k, cls)) continue;
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

// One launch of the factor kernel of class CLS over tasks [t0, t1) of the plan.
template <typename T, bool SEL, int CLS>
qrkit_status launch_class(qrkit_ctx* ctx, TaskArgs<T> A, int64_t t0, int64_t t1, int slot) {
  const Plan& P = ctx->plan;
  if (t1 <= t0) return QRKIT_OK;
  const int es = (int)sizeof(T);
  const int wpc = P.task_warps;
  const int threads = 32 * wpc;
  A.hdr += t0;
  A.num_tasks = t1 - t0;
  A.data_bytes = warp_slot_bytes(P, es, CLS);
  A.warp_bytes = (warp_desc_bytes((int)sizeof(TaskEntry)) + 2 * A.data_bytes + 127) / 128 * 128;
  const size_t smem = (size_t)wpc * A.warp_bytes;
  int per_sm = 0;
  qrkit_status st;
  if ((st = resident(ctx, kernel_setup<T, SEL, CLS>, threads, smem, slot, per_sm)) != QRKIT_OK) return st;
  const int64_t want = (A.num_tasks + wpc - 1) / wpc;
  const int64_t full = (int64_t)ctx->num_sms * per_sm;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min(want, full));
  QRKIT_CUDA_TRY(ctx, (kernel_launch<T, SEL, CLS>(A, grid, threads, smem, ctx->stream)));
  ctx->launches += 1;
  return QRKIT_OK;
}

template <typename T, bool SEL>
qrkit_status launch_tasks_typed(qrkit_ctx* ctx, const void* J, const void* b, void* p, void* qtb,
                                int refine_steps) {
  Plan& P = ctx->plan;
  static_assert(sizeof(TaskHdr) % 16 == 0 && sizeof(RefEntry) % 16 == 0, "16-byte copies");
  TaskArgs<T> A;
  A.hdr = (const TaskHdr*)P.d_task_hdr.ptr;
  A.ent = (const TaskEntry*)P.d_task_ent.ptr;
  A.num_tasks = P.num_tasks;
  A.J = (const T*)J;
  A.b = (const T*)b;
  A.J_end = A.J + P.values;
  A.b_end = A.b + P.rows;
  A.tF = (T*)ctx->ws.tfactor.ptr;
  A.tTau = (T*)ctx->ws.ttau.ptr;
  A.qtb = (T*)qtb;
  A.x = (T*)p;
  A.q_vec = qtb && ((reinterpret_cast<uintptr_t>(qtb) ^ reinterpret_cast<uintptr_t>(b)) & 15) == 0;
  A.status = ctx->d_status;
  A.select = ctx->refine_select;
  A.rlist = nullptr;
  A.rcount = nullptr;
  A.key_off = (const int64_t*)P.d_key_off.ptr;
  A.rec = nullptr;
  A.rec_off = (const int64_t*)P.d_rec_off.ptr;
  qrkit_status st;
  if (SEL) {
    if ((st = ensure(ctx, ctx->ws.tlist, (size_t)std::max<int64_t>(P.K, 1) * sizeof(RefEntry), "refinement lists")) !=
        QRKIT_OK)
      return st;
    if ((st = ensure(ctx, ctx->ws.rrec, (size_t)std::max<int64_t>(P.rec_off[kTaskKeys], 1) * sizeof(float),
                     "refinement records")) != QRKIT_OK)
      return st;
    A.rec = (float*)ctx->ws.rrec.ptr;
    // counts per shape key, then the most steps a block took
    if ((st = ensure(ctx, ctx->ws.tcount, (kTaskKeys + 1) * sizeof(int), "refinement counts")) != QRKIT_OK) return st;
    QRKIT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->ws.tcount.ptr, 0, (kTaskKeys + 1) * sizeof(int), ctx->stream));
    A.rlist = (RefEntry*)ctx->ws.tlist.ptr;
    A.rcount = (int*)ctx->ws.tcount.ptr;
  }
  ctx->refine_stats = SEL && sizeof(T) == sizeof(float);
  if constexpr (sizeof(T) == sizeof(double) || !SEL) {
    // one kernel over every task: double, and float without the refinement selection (whose
    // register needs fit 2 CTAs per SM for every key)
    if ((st = launch_class<T, false, 0>(ctx, A, 0, P.num_tasks, sizeof(T) == 8 ? 10 : 8)) != QRKIT_OK) return st;
  } else {
    // float with the selection: a refined plan puts the tasks of blocks with at most 4 columns
    // first; each class runs in the kernel compiled for it
    if ((st = launch_class<T, SEL, 1>(ctx, A, 0, P.narrow_tasks, 9)) != QRKIT_OK) return st;
    if ((st = launch_class<T, SEL, 2>(ctx, A, P.narrow_tasks, P.num_tasks, 14)) != QRKIT_OK) return st;
  }
  if constexpr (SEL && sizeof(T) == sizeof(float)) {
    RefineTaskArgs R;
    R.tF = (const float*)A.tF;
    R.rec = A.rec;
    R.rec_off = A.rec_off;
    R.x = (float*)p;
    R.rlist = A.rlist;
    R.rcount = A.rcount;
    R.key_off = A.key_off;
    R.steps = refine_steps;
    R.tol = 1e-6f;
    R.steps_max = A.rcount + kTaskKeys;
    R.status = A.status;
    const int threads2 = 32 * kRefineWarps;
    const bool res64 = ctx->refine_residual != 0;
    int per_sm2 = 0;
    if ((st = resident(ctx, res64 ? refine_setup<1> : refine_setup<0>, threads2, 0, res64 ? 12 : 11, per_sm2)) !=
        QRKIT_OK)
      return st;
    const int64_t want2 = (P.max_refine_tasks + kRefineWarps - 1) / kRefineWarps;
    const int64_t full2 = (int64_t)ctx->num_sms * per_sm2;
    const unsigned grid2 = (unsigned)std::max<int64_t>(1, std::min(want2, full2));
    QRKIT_CUDA_TRY(ctx, res64 ? refine_launch<1>(R, grid2, threads2, 0, ctx->stream)
                              : refine_launch<0>(R, grid2, threads2, 0, ctx->stream));
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
  release(P.d_rec_off);
  P.factor_planes = 0;
  P.rec_off.clear();
  P.num_tasks = 0;
  P.narrow_tasks = 0;
  P.max_refine_tasks = 0;
  P.key_off.clear();
}

namespace tasks {

// The task lists of K blocks with the given shapes and offsets (K + 1 prefix sums each), no
// CUDA call: per supertile of consecutive blocks a stable counting sort by shape key, each
// key's run cut into tasks of task_blocks(G) entries (unused entries have n = 0); with
// key_major the tasks are stably reordered by key.  key_count[k] = blocks of key k.  Returns
// QRKIT_OK, or an error status with its message in err.
qrkit_status make_task_lists(int64_t K, const uint8_t* n, const uint8_t* m, const int64_t* val_off,
                             const int64_t* row_off, const int64_t* col_off, int64_t supertile,
                             bool key_major, std::vector<TaskHdr>& hdr, std::vector<TaskEntry>& ent,
                             std::vector<int64_t>& key_count, int64_t& planes, std::string& err) {
  if (supertile < 32 || supertile > 65536) {
    err = "supertile must be in [32, 65536]";
    return QRKIT_EINVAL;
  }
  if (K > (int64_t)INT32_MAX) {
    err = "more than 2^31 - 1 blocks";
    return QRKIT_EUNSUPPORTED;
  }
  hdr.clear();
  ent.clear();
  hdr.reserve((size_t)(K / 8 + kTaskKeys));
  ent.reserve((size_t)(K + K / 16 + 32 * kTaskKeys));
  key_count.assign(kTaskKeys, 0);
  std::vector<int64_t> cnt(kTaskKeys), pos(kTaskKeys);
  std::vector<int32_t> order;
  planes = 0;
  auto key_of = [&](int64_t i) { return ((n[i] - 1) >> 2) * 8 + (m[i] - 1); };
  for (int64_t s0 = 0; s0 < K; s0 += supertile) {
    const int64_t s1 = std::min(K, s0 + supertile);
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
        h.v0 = val_off[s0];
        h.r0 = row_off[s0];
        h.c0 = col_off[s0];
        h.b0 = s0;
        h.first = (int64_t)ent.size();
        h.key = k;
        if (planes > (int64_t)INT32_MAX - kMaxCols) {
          err = "the factor needs more than 2^31 planes";
          return QRKIT_EUNSUPPORTED;
        }
        h.plane = (int32_t)planes;
        planes += (k & 7) + 1;
        hdr.push_back(h);
        for (int l = 0; l < per; ++l) {
          TaskEntry e{};
          if (c0 + l < cnt[k]) {
            const int64_t i = s0 + order[(size_t)(at + c0 + l)];
            e.v = (uint32_t)(val_off[i] - h.v0);
            e.r = (uint32_t)(row_off[i] - h.r0);
            e.c = (uint32_t)(col_off[i] - h.c0);
            e.blk = (uint16_t)(i - s0);
            e.n = n[i];
            e.m = m[i];
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
  return QRKIT_OK;
}

}  // namespace tasks

qrkit_status build_block_tasks(qrkit_ctx* ctx, int64_t supertile, int warps, bool key_major) {
  Plan& P = ctx->plan;
  if (warps < 1 || warps > kTaskMaxWarps) return fail(ctx, QRKIT_EINVAL, "warps per CTA must be in [1, 8]");
  std::vector<TaskHdr> hdr;
  std::vector<TaskEntry> ent;
  std::vector<int64_t> key_count;
  std::string err;
  int64_t planes = 0;
  qrkit_status st = make_task_lists(P.K, P.n.data(), P.m.data(), P.val_off.data(), P.row_off.data(),
                                    P.col_off.data(), supertile, key_major, hdr, ent, key_count, planes, err);
  if (st != QRKIT_OK) return fail(ctx, st, err);
  // FP32-refined plans: the tasks of blocks with at most 4 columns first (kept in order), then
  // the others; the two runs go to the factor kernels compiled for each class (the other
  // precisions keep the supertile order, in which neighbouring blocks' shared sectors are read
  // together)
  P.narrow_tasks = 0;
  if (ctx->precision == QRKIT_FP32_REFINED) {
    auto mid = std::stable_partition(hdr.begin(), hdr.end(), [](const TaskHdr& h) { return key_in_class(h.key, 1); });
    P.narrow_tasks = (int64_t)(mid - hdr.begin());
  }
  P.key_off.assign(kTaskKeys + 1, 0);
  P.rec_off.assign(kTaskKeys + 1, 0);
  P.max_refine_tasks = 0;
  for (int k = 0; k < kTaskKeys; ++k) {
    P.key_off[k + 1] = P.key_off[k] + key_count[k];
    P.rec_off[k + 1] = P.rec_off[k] + key_count[k] * record_values(group_lanes(k), (k & 7) + 1);
    const int per = task_blocks(group_lanes(k));
    P.max_refine_tasks += (key_count[k] + per - 1) / per;
  }
  P.factor_planes = planes;
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
  if ((st = up(P.d_rec_off, P.rec_off.data(), P.rec_off.size() * sizeof(int64_t), "record offsets")) != QRKIT_OK)
    return st;
  const size_t es = elem_size(ctx);
  if ((st = ensure(ctx, ctx->ws.tfactor, (size_t)std::max<int64_t>(planes, 1) * kPlaneValues * es, "factor planes")) !=
      QRKIT_OK)
    return st;
  if ((st = ensure(ctx, ctx->ws.ttau, (size_t)std::max<int64_t>(planes, 1) * kTauPlane * es, "tau planes")) !=
      QRKIT_OK)
    return st;
  P.num_tasks = (int64_t)hdr.size();
  P.supertile = supertile;
  P.task_warps = warps;
  P.key_major = key_major;
  return QRKIT_OK;
}

qrkit_status unpack_block_tasks_factor(qrkit_ctx* ctx, void* factor_out, void* tau_out) {
  const Plan& P = ctx->plan;
  if (P.num_tasks < 1) return fail(ctx, QRKIT_ESTATE, "the plan has no warp tasks");
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((P.num_tasks + 7) / 8, (int64_t)ctx->num_sms * 8);
  const TaskHdr* hdr = (const TaskHdr*)P.d_task_hdr.ptr;
  const TaskEntry* ent = (const TaskEntry*)P.d_task_ent.ptr;
  if (ctx->precision == QRKIT_FP64)
    unpack_factor_kernel<double><<<(unsigned)blocks, threads, 0, ctx->stream>>>(
        hdr, ent, P.num_tasks, (const double*)ctx->ws.tfactor.ptr, (const double*)ctx->ws.ttau.ptr,
        (double*)factor_out, (double*)tau_out);
  else
    unpack_factor_kernel<float><<<(unsigned)blocks, threads, 0, ctx->stream>>>(
        hdr, ent, P.num_tasks, (const float*)ctx->ws.tfactor.ptr, (const float*)ctx->ws.ttau.ptr,
        (float*)factor_out, (float*)tau_out);
  QRKIT_CUDA_TRY(ctx, cudaGetLastError());
  ctx->launches += 1;
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

extern "C" qrkit_status qrkit_task_layout(int64_t num_blocks, const uint8_t* block_rows,
                                          const uint8_t* block_cols, int64_t supertile, int key_major,
                                          int64_t* num_tasks, int32_t* task_key, int64_t* task_slots,
                                          int64_t capacity) {
  using namespace qrkit;
  using namespace qrkit::tasks;
  if (num_blocks < 1 || !block_rows || !block_cols || !num_tasks || capacity < 0) return QRKIT_EINVAL;
  std::vector<int64_t> val_off((size_t)num_blocks + 1, 0), row_off((size_t)num_blocks + 1, 0),
      col_off((size_t)num_blocks + 1, 0);
  for (int64_t i = 0; i < num_blocks; ++i) {
    const int n = block_rows[i], m = block_cols[i];
    if (n < 1 || m < 1) return QRKIT_EINVAL;
    if (n > 16 || m > kMaxCols) return QRKIT_EUNSUPPORTED;
    val_off[i + 1] = val_off[i] + (int64_t)n * m;
    row_off[i + 1] = row_off[i] + n;
    col_off[i + 1] = col_off[i] + m;
  }
  std::vector<TaskHdr> hdr;
  std::vector<TaskEntry> ent;
  std::vector<int64_t> key_count;
  std::string err;
  int64_t planes = 0;
  const qrkit_status st = make_task_lists(num_blocks, block_rows, block_cols, val_off.data(), row_off.data(),
                                          col_off.data(), supertile, key_major != 0, hdr, ent, key_count, planes, err);
  if (st != QRKIT_OK) return st;
  *num_tasks = (int64_t)hdr.size();
  if (!task_key && !task_slots) return QRKIT_OK;
  if (capacity < (int64_t)hdr.size()) return QRKIT_EINVAL;
  for (size_t t = 0; t < hdr.size(); ++t) {
    const TaskHdr& h = hdr[t];
    if (task_key) task_key[t] = h.key;
    if (!task_slots) continue;
    const int per = task_blocks(group_lanes(h.key));
    for (int l = 0; l < 32; ++l) {
      int64_t* o = task_slots + ((int64_t)t * 32 + l) * 4;
      const TaskEntry* e = l < per ? &ent[(size_t)(h.first + l)] : nullptr;
      if (e && e->n > 0) {
        o[0] = h.b0 + e->blk;
        o[1] = h.v0 + e->v;
        o[2] = h.r0 + e->r;
        o[3] = h.c0 + e->c;
      } else {
        o[0] = o[1] = o[2] = o[3] = -1;
      }
    }
  }
  return QRKIT_OK;
}
