// Autotuning of launch configurations for the current plan, with a persistent text cache.
//
// Block plans (QRKIT_STRUCT_BLOCKS, no coupling): the block-to-warp mapping of the fused
// solve: shape-uniform warp tasks (supertile of consecutive blocks sorted by shape, warps per
// CTA) or tiles of consecutive blocks (blocks / values / rows / columns / padded working area
// per tile, which set the tile count, the work per barrier phase and the shared memory per
// CTA).  Banded plans: the
// compression strategy of the parallel banded QR (one thread per column block, or warps with
// a number of splits).  Every candidate is timed with CUDA events on the context's stream on
// the caller's inputs (one warm-up, three timed runs), the fastest is kept.  The cache holds
// one line per structure key: "<key>\t<choice>"; a key already present is applied without
// timing.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

namespace qrkit {
namespace {

std::string gpu_name(int device) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return "unknown";
  std::string s = p.name;
  std::replace(s.begin(), s.end(), ' ', '_');
  return s;
}

// FNV-1a over the block shapes: the key of a block structure.
uint64_t shape_hash(const Plan& P) {
  uint64_t h = 1469598103934665603ull;
  for (int64_t i = 0; i < P.K; ++i) {
    h = (h ^ P.n[i]) * 1099511628211ull;
    h = (h ^ P.m[i]) * 1099511628211ull;
  }
  return h;
}

std::string plan_key(const qrkit_ctx* ctx) {
  const Plan& P = ctx->plan;
  std::ostringstream k;
  k << "v2:" << gpu_name(ctx->device) << ":prec" << ctx->precision << ":";
  if (P.s.kind == QRKIT_STRUCT_BANDED) {
    const Band& B = ctx->band;
    k << "banded:inst" << B.num_inst << ":cols" << B.total_cols << ":rpc" << B.rows_per_col << ":w" << B.w;
  } else {
    k << "blocks:K" << P.K << ":shapes" << std::hex << shape_hash(P);
  }
  return k.str();
}

bool cache_lookup(const char* path, const std::string& key, std::string& value) {
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    const size_t tab = line.find('\t');
    if (tab != std::string::npos && line.compare(0, tab, key) == 0 && tab == key.size()) {
      value = line.substr(tab + 1);
      found = true;   // the last entry wins
    }
  }
  return found;
}

void cache_store(const char* path, const std::string& key, const std::string& value) {
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << '\t' << value << '\n';
}

std::vector<TileBudget> budget_candidates(size_t elem) {
  std::vector<TileBudget> c;
  const TileBudget d = block_solve_budget(elem);
  c.push_back(d);
  for (const double f : {0.5, 0.75, 1.25}) {
    TileBudget t;
    t.blocks = std::min(d.blocks, std::max(32, (int)(d.blocks * f) / 32 * 32));   // <= threads per CTA
    t.values = (int)(d.values * f);
    t.rows = (int)(d.rows * f);
    t.cols = (int)(d.cols * f);
    t.padded = (int)(d.padded * f) / 4 * 4;
    c.push_back(t);
  }
  return c;
}

std::string budget_str(const TileBudget& t) {
  std::ostringstream s;
  s << "budget " << t.blocks << " " << t.values << " " << t.rows << " " << t.cols << " " << t.padded;
  return s.str();
}

bool parse_budget(const std::string& v, TileBudget& t) {
  std::istringstream s(v);
  std::string tag;
  s >> tag >> t.blocks >> t.values >> t.rows >> t.cols >> t.padded;
  return tag == "budget" && !s.fail();
}

qrkit_status apply_budget(qrkit_ctx* ctx, const TileBudget& t) {
  Plan& P = ctx->plan;
  // a budget must still hold the largest block
  const int pad_max = 16 * 8;
  if (t.blocks < 1 || t.values < 16 * 8 || t.rows < 16 || t.cols < 8 || t.padded < pad_max)
    return fail(ctx, QRKIT_EINVAL, "tile budget too small");
  P.budget = t;
  P.mapping = 1;
  cut_tiles_for(P);
  const size_t tb = (size_t)(P.num_tiles + 1) * sizeof(int64_t);
  qrkit_status st;
  auto up = [&](DevBuf& d, const std::vector<int64_t>& v) -> qrkit_status {
    qrkit_status r = ensure(ctx, d, tb, "plan tiles");
    if (r != QRKIT_OK) return r;
    QRKIT_CUDA_TRY(ctx, cudaMemcpy(d.ptr, v.data(), tb, cudaMemcpyHostToDevice));
    return QRKIT_OK;
  };
  if ((st = up(P.d_tile_block, P.tile_block)) != QRKIT_OK) return st;
  if ((st = up(P.d_tile_val, P.tile_val)) != QRKIT_OK) return st;
  if ((st = up(P.d_tile_row, P.tile_row)) != QRKIT_OK) return st;
  if ((st = up(P.d_tile_col, P.tile_col)) != QRKIT_OK) return st;
  return QRKIT_OK;
}

// Block mapping choices: "tasks <supertile> <warps per CTA> [<key-major 0/1>]" or
// "budget <tile budget>".
struct BlockChoice {
  bool tasks = true;
  int64_t supertile = kDefaultSupertile;
  int warps = 8;
  int key_major = 0;
  TileBudget budget{};
};

std::string choice_str(const BlockChoice& c) {
  if (!c.tasks) return budget_str(c.budget);
  std::ostringstream s;
  s << "tasks " << c.supertile << " " << c.warps << " " << c.key_major;
  return s.str();
}

bool parse_choice(const std::string& v, BlockChoice& c) {
  if (v.compare(0, 7, "budget ") == 0) {
    c.tasks = false;
    return parse_budget(v, c.budget);
  }
  std::istringstream s(v);
  std::string tag;
  s >> tag >> c.supertile >> c.warps;
  c.tasks = true;
  if (tag != "tasks" || s.fail()) return false;
  int km = 0;
  if (s >> km) c.key_major = km != 0;   // optional, supertile-major by default
  return true;
}

qrkit_status apply_choice(qrkit_ctx* ctx, const BlockChoice& c) {
  if (!c.tasks) return apply_budget(ctx, c.budget);
  qrkit_status st = build_block_tasks(ctx, c.supertile, c.warps, c.key_major != 0);
  if (st == QRKIT_OK) ctx->plan.mapping = 0;
  return st;
}

std::vector<BlockChoice> block_candidates(size_t elem) {
  std::vector<BlockChoice> c;
  for (const int km : {0, 1})
    for (const int64_t s : {kDefaultSupertile, (int64_t)16384}) {
      BlockChoice t;
      t.supertile = s;
      t.key_major = km;
      c.push_back(t);
    }
  for (const int w : {4, 6}) {
    BlockChoice t;
    t.warps = w;
    c.push_back(t);
  }
  for (const TileBudget& b : budget_candidates(elem)) {
    BlockChoice t;
    t.tasks = false;
    t.budget = b;
    c.push_back(t);
  }
  return c;
}

template <typename F>
qrkit_status time_runs(qrkit_ctx* ctx, F run, float& ms) {
  qrkit_status st = run();
  if (st != QRKIT_OK) return st;
  cudaEvent_t e0, e1;
  QRKIT_CUDA_TRY(ctx, cudaEventCreate(&e0));
  QRKIT_CUDA_TRY(ctx, cudaEventCreate(&e1));
  QRKIT_CUDA_TRY(ctx, cudaEventRecord(e0, ctx->stream));
  for (int i = 0; i < 3 && st == QRKIT_OK; ++i) st = run();
  QRKIT_CUDA_TRY(ctx, cudaEventRecord(e1, ctx->stream));
  QRKIT_CUDA_TRY(ctx, cudaEventSynchronize(e1));
  QRKIT_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ms /= 3.f;
  return st;
}

}  // namespace
}  // namespace qrkit

using namespace qrkit;

extern "C" qrkit_status qrkit_autotune(qrkit_ctx* ctx, const void* J, const void* b, void* p, int refine_steps,
                                       const char* cache_path, char* chosen, int64_t chosen_len) {
  if (!ctx) return QRKIT_EINVAL;
  Plan& P = ctx->plan;
  if (!P.valid) return fail(ctx, QRKIT_ESTATE, "qrkit_autotune before qrkit_plan");
  if (!J || !b || !p) return fail(ctx, QRKIT_EINVAL, "J, b and p are required");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const std::string key = plan_key(ctx);
  std::string value;
  qrkit_status st = QRKIT_OK;
  if (P.s.kind == QRKIT_STRUCT_BLOCKS) {
    if (P.composed) return fail(ctx, QRKIT_EUNSUPPORTED, "qrkit_autotune: block structures without coupling");
    BlockChoice c;
    if (cache_lookup(cache_path, key, value) && parse_choice(value, c)) {
      if ((st = apply_choice(ctx, c)) != QRKIT_OK) return st;
    } else {
      float best = 1e30f;
      BlockChoice bc;
      for (const BlockChoice& cand : block_candidates(elem_size(ctx))) {
        if ((st = apply_choice(ctx, cand)) != QRKIT_OK) return st;
        float ms = 0.f;
        st = time_runs(ctx, [&] { return launch_block_solve(ctx, J, b, nullptr, p, nullptr, refine_steps); }, ms);
        if (st != QRKIT_OK) return st;
        if (ms < best) {
          best = ms;
          bc = cand;
        }
      }
      if ((st = apply_choice(ctx, bc)) != QRKIT_OK) return st;
      value = choice_str(bc);
      cache_store(cache_path, key, value);
    }
    ctx->factored = false;
  } else {
    Band& B = ctx->band;
    if (!B.parallel || !B.cr) return fail(ctx, QRKIT_EUNSUPPORTED, "qrkit_autotune: parallel banded plans only");
    int tr = 1, sp = 1;
    if (cache_lookup(cache_path, key, value) && sscanf(value.c_str(), "compress %d %d", &tr, &sp) == 2) {
      if ((st = cr_set_strategy(ctx, *B.cr, tr != 0, sp)) != QRKIT_OK) return st;
    } else {
      float best = 1e30f;
      int btr = 1, bsp = 1;
      for (const int cand_tr : {1, 0})
        for (const int cand_sp : {1, 2, 4, 8}) {
          if (cand_tr && cand_sp != 1) continue;
          if ((st = cr_set_strategy(ctx, *B.cr, cand_tr != 0, cand_sp)) != QRKIT_OK) return st;
          float ms = 0.f;
          st = time_runs(ctx, [&] { return banded_factor_solve(ctx, J, b, nullptr, 1e-3, p, refine_steps); }, ms);
          if (st != QRKIT_OK) return st;
          if (ms < best) {
            best = ms;
            btr = cand_tr;
            bsp = cand_sp;
          }
        }
      if ((st = cr_set_strategy(ctx, *B.cr, btr != 0, bsp)) != QRKIT_OK) return st;
      std::ostringstream v;
      v << "compress " << btr << " " << bsp;
      value = v.str();
      cache_store(cache_path, key, value);
    }
    ctx->band_factored = false;
  }
  if (chosen && chosen_len > 0) {
    std::snprintf(chosen, (size_t)chosen_len, "%s", value.c_str());
  }
  return QRKIT_OK;
}

extern "C" qrkit_status qrkit_apply_tuning(qrkit_ctx* ctx, const char* choice) {
  if (!ctx) return QRKIT_EINVAL;
  if (!choice) return fail(ctx, QRKIT_EINVAL, "choice is required");
  Plan& P = ctx->plan;
  if (!P.valid) return fail(ctx, QRKIT_ESTATE, "qrkit_apply_tuning before qrkit_plan");
  QRKIT_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const std::string v(choice);
  if (P.s.kind == QRKIT_STRUCT_BLOCKS) {
    if (P.composed) return fail(ctx, QRKIT_EUNSUPPORTED, "qrkit_apply_tuning: block structures without coupling");
    BlockChoice c;
    if (!parse_choice(v, c)) return fail(ctx, QRKIT_EINVAL, "cannot parse block mapping '" + v + "'");
    const qrkit_status st = apply_choice(ctx, c);
    ctx->factored = false;
    return st;
  }
  Band& B = ctx->band;
  if (!B.parallel || !B.cr) return fail(ctx, QRKIT_EUNSUPPORTED, "qrkit_apply_tuning: parallel banded plans only");
  int tr = 1, sp = 1;
  if (sscanf(v.c_str(), "compress %d %d", &tr, &sp) != 2)
    return fail(ctx, QRKIT_EINVAL, "cannot parse compression strategy '" + v + "'");
  const qrkit_status st = cr_set_strategy(ctx, *B.cr, tr != 0, sp);
  ctx->band_factored = false;
  return st;
}
