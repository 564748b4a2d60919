// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qrkit.h"

namespace qrkit {

// Device status word values mirror qrkit_status.  Kernels record the first failure with
// atomicCAS and never trap.
constexpr int kDevOk = QRKIT_OK;

// Tile budgets of the persistent block kernels (one tile = consecutive blocks staged in
// shared memory; the plan cuts tiles greedily so no budget is exceeded).
struct TileBudget {
  int blocks;   // blocks per tile
  int values;   // J values per tile
  int rows;     // J rows per tile
  int cols;     // columns per tile
};

// A device buffer owned by the context.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Plan {
  bool valid = false;
  qrkit_structure s{};
  int64_t K = 0;          // blocks
  int64_t rows = 0;       // sum n_i (J rows)
  int64_t cols = 0;       // sum m_i (block columns)
  int64_t values = 0;     // sum n_i m_i
  int max_n = 0, max_m = 0;
  // host copies
  std::vector<uint8_t> n, m;
  std::vector<int64_t> tile_block, tile_val, tile_row, tile_col;
  int64_t num_tiles = 0;
  TileBudget budget{};
  // device copies
  DevBuf d_n, d_m, d_tile_block, d_tile_val, d_tile_row, d_tile_col;
};

struct Workspace {
  DevBuf factor;   // factor values (J packing)
  DevBuf tau;      // sum m_i
};

}  // namespace qrkit

struct qrkit_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = QRKIT_FP32_REFINED;
  int num_sms = 0;
  size_t max_smem_optin = 0;
  std::string last_error;
  qrkit::Plan plan;
  qrkit::Workspace ws;
  int* d_status = nullptr;   // device status word
  int64_t launches = 0;
  bool factored = false;
};

namespace qrkit {

qrkit_status fail(qrkit_ctx* ctx, qrkit_status st, const std::string& msg);
qrkit_status cuda_fail(qrkit_ctx* ctx, cudaError_t e, const char* what);
qrkit_status ensure(qrkit_ctx* ctx, DevBuf& buf, size_t bytes, const char* what);
void release(DevBuf& buf);
inline size_t elem_size(const qrkit_ctx* ctx) {
  return ctx->precision == QRKIT_FP64 ? sizeof(double) : sizeof(float);
}

// Launchers implemented in the kernel translation units.
qrkit_status launch_block_solve(qrkit_ctx* ctx, const void* J, const void* b, const void* D,
                                void* p, void* qtb, int refine_steps);

}  // namespace qrkit

#define QRKIT_CUDA_TRY(ctx, call)                                  \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return ::qrkit::cuda_fail(ctx, e_, #call); \
  } while (0)
