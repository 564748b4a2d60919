// Instantiation of the warp-task refinement kernel (one kernel per translation unit, so that
// the variants compile in parallel).
#include "block_tasks.cuh"

namespace qrkit {
namespace tasks {

cudaError_t refine_setup(size_t smem, int threads, int* per_sm) {
  auto k = block_task_refine_kernel<0>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem);
}

cudaError_t refine_launch(const RefineTaskArgs& A, unsigned grid, int threads, size_t smem, cudaStream_t st) {
  block_task_refine_kernel<0><<<grid, threads, smem, st>>>(A);
  return cudaGetLastError();
}

}  // namespace tasks
}  // namespace qrkit
