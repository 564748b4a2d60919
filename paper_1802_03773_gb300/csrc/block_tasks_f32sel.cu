// Instantiation of the warp-task block solve kernel for float with the refinement selection
// (one kernel per translation unit, so that the variants compile in parallel).
#include "block_tasks.cuh"

namespace qrkit {
namespace tasks {

template <>
cudaError_t kernel_setup<float, true>(size_t smem, int threads, int* per_sm) {
  auto k = block_task_kernel<float, true>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem);
}

template <>
cudaError_t kernel_launch<float, true>(const TaskArgs<float>& A, unsigned grid, int threads, size_t smem,
                                  cudaStream_t st) {
  block_task_kernel<float, true><<<grid, threads, smem, st>>>(A);
  return cudaGetLastError();
}

}  // namespace tasks
}  // namespace qrkit
