// Instantiation of the warp-task block solve kernel for float
// (one kernel per translation unit, so that the variants compile in parallel).
#include "block_tasks.cuh"

namespace qrkit {
namespace tasks {

template <>
cudaError_t kernel_setup<float, false>(size_t smem, int threads, int* per_sm) {
  auto k = block_task_kernel<float, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem);
}

template <>
cudaError_t kernel_launch<float, false>(const TaskArgs<float>& A, unsigned grid, int threads, size_t smem,
                                  cudaStream_t st) {
  block_task_kernel<float, false><<<grid, threads, smem, st>>>(A);
  return cudaGetLastError();
}

}  // namespace tasks
}  // namespace qrkit
