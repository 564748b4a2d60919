// Instantiation of the warp-task refinement kernel with the double residual (one kernel per
// translation unit, so that the variants compile in parallel).
#include "block_tasks.cuh"

namespace qrkit {
namespace tasks {

template <int RES>
cudaError_t refine_setup(size_t smem, int threads, int* per_sm) {
  auto k = block_task_refine_kernel<RES>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem);
}

template <int RES>
cudaError_t refine_launch(const RefineTaskArgs& A, unsigned grid, int threads, size_t smem, cudaStream_t st) {
  block_task_refine_kernel<RES><<<grid, threads, smem, st>>>(A);
  return cudaGetLastError();
}

template cudaError_t refine_setup<1>(size_t, int, int*);
template cudaError_t refine_launch<1>(const RefineTaskArgs&, unsigned, int, size_t, cudaStream_t);

}  // namespace tasks
}  // namespace qrkit
