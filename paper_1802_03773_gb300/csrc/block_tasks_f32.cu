// Instantiation of the warp-task block solve kernel for float without the refinement selection
// (every key)
// (one or two kernels per translation unit, so that the variants compile in parallel).
#include "block_tasks.cuh"

namespace qrkit {
namespace tasks {

QRKIT_TASK_KERNEL_ENTRIES(float, false, 0)

}  // namespace tasks
}  // namespace qrkit
