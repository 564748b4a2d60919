// Instantiation of the warp-task block solve kernel for float with the refinement selection,
// blocks of at most 4 columns
// (one or two kernels per translation unit, so that the variants compile in parallel).
#include "block_tasks.cuh"

namespace qrkit {
namespace tasks {

QRKIT_TASK_KERNEL_ENTRIES(float, true, 1)

}  // namespace tasks
}  // namespace qrkit
