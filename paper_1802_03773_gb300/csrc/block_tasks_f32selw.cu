// Instantiation of the warp-task block solve kernel for float with the refinement selection,
// blocks of 5 to 8 columns
// (one or two kernels per translation unit, so that the variants compile in parallel).
#include "block_tasks.cuh"

namespace qrkit {
namespace tasks {

QRKIT_TASK_KERNEL_ENTRIES(float, true, 2)

}  // namespace tasks
}  // namespace qrkit
