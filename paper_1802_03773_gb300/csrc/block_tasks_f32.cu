// Instantiation of the warp-task block solve kernel for float, both key classes
// (one or two kernels per translation unit, so that the variants compile in parallel).
#include "block_tasks.cuh"

namespace qrkit {
namespace tasks {

QRKIT_TASK_KERNEL_ENTRIES(float, false, 1)
QRKIT_TASK_KERNEL_ENTRIES(float, false, 2)

}  // namespace tasks
}  // namespace qrkit
