// Batched TS-SpGEMM: many independent products of uneven shapes per launch.
#include "common.cuh"
#include "kernels.h"

namespace ts {}  // namespace ts
