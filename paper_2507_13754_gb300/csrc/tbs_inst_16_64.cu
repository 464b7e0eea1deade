// tbs_inst_16_64.cu -- the row and column kernels and their launchers for M = 16, 32 and 64
// (one translation unit per group of sizes, so that they compile in
// parallel).
#include "tbs_kernels.cuh"

namespace tbs {
TBS_PER_M(, 16)
TBS_PER_M(, 32)
TBS_PER_M(, 64)
}  // namespace tbs
