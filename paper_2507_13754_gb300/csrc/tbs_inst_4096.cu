// tbs_inst_4096.cu -- the row and column kernels and their launchers for M = 4096
// (one translation unit per group of sizes, so that they compile in
// parallel).
#include "tbs_kernels.cuh"

namespace tbs {
TBS_PER_M(, 4096)
}  // namespace tbs
