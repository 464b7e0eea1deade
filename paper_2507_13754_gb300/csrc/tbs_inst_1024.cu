// tbs_inst_1024.cu -- the row and column kernels and their launchers for M = 1024
// (one translation unit per group of sizes, so that they compile in
// parallel).
#include "tbs_kernels.cuh"

namespace tbs {
TBS_PER_M(, 1024)
}  // namespace tbs
