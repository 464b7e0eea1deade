// tbs_inst_2048.cu -- the row and column kernels and their launchers for M = 2048
// (one translation unit per group of sizes, so that they compile in
// parallel).
#include "tbs_kernels.cuh"

namespace tbs {
TBS_PER_M(, 2048)
}  // namespace tbs
