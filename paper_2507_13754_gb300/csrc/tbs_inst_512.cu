// tbs_inst_512.cu -- the row and column kernels and their launchers for M = 512
// (one translation unit per group of sizes, so that they compile in
// parallel).
#include "tbs_kernels.cuh"

namespace tbs {
TBS_PER_M(, 512)
}  // namespace tbs
