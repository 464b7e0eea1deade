// tbs_inst_128_256.cu -- the row and column kernels and their launchers for M = 128 and 256
// (one translation unit per group of sizes, so that they compile in
// parallel).
#include "tbs_kernels.cuh"

namespace tbs {
TBS_PER_M(, 128)
TBS_PER_M(, 256)
}  // namespace tbs
