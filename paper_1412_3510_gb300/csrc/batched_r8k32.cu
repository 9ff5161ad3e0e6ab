// The batched kernel with pass tiles of 8 rows (columns) of A per thread, 32 deep.
#include "batched_kernels.cuh"

namespace rpca {

int launch_batched_r8k32(const BatchLaunch &a) { return launch_batched_rpt<8, 32>(a); }

}  // namespace rpca
