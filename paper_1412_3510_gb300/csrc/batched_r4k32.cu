// The batched kernel with pass tiles of 4 rows (columns) of A per thread, 32 deep.
#include "batched_kernels.cuh"

namespace rpca {

int launch_batched_r4k32(const BatchLaunch &a) { return launch_batched_rpt<4, 32>(a); }

}  // namespace rpca
