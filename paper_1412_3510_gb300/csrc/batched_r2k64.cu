// The batched kernel with pass tiles of 2 rows (columns) of A per thread, 64 deep.
#include "batched_kernels.cuh"

namespace rpca {

int launch_batched_r2k64(const BatchLaunch &a) { return launch_batched_rpt<2, 64>(a); }

}  // namespace rpca
