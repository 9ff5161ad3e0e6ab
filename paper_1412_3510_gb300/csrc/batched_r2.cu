// The batched kernel with 2 rows (or columns) of A per thread in its passes.
#include "batched_kernels.cuh"

namespace rpca {

int launch_batched_r2(const BatchLaunch &a) { return launch_batched_rpt<2>(a); }

}  // namespace rpca
