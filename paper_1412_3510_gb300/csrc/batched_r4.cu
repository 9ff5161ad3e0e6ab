// The batched kernel with 4 rows (or columns) of A per thread in its passes.
#include "batched_kernels.cuh"

namespace rpca {

int launch_batched_r4(const BatchLaunch &a) { return launch_batched_rpt<4>(a); }

}  // namespace rpca
