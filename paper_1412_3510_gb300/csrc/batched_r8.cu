// The batched kernel with 8 rows (or columns) of A per thread in its passes.
#include "batched_kernels.cuh"

namespace rpca {

int launch_batched_r8(const BatchLaunch &a) { return launch_batched_rpt<8>(a); }

}  // namespace rpca
