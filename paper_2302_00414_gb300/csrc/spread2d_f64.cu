// Two-dimensional spreading, double instantiation.
#include "spread2d.cuh"

namespace infft {

template infft_status spread2d_try<double>(JobSet<double>&, cudaStream_t, bool*);

}  // namespace infft
