// Three-dimensional spreading, double instantiation.
#include "spread3d.cuh"

namespace infft {

template infft_status spread3d_try<double>(JobSet<double>&, cudaStream_t, bool*);

}  // namespace infft
