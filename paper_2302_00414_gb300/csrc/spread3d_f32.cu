// Three-dimensional spreading, float instantiation.
#include "spread3d.cuh"

namespace infft {

template infft_status spread3d_try<float>(JobSet<float>&, cudaStream_t, bool*);

}  // namespace infft
