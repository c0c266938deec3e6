// Two-dimensional spreading, float instantiation.
#include "spread2d.cuh"

namespace infft {

template infft_status spread2d_try<float>(JobSet<float>&, cudaStream_t, bool*);

}  // namespace infft
