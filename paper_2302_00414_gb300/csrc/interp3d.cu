// Fixed-m interpolation for d = 3 (Algorithm 2.1 step 3).
#include "interp.cuh"

namespace infft {

template <class R>
infft_status interp3d_try(JobSet<R>& js, cudaStream_t st, bool* used) {
    return interp_try_d<R, 3>(js, st, used);
}

template infft_status interp3d_try<float>(JobSet<float>&, cudaStream_t, bool*);
template infft_status interp3d_try<double>(JobSet<double>&, cudaStream_t, bool*);

}  // namespace infft
