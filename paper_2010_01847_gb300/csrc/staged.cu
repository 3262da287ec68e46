// Bulk-copy staged stream-collide kernel (placeholder until implemented).
#include "lbm_kernels.h"

namespace plbm {

bool staged_supported(int, int, int) { return false; }

template <typename T>
cudaError_t launch_step_staged(const T *, T *, int, int, int, int,
                               const Coef<typename Store<T>::C> &, cudaStream_t) {
    return cudaErrorNotSupported;
}

template cudaError_t launch_step_staged<float>(const float *, float *, int, int, int, int,
                                               const Coef<float> &, cudaStream_t);
template cudaError_t launch_step_staged<double>(const double *, double *, int, int, int, int,
                                                const Coef<double> &, cudaStream_t);
template cudaError_t launch_step_staged<__half>(const __half *, __half *, int, int, int, int,
                                                const Coef<float> &, cudaStream_t);
template cudaError_t launch_step_staged<__nv_bfloat16>(const __nv_bfloat16 *, __nv_bfloat16 *,
                                                       int, int, int, int, const Coef<float> &,
                                                       cudaStream_t);

}  // namespace plbm
