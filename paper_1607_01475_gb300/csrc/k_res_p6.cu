// Residual and line-search kernels instantiated for the vertex factor
// |G|^4 = (|G|^2)^2 (p = 6), in both precisions and every residual mode.
#include "stencil_kernels.cuh"

namespace psd {
namespace detail {

#define PSD_INST_PK(T)                                                                                   \
  template cudaError_t res_impl<T, PK_6, RM_PLAIN>(const ResArgs<T>&, const KParams&, Ctrl*, double*,      \
                                                    cudaStream_t);                                        \
  template cudaError_t res_impl<T, PK_6, RM_INNER>(const ResArgs<T>&, const KParams&, Ctrl*, double*,      \
                                                    cudaStream_t);                                        \
  template cudaError_t res_impl<T, PK_6, RM_HVP>(const ResArgs<T>&, const KParams&, Ctrl*, double*,        \
                                                  cudaStream_t);                                          \
  template cudaError_t ls_impl<T, PK_6, true>(const T*, const T*, const T*, const KParams&, Ctrl*, double*, \
                                               cudaStream_t);                                             \
  template cudaError_t ls_impl<T, PK_6, false>(const T*, const T*, const T*, const KParams&, Ctrl*, double*, \
                                                cudaStream_t);
PSD_INST_PK(float)
PSD_INST_PK(double)
#undef PSD_INST_PK

}  // namespace detail
}  // namespace psd
