// Residual and line-search kernels instantiated for the vertex factor
// |G|^{p-2} of a general p (pow), in both precisions and every residual mode.
#include "stencil_kernels.cuh"

namespace psd {
namespace detail {

#define PSD_INST_PK(T)                                                                                   \
  template cudaError_t res_impl<T, PK_GEN, RM_PLAIN>(const ResArgs<T>&, const KParams&, Ctrl*, double*,      \
                                                    cudaStream_t);                                        \
  template cudaError_t res_impl<T, PK_GEN, RM_INNER>(const ResArgs<T>&, const KParams&, Ctrl*, double*,      \
                                                    cudaStream_t);                                        \
  template cudaError_t res_impl<T, PK_GEN, RM_HVP>(const ResArgs<T>&, const KParams&, Ctrl*, double*,        \
                                                  cudaStream_t);                                          \
  template cudaError_t ls_impl<T, PK_GEN, true>(const T*, const T*, const T*, const KParams&, Ctrl*, double*, \
                                               cudaStream_t);                                             \
  template cudaError_t ls_impl<T, PK_GEN, false>(const T*, const T*, const T*, const KParams&, Ctrl*, double*, \
                                                cudaStream_t);
PSD_INST_PK(float)
PSD_INST_PK(double)
#undef PSD_INST_PK

}  // namespace detail
}  // namespace psd
