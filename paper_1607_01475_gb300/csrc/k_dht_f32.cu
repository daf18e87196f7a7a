// FP32 instantiations of the Hartley transform passes and the middle pass
// (the mixed solver's inner iteration).
#include "dht_kernels.cuh"

namespace psd {

#define PSD_INST(T)                                                                                    \
  template cudaError_t launch_dht_rows<T>(const T*, T*, int, int, T, const int*, const AxisTables<T>&, \
                                          cudaStream_t);                                               \
  template cudaError_t launch_dht_cols<T>(T*, const KParams&, int, T, const int*, const AxisTables<T>&, \
                                          cudaStream_t);                                               \
  template cudaError_t launch_mid<T>(T*, const KParams&, Ctrl*, double*, T*, T*, const AxisTables<T>&,  \
                                     cudaStream_t);                                                    \
  template cudaError_t launch_spec6_combine<T>(T*, const T*, const KParams&, const AxisTables<T>&,      \
                                               cudaStream_t);                                          \
  template cudaError_t launch_spec_apply_T<T>(T*, T, const KParams&, const AxisTables<T>&, cudaStream_t);
PSD_INST(float)

void init_dht_attributes_f32() {
  set_attrs_T<float, 8>();
  set_attrs_T<float, 16>();
  set_attrs_T<float, 32>();
  set_attrs_T<float, 64>();
  set_attrs_T<float, 128>();
  set_attrs_T<float, 256>();
  set_attrs_T<float, 512>();
  set_attrs_T<float, 1024>();
}

}  // namespace psd
