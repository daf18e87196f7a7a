// FP64 instantiations of the Hartley transform passes, the middle pass and
// the spectral helpers (the plain FP64 solver, the FP64 preconditioner and
// residual entry points).
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
PSD_INST(double)
template cudaError_t launch_spec_quad<double>(const double*, const KParams&, Ctrl*, double*, const AxisTables<double>&,
                                              cudaStream_t);

void init_dht_attributes_f64() {
  set_attrs_T<double, 8>();
  set_attrs_T<double, 16>();
  set_attrs_T<double, 32>();
  set_attrs_T<double, 64>();
  set_attrs_T<double, 128>();
  set_attrs_T<double, 256>();
  set_attrs_T<double, 512>();
  set_attrs_T<double, 1024>();
}

}  // namespace psd
