// Float-float (double-word on FP64 storage) Hartley transform passes of the
// mixed solver's outer loop, with the fused epilogues of the last pass.
#include "dht_kernels.cuh"

namespace psd {
namespace {

template <int N>
void set_attrs_ff() {
  constexpr int RF = radix_pass<ff>();
  cudaFuncSetAttribute(k_dht_rows<ff, ff, N, RF, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
  cudaFuncSetAttribute(k_dht_rows<ff, ff, N, RF, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
  cudaFuncSetAttribute(k_dht_cols<ff, ff, N, RF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
  cudaFuncSetAttribute(k_dht_last_ff<N, RF, EPI_THETA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kMaxSmemPre);
  cudaFuncSetAttribute(k_dht_last_ff<N, RF, EPI_RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kMaxSmemPre);
}

}  // namespace

cudaError_t launch_dht_rows_ff(const double* src, ff* dst, int nx, int nrows, const AxisTables<ff>& tb,
                               cudaStream_t st, const int* skip) {
  PSD_DISPATCH_N(nx, (rows_impl<ff, ff, NN, double>(src, dst, nrows, ff(1.0f, 0.0f), skip, tb.twc[0], tb.tws[0],
                                                     st)));
}

cudaError_t launch_dht_cols_ff(ff* data, const KParams& kp, int ax, const AxisTables<ff>& tb, cudaStream_t st,
                               const int* skip) {
  const ff scale(1.0f, 0.0f);
  const int n = ax == 1 ? kp.ny : kp.nz;
  const size_t line_stride = ax == 1 ? (size_t)kp.nx : (size_t)kp.nx * kp.ny;
  const size_t outer_stride = ax == 1 ? (size_t)kp.nx * kp.ny : (size_t)kp.nx;
  const int nouter = ax == 1 ? kp.nz : kp.ny;
  PSD_DISPATCH_N(n, (cols_impl<ff, ff, NN>(data, kp.nx, nouter, line_stride, outer_stride, scale, skip,
                                           tb.twc[ax], tb.tws[ax], st)));
}

cudaError_t launch_dht_rows_ff_from_f32(const float* src, ff* dst, int nx, int nrows, const AxisTables<ff>& tb,
                                        cudaStream_t st, const int* skip) {
  PSD_DISPATCH_N(nx, (rows_impl<ff, ff, NN, float>(src, dst, nrows, ff(1.0f, 0.0f), skip, tb.twc[0], tb.tws[0],
                                                    st)));
}

template <int N>
cudaError_t last_ff_impl(const ff* data, double* theta, float* out32, const KParams& kp, Ctrl* ctrl,
                         double* partials, const AxisTables<ff>& tb, cudaStream_t st, double* dc, const int* skip) {
  constexpr int RM = radix_pass<ff>();
  using F = LineFFT<ff, N, RM>;
  const int nx = kp.nx;
  const int pairs = pick_pairs<ff, N, RM, false>(nx / 2);
  const bool d3 = kp.dim == 3;
  const size_t line_stride = d3 ? (size_t)nx * kp.ny : (size_t)nx;
  const size_t outer_stride = d3 ? (size_t)nx : 0;
  const int nouter = d3 ? kp.ny : 1;
  const int ax = d3 ? 2 : 1;
  dim3 grid(nx / (2 * pairs), nouter);
  const size_t sm = align16(pairs * pair_smem<ff, N, RM, false>()) + (size_t)N * pairs * sizeof(double2);
  if (sm > kMaxSmemPre) return cudaErrorInvalidConfiguration;
  const ff* symo = d3 ? tb.sym[1] : nullptr;
  if (out32 == nullptr)
    k_dht_last_ff<N, RM, EPI_THETA><<<grid, pairs * F::TS, sm, st>>>(data, theta, out32, line_stride, outer_stride,
                                                                    kp, ctrl, partials, tb.twc[ax], tb.tws[ax],
                                                                    tb.sym[0], symo, tb.sym[ax], dc, skip);
  else
    k_dht_last_ff<N, RM, EPI_RESID><<<grid, pairs * F::TS, sm, st>>>(data, theta, out32, line_stride, outer_stride,
                                                                    kp, ctrl, partials, tb.twc[ax], tb.tws[ax],
                                                                    tb.sym[0], symo, tb.sym[ax], nullptr, skip);
  return cudaGetLastError();
}

cudaError_t launch_dht_last_ff(const ff* data, double* theta, float* out32, const KParams& kp, Ctrl* ctrl,
                               double* partials, const AxisTables<ff>& tb, cudaStream_t st, double* dc,
                               const int* skip) {
  const int n = kp.dim == 3 ? kp.nz : kp.ny;
  PSD_DISPATCH_N(n, (last_ff_impl<NN>(data, theta, out32, kp, ctrl, partials, tb, st, dc, skip)));
}




void init_dht_attributes_f32();
void init_dht_attributes_f64();

void init_dht_attributes() {
  init_dht_attributes_f32();
  init_dht_attributes_f64();
  set_attrs_ff<8>();
  set_attrs_ff<16>();
  set_attrs_ff<32>();
  set_attrs_ff<64>();
  set_attrs_ff<128>();
  set_attrs_ff<256>();
  set_attrs_ff<512>();
  set_attrs_ff<1024>();
}

}  // namespace psd
