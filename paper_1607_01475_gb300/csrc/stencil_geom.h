// Launch geometry of the residual and line-search kernels, shared by the
// translation units that instantiate them (one per kind of vertex factor)
// and by the dispatching launchers.
#pragma once

#include "kernels.h"

namespace psd {

constexpr int BX = 32;   // tile width (x)
constexpr int BY3 = 8;   // tile height (y), 3D
constexpr int BY2 = 32;  // tile height (y), 2D
constexpr int NT = 256;  // threads per block

enum ResKind { RK_2D, RK_SMALL3D, RK_COL, RK_RB4 };
struct ResGeom {
  int kind;
  dim3 grid;
  int zc;
};
// Geometry for a kernel whose __launch_bounds__ guarantee ctas_per_sm
// resident CTAs per SM (defined in k_stencil.cu).
ResGeom res_geometry(const KParams& kp, bool fp32, int ctas_per_sm);
// The residual launch: k_res3d_rb keeps 2 CTAs per SM resident, k_res3d_col 3.
ResGeom residual_geometry(const KParams& kp, bool fp32);

namespace detail {
// Residual and line-search launchers for one vertex-factor kind PK (PK_4,
// PK_6 or PK_GEN), explicitly instantiated by k_res_p4.cu, k_res_p6.cu and
// k_res_pgen.cu.
template <typename T, int PK, int MODE>
cudaError_t res_impl(const ResArgs<T>& a, const KParams& kp, Ctrl* ctrl, double* partials, cudaStream_t st);
template <typename T, int PK, bool INNER>
cudaError_t ls_impl(const T* u, const T* ubase, const T* d, const KParams& kp, Ctrl* ctrl, double* partials,
                    cudaStream_t st);
}  // namespace detail

}  // namespace psd
