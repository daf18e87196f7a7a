// Fused x and y DHT passes of one z-plane per thread-block cluster (FP32,
// nx = ny = N): the preconditioner's transform (Sec. 6) is separable and the
// DHT is its own inverse up to 1/N, so both the forward and the inverse half
// of the 3D transform can apply the x lines and then the y lines of each
// plane.  A cluster of 8 CTAs holds one N x N plane in its distributed
// shared memory:
//   phase 1: CTA r transforms the x lines y = r N/8 .. (r+1) N/8 - 1 of the
//            plane into its own shared memory;
//   cluster barrier;
//   phase 2: CTA r gathers the y lines of the columns x = r N/8 .. from all
//            8 CTAs' shared memory, transforms them and writes the plane.
// The plane crosses HBM once in each direction (8 bytes per cell, against
// 16 for two separate passes).
#include <cooperative_groups.h>

#include "fft_line.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace psd {
namespace {

constexpr int kCluster = 8;

template <int N>
struct XY {
  static constexpr int R = 16;                  // radix of the line FFT
  using F = LineFFT<float, N, R>;
  static constexpr int TS = F::TS;              // threads per line pair
  static constexpr int ROWS = N / kCluster;     // lines per CTA in each phase
  static constexpr int PAIRS = ROWS / 2;
  static constexpr int THREADS = PAIRS * TS;
  static constexpr int L = F::L;
  // pair strides (words) spreading each phase's accesses over the banks:
  // phase 1 puts 32/TS pairs in a warp, phase 2 PAIRS pairs
  static constexpr int M1 = TS >= 32 ? 1 : (TS < 2 ? 2 : TS), R1 = TS >= 32 ? 0 : (TS < 2 ? 1 : TS / 2);
  static constexpr int K2 = PAIRS < 16 ? PAIRS : 16, M2 = 32 / K2, R2 = 16 / K2;
  static constexpr int LS1 = L + (((R1 - L) % M1) + M1) % M1;
  static constexpr int LS2 = L + (((R2 - L) % M2) + M2) % M2;
  static constexpr int LSM = LS1 > LS2 ? LS1 : LS2;
  static constexpr int PBS = N + 8;             // plane-buffer row stride (words)
  static constexpr size_t SMEM = ((size_t)ROWS * PBS + (size_t)PAIRS * 2 * LSM) * sizeof(float);
  static_assert(THREADS <= 1024 && PAIRS >= 1, "unsupported N");
};

template <int N>
__global__ void __cluster_dims__(kCluster, 1, 1) __launch_bounds__(XY<N>::THREADS)
    k_dht_xy(const float* src, float* dst, const int* done, const float* __restrict__ twxc,
             const float* __restrict__ twxs, const float* __restrict__ twyc, const float* __restrict__ twys) {
  using C = XY<N>;
  using F = typename C::F;
  // every CTA of the cluster reads the same flag (set before this launch),
  // so either all of them return here or none does
  if (done != nullptr && *done) return;
  extern __shared__ __align__(16) float smx[];
  float* pb = smx;                                  // [ROWS][PBS]: this CTA's x-transformed lines
  float* scratch = smx + (size_t)C::ROWS * C::PBS;  // line pairs of the FFTs
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const size_t plane = (size_t)N * N;
  const float* sp = src + (size_t)blockIdx.y * plane;
  float* dp = dst + (size_t)blockIdx.y * plane;
  const int tid = threadIdx.x;
  {
    // phase 1: x lines (2p, 2p + 1) of this CTA's row block
    const int p = tid / C::TS, j = tid - p * C::TS;
    float* sr = scratch + (size_t)p * 2 * C::LS1;
    float* si = sr + C::LS1;
    const float* r0 = sp + (size_t)(rank * C::ROWS + 2 * p) * N;
    float vr[F::R], vi[F::R];
#pragma unroll
    for (int q = 0; q < F::R; ++q) {
      vr[q] = r0[j + q * C::TS];
      vi[q] = r0[N + j + q * C::TS];
    }
    F::run(vr, vi, j, sr, si, twxc, twxs);
#pragma unroll
    for (int q = 0; q < F::R; ++q) {
      const int k = j + q * C::TS;
      float h1, h2;
      dht_split(sr, si, k, N, h1, h2);
      pb[(size_t)(2 * p) * C::PBS + k] = h1;
      pb[(size_t)(2 * p + 1) * C::PBS + k] = h2;
    }
  }
  cluster.sync();  // every CTA's row block is complete and visible to the cluster
  {
    // phase 2: y lines of the column pair (x, x + 1), x = rank ROWS + 2p
    const int p = tid % C::PAIRS, j = tid / C::PAIRS;
    float* sr = scratch + (size_t)p * 2 * C::LS2;
    float* si = sr + C::LS2;
    const int x = rank * C::ROWS + 2 * p;
    float vr[F::R], vi[F::R];
#pragma unroll
    for (int q = 0; q < F::R; ++q) {
      const int y = j + q * C::TS;
      const float* rpb = cluster.map_shared_rank(pb, y / C::ROWS);
      const float2 v = *reinterpret_cast<const float2*>(rpb + (size_t)(y % C::ROWS) * C::PBS + x);
      vr[q] = v.x;
      vi[q] = v.y;
    }
    F::run(vr, vi, j, sr, si, twyc, twys);
#pragma unroll
    for (int q = 0; q < F::R; ++q) {
      const int k = j + q * C::TS;
      float h1, h2;
      dht_split(sr, si, k, N, h1, h2);
      *reinterpret_cast<float2*>(dp + (size_t)k * N + x) = make_float2(h1, h2);
    }
  }
  cluster.sync();  // no CTA leaves while another may still read its row block
}

// The kernel's shared-memory limit, set once per process (thread-safe; first
// reached from psd_create, so never inside a stream capture).
template <int N>
cudaError_t xy_attr() {
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_dht_xy<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XY<N>::SMEM);
  return attr;
}

template <int N>
cudaError_t xy_impl(const float* src, float* dst, int nz, const int* done, const AxisTables<float>& tb,
                    cudaStream_t st) {
  using C = XY<N>;
  const cudaError_t attr = xy_attr<N>();
  if (attr != cudaSuccess) return attr;
  dim3 grid(kCluster, nz);
  k_dht_xy<N><<<grid, C::THREADS, C::SMEM, st>>>(src, dst, done, tb.twc[0], tb.tws[0], tb.twc[1], tb.tws[1]);
  return cudaGetLastError();
}

}  // namespace

bool dht_xy_supported(const KParams& kp) {
  return kp.dim == 3 && kp.nx == kp.ny && (kp.nx == 64 || kp.nx == 128 || kp.nx == 256);
}

cudaError_t prepare_dht_xy(const KParams& kp) {
  if (!dht_xy_supported(kp)) return cudaSuccess;
  switch (kp.nx) {
    case 64: return xy_attr<64>();
    case 128: return xy_attr<128>();
    default: return xy_attr<256>();
  }
}

cudaError_t launch_dht_xy(const float* src, float* dst, const KParams& kp, const int* done,
                          const AxisTables<float>& tb, cudaStream_t st) {
  switch (kp.nx) {
    case 64: return xy_impl<64>(src, dst, kp.nz, done, tb, st);
    case 128: return xy_impl<128>(src, dst, kp.nz, done, tb, st);
    case 256: return xy_impl<256>(src, dst, kp.nz, done, tb, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace psd
