// Device check of psd::recip_ge1<float>, the reciprocal that every FP32
// symbol division of the preconditioner goes through (1 / P with
// P = 1 + mu (...) >= 1): the hardware estimate refined by one
// Newton-Raphson step, against the correctly rounded reciprocal __frcp_rn,
// over x in [1, 2^125) (random mantissas in every binade, plus the binade
// edges).  Built and run by tests/test_recip.py on a GPU.  Prints the worst
// distance in units in the last place and the share of exactly rounded
// results; exit status 0 = every result within 1 ulp.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../paper_1607_01475_gb300/csrc/psd_common.cuh"

__global__ void k_recip(const float* x, float* approx, float* exact, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    approx[i] = psd::recip_ge1(x[i]);
    exact[i] = __frcp_rn(x[i]);
  }
}

static uint64_t rng_state = 0x5eed1607ULL;
static uint64_t next_u64() {  // SplitMix64
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static int32_t bits(float v) {
  int32_t b;
  std::memcpy(&b, &v, 4);
  return b;
}

int main() {
  std::vector<float> x;
  for (int e = 0; e < 125; ++e) {
    const uint32_t expo = (uint32_t)(127 + e) << 23;
    for (uint32_t m : {0u, 1u, 0x7FFFFFu, 0x400000u}) {
      uint32_t b = expo | m;
      float v;
      std::memcpy(&v, &b, 4);
      x.push_back(v);
    }
    for (int t = 0; t < 8192; ++t) {
      uint32_t b = expo | (uint32_t)(next_u64() & 0x7FFFFFu);
      float v;
      std::memcpy(&v, &b, 4);
      x.push_back(v);
    }
  }
  const int n = (int)x.size();
  float *dx = nullptr, *da = nullptr, *de = nullptr;
  if (cudaMalloc(&dx, n * sizeof(float)) != cudaSuccess || cudaMalloc(&da, n * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&de, n * sizeof(float)) != cudaSuccess) {
    std::printf("cudaMalloc failed\n");
    return 2;
  }
  cudaMemcpy(dx, x.data(), n * sizeof(float), cudaMemcpyHostToDevice);
  k_recip<<<152 * 4, 256>>>(dx, da, de, n);
  std::vector<float> a(n), ex(n);
  cudaMemcpy(a.data(), da, n * sizeof(float), cudaMemcpyDeviceToHost);
  const cudaError_t err = cudaMemcpy(ex.data(), de, n * sizeof(float), cudaMemcpyDeviceToHost);
  if (err != cudaSuccess) {
    std::printf("CUDA error: %s\n", cudaGetErrorString(err));
    return 2;
  }
  int worst = 0, exact_count = 0;
  float worst_x = 0.0f;
  for (int i = 0; i < n; ++i) {
    // both results are positive normal floats: the distance of their bit
    // patterns is the distance in units in the last place
    const int d = std::abs(bits(a[i]) - bits(ex[i]));
    if (d == 0) ++exact_count;
    if (d > worst) {
      worst = d;
      worst_x = x[i];
    }
  }
  std::printf("n %d worst %d ulp (x = %.9g) exactly rounded %.6f\n", n, worst, worst_x,
              (double)exact_count / n);
  cudaFree(dx);
  cudaFree(da);
  cudaFree(de);
  if (worst <= 1) std::printf("OK\n");
  return worst <= 1 ? 0 : 1;
}
