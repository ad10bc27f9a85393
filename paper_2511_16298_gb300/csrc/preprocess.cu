// Preprocessing kernel (Sec. II-A; inputs Table I, outputs Table IV Groups
// 1-2): one thread per 3D Gaussian projects its mean and covariance for one
// pinhole camera (proj::project, project.cuh) and writes the 16-byte record
// the sort path consumes (2D mean, depth, radius) and the 16-byte
// conic/opacity word.  Traffic: 48 bytes in, 32 bytes out per Gaussian (16
// without the conic).
#include "project.cuh"

namespace tdgs {

namespace {

__global__ void __launch_bounds__(256)
    k_preprocess(const float4* __restrict__ g, const float4* __restrict__ cov, uint32_t n, CameraDev cam,
                 float4* __restrict__ rec, float4* __restrict__ conic) {
  const float2 lim = proj::slope_limits(cam);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 p = __ldg(g + i);
    const float4 c0 = __ldg(cov + 2 * static_cast<size_t>(i));
    const float4 c1 = __ldg(cov + 2 * static_cast<size_t>(i) + 1);
    float4 out, co;
    proj::project(p, c0, c1, cam, lim, out, co);
    rec[i] = out;
    if (conic) conic[i] = co;
  }
}

}  // namespace

cudaError_t launch_preprocess(const float4* g, const float4* cov, uint32_t n, const CameraDev& cam, float4* rec,
                              float4* conic, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint32_t blocks = (n + 255) / 256;
  const uint32_t grid = blocks < 152u * 16u ? blocks : 152u * 16u;
  k_preprocess<<<grid, 256, 0, s>>>(g, cov, n, cam, rec, conic);
  return cudaGetLastError();
}

}  // namespace tdgs
