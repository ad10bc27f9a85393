// Projection of one 3D Gaussian for one camera (the preprocessing stage,
// Sec. II-A; Table I inputs, Table IV outputs), shared by the
// preprocessing kernel and the count kernel that fuses it.  Every
// floating-point step is an explicitly rounded float32 operation
// (__fmul_rn, __fadd_rn, __fdiv_rn, __fsqrt_rn: no contraction into fused
// multiply-adds) in a fixed order, because the integer radius is decided by
// this arithmetic:
//   t = R p + T; culled unless t.z > near
//   u = t.x / t.z, v = t.y / t.z; mean = (fx u + cx, fy v + cy)
//   uc, vc = u, v clamped to +-0.65 W / fx, +-0.65 H / fy (1.3 x the half
//   field of view)
//   J = [[fx / t.z, 0, -fx uc / t.z], [0, fy / t.z, -fy vc / t.z]]
//   S2 = (J R) S3 (J R)^T + 0.3 I; culled unless det > 0
//   conic = (S2yy, -S2xy, S2xx) / det
//   lambda = mid + sqrt(max(0.1, mid^2 - det)); radius = ceil(3 sqrt(lambda))
//   culled unless mean, depth and radius are finite; radius capped at 2^30.
// A culled Gaussian gets the record {0, 0, 0, 0} and the conic {0, 0, 0, 0}.
#pragma once
#include "tdgs_internal.cuh"

namespace tdgs {
namespace proj {

__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float dvd(float a, float b) { return __fdiv_rn(a, b); }
// a*b + c*d, each product rounded, then the sum
__device__ __forceinline__ float dot2(float a, float b, float c, float d) { return add(mul(a, b), mul(c, d)); }
// (a*b + c*d) + e*f
__device__ __forceinline__ float dot3(float a, float b, float c, float d, float e, float f) {
  return add(dot2(a, b, c, d), mul(e, f));
}

// Slope limits of the camera (computed once per thread).
__device__ __forceinline__ float2 slope_limits(const CameraDev& cam) {
  return make_float2(dvd(mul(0.65f, __uint2float_rn(cam.width)), cam.fx),
                     dvd(mul(0.65f, __uint2float_rn(cam.height)), cam.fy));
}

// p: mean + opacity; c0 = (xx, xy, xz, yy), c1 = (yz, zz, -, -).
__device__ __forceinline__ void project(const float4 p, const float4 c0, const float4 c1, const CameraDev& cam,
                                        const float2 lim, float4& out, float4& co) {
  const float* R = cam.rot;
  const float lim_x = lim.x, lim_y = lim.y;
  out = make_float4(0.f, 0.f, 0.f, 0.f);
  co = make_float4(0.f, 0.f, 0.f, 0.f);
  const float tx = add(dot3(R[0], p.x, R[1], p.y, R[2], p.z), cam.trans[0]);
  const float ty = add(dot3(R[3], p.x, R[4], p.y, R[5], p.z), cam.trans[1]);
  const float tz = add(dot3(R[6], p.x, R[7], p.y, R[8], p.z), cam.trans[2]);
  if (tz > cam.near_z) {
    const float u = dvd(tx, tz), v = dvd(ty, tz);
    const float px = add(mul(cam.fx, u), cam.cx);
    const float py = add(mul(cam.fy, v), cam.cy);
    const float uc = fminf(lim_x, fmaxf(-lim_x, u));
    const float vc = fminf(lim_y, fmaxf(-lim_y, v));
    const float j00 = dvd(cam.fx, tz), j02 = -dvd(mul(cam.fx, uc), tz);
    const float j11 = dvd(cam.fy, tz), j12 = -dvd(mul(cam.fy, vc), tz);
    float T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = dot2(j00, R[k], j02, R[6 + k]);
      T1[k] = dot2(j11, R[3 + k], j12, R[6 + k]);
    }
    // S3 rows: (xx, xy, xz), (xy, yy, yz), (xz, yz, zz); c0 = (xx, xy, xz, yy), c1 = (yz, zz, -, -)
    const float S[3][3] = {{c0.x, c0.y, c0.z}, {c0.y, c0.w, c1.x}, {c0.z, c1.x, c1.y}};
    float M0[3], M1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      M0[k] = dot3(T0[0], S[0][k], T0[1], S[1][k], T0[2], S[2][k]);
      M1[k] = dot3(T1[0], S[0][k], T1[1], S[1][k], T1[2], S[2][k]);
    }
    const float a = add(dot3(M0[0], T0[0], M0[1], T0[1], M0[2], T0[2]), 0.3f);
    const float b = dot3(M0[0], T1[0], M0[1], T1[1], M0[2], T1[2]);
    const float d = add(dot3(M1[0], T1[0], M1[1], T1[1], M1[2], T1[2]), 0.3f);
    const float det = sub(mul(a, d), mul(b, b));
    if (det > 0.0f) {
      const float mid = mul(0.5f, add(a, d));
      const float disc = sub(mul(mid, mid), det);
      const float lambda = add(mid, __fsqrt_rn(fmaxf(0.1f, disc)));
      float r = ceilf(mul(3.0f, __fsqrt_rn(lambda)));
      if (isfinite(px) && isfinite(py) && isfinite(tz) && isfinite(r)) {
        r = fminf(r, 1073741824.0f);
        out = make_float4(px, py, tz, __int_as_float(static_cast<int32_t>(r)));
        co = make_float4(dvd(d, det), -dvd(b, det), dvd(a, det), p.w);
      }
    }
  }
}

}  // namespace proj
}  // namespace tdgs
