// Launchers of the heaviest-first rendering path (render.cu; Sec. IV-C).
// The raster-order launcher, launch_render, is declared with the other
// kernels' launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tdgs {

// order[0 .. tiles): every tile index once, tiles with more Gaussians
// (ranges[t].end - ranges[t].start, in 64 buckets) first.  One block.
cudaError_t launch_render_order(const uint2* ranges, uint32_t tiles, uint32_t* order, cudaStream_t s);

// Rendering with block b on tile order[b] (order from launch_render_order,
// device, one entry per tile); the other arguments as launch_render.
cudaError_t launch_render_ordered(const float4* rec, const float4* conic, const float* rgb, const uint32_t* values,
                                  const uint2* ranges, const uint32_t* order, uint32_t width, uint32_t height,
                                  const float* bg, uint32_t n, float* image, uint32_t* err, cudaStream_t s);

// Rendering blocks resident on `device` at once (one wave); 0 if the
// query fails.
uint32_t render_wave_blocks(int device);

}  // namespace tdgs
