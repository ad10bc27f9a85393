// CPU oracle for the 3DGS tile depth sort -- TEST INFRASTRUCTURE ONLY.
//
// Only the test suite, the smoke check and the benchmark's CPU-baseline leg
// may load this library.  It shares no code, header or constant with the
// CUDA path: it is the plain, slow definition of each step, written from the
// paper's statement of the pipeline (Sec. II-A "Duplication with Tiles" and
// "Sorting"; Table III lists which buffers feed PrefixSum and
// DuplicateWithTile; Table VI names the stages Scan, Duplicate with tiles,
// Sorting and Identify Range).  Every function runs on one host thread.
//
// Readings where the paper is silent (the exact rectangle rule, validity of
// depths, tile numbering, the key layout, tie order, empty tiles) are stated
// beside the code that applies them.
//
// Status codes (same numbering as the library's public header, restated
// here on purpose so nothing is shared):
//   0 ok, 1 invalid argument, 3 pair-count overflow.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

constexpr int kOk = 0;
constexpr int kInvalid = 1;
constexpr int kOverflow = 3;

struct G2 {       // one projected Gaussian (Table IV, Group 1: xy, depth, radius)
  float x, y, depth;
  int32_t radius;
};
static_assert(sizeof(G2) == 16, "record is 16 bytes");

struct Rect {
  int32_t x0, y0, x1, y1;  // tiles [x0,x1) x [y0,y1)
};

// Tile rectangle of a Gaussian's 3-sigma box (Sec. II-A: the AABB of the
// projected ellipse is intersected with the 16x16 tile grid).  Reading: the
// box is [x - r, x + r] in pixels; the first touched column is
// floor((x - r) / 16) and the end column is floor((x + r + 15) / 16), each
// evaluated in float32 in exactly this order, then clamped to [0, grid].
// Division by 16 is written as multiplication by 1/16, which is exact.
// `volatile` keeps every intermediate a rounded float32 (no contraction,
// no excess precision).
Rect tile_rect(const G2& g, int32_t gx, int32_t gy) {
  volatile float r = static_cast<float>(g.radius);
  volatile float sx0 = g.x - r;
  volatile float sx1 = g.x + r;
  sx1 = sx1 + 15.0f;
  volatile float sy0 = g.y - r;
  volatile float sy1 = g.y + r;
  sy1 = sy1 + 15.0f;
  float fx0 = std::floor(sx0 * 0.0625f);
  float fx1 = std::floor(sx1 * 0.0625f);
  float fy0 = std::floor(sy0 * 0.0625f);
  float fy1 = std::floor(sy1 * 0.0625f);
  auto clampf = [](float v, float hi) { return v < 0.0f ? 0.0f : (v > hi ? hi : v); };
  Rect q;
  q.x0 = static_cast<int32_t>(clampf(fx0, static_cast<float>(gx)));
  q.x1 = static_cast<int32_t>(clampf(fx1, static_cast<float>(gx)));
  q.y0 = static_cast<int32_t>(clampf(fy0, static_cast<float>(gy)));
  q.y1 = static_cast<int32_t>(clampf(fy1, static_cast<float>(gy)));
  return q;
}

bool rect_empty(const Rect& q) { return q.x1 <= q.x0 || q.y1 <= q.y0; }

// Reading of validity: radius <= 0 means culled (no tiles, nothing checked).
// A Gaussian with radius > 0 must have a finite mean; one whose rectangle is
// non-empty must have a finite depth > +0.0, because the key carries the raw
// float bits of the depth and only positive finite floats keep their order
// when compared as unsigned integers.
bool depth_ok(float d) { return std::isfinite(d) && d > 0.0f; }

uint32_t grid_dim(uint32_t px) { return (px + 15u) / 16u; }

uint32_t bits_of(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

}  // namespace

extern "C" {

// Step 1, tile count: counts[i] = number of 16x16 tiles the i-th Gaussian's
// rectangle covers (0 when culled or off-screen).  Returns 1 on an invalid
// Gaussian (its count is written as 0 and the scan continues).
int oracle_count_tiles(const G2* g, uint32_t n, uint32_t width, uint32_t height,
                       uint32_t* counts) {
  if (width == 0 || height == 0) return kInvalid;
  const int32_t gx = static_cast<int32_t>(grid_dim(width));
  const int32_t gy = static_cast<int32_t>(grid_dim(height));
  int status = kOk;
  for (uint32_t i = 0; i < n; ++i) {
    counts[i] = 0;
    if (g[i].radius <= 0) continue;
    if (!std::isfinite(g[i].x) || !std::isfinite(g[i].y)) {
      status = kInvalid;
      continue;
    }
    Rect q = tile_rect(g[i], gx, gy);
    if (rect_empty(q)) continue;
    if (!depth_ok(g[i].depth)) {
      status = kInvalid;
      continue;
    }
    counts[i] = static_cast<uint32_t>(q.x1 - q.x0) * static_cast<uint32_t>(q.y1 - q.y0);
  }
  return status;
}

// Step 2, PrefixSum (Table III): offsets[i] = sum of counts[j] for j < i,
// accumulated in 64 bits; *total = the full sum.  A total above 2^32 - 1
// cannot index uint32 offsets and returns the overflow status.
int oracle_scan(const uint32_t* counts, uint32_t n, uint32_t* offsets, uint64_t* total) {
  uint64_t run = 0;
  for (uint32_t i = 0; i < n; ++i) {
    offsets[i] = static_cast<uint32_t>(run);
    run += counts[i];
  }
  *total = run;
  return run > 0xFFFFFFFFull ? kOverflow : kOk;
}

// Step 3, DuplicateWithTile (Sec. II-A): each Gaussian i writes one pair per
// covered tile, rows (ty) outer and columns (tx) inner, starting at
// offsets[i].  Key = (tile id << 32) | raw bits of the float32 depth, with
// tile id = ty * gx + tx (row-major); value = i.  m is the capacity of keys
// and values; a pair that would land at or beyond it is an invalid argument.
int oracle_duplicate(const G2* g, const uint32_t* offsets, uint32_t n, uint32_t width,
                     uint32_t height, uint64_t* keys, uint32_t* values, uint32_t m) {
  if (width == 0 || height == 0) return kInvalid;
  const int32_t gx = static_cast<int32_t>(grid_dim(width));
  const int32_t gy = static_cast<int32_t>(grid_dim(height));
  for (uint32_t i = 0; i < n; ++i) {
    if (g[i].radius <= 0) continue;
    if (!std::isfinite(g[i].x) || !std::isfinite(g[i].y)) return kInvalid;
    Rect q = tile_rect(g[i], gx, gy);
    if (rect_empty(q)) continue;
    if (!depth_ok(g[i].depth)) return kInvalid;
    uint64_t k = offsets[i];
    const uint64_t dbits = bits_of(g[i].depth);
    for (int32_t ty = q.y0; ty < q.y1; ++ty)
      for (int32_t tx = q.x0; tx < q.x1; ++tx) {
        const uint64_t tile = static_cast<uint64_t>(ty) * static_cast<uint64_t>(gx) +
                              static_cast<uint64_t>(tx);
        if (k >= m) return kInvalid;
        keys[k] = (tile << 32) | dbits;
        values[k] = i;
        ++k;
      }
  }
  return kOk;
}

// Step 4, Sorting (Sec. II-A: by tile, then by depth within the tile): a
// stable ascending sort of the pairs by the whole 64-bit key.  Equal keys
// keep their input order.
int oracle_sort_pairs(uint64_t* keys, uint32_t* values, uint32_t m) {
  std::vector<uint32_t> idx(m);
  for (uint32_t k = 0; k < m; ++k) idx[k] = k;
  std::stable_sort(idx.begin(), idx.end(),
                   [keys](uint32_t a, uint32_t b) { return keys[a] < keys[b]; });
  std::vector<uint64_t> k2(m);
  std::vector<uint32_t> v2(m);
  for (uint32_t k = 0; k < m; ++k) {
    k2[k] = keys[idx[k]];
    v2[k] = values[idx[k]];
  }
  std::copy(k2.begin(), k2.end(), keys);
  std::copy(v2.begin(), v2.end(), values);
  return kOk;
}

// Step 5, Identify Range (Sec. IV-B): ranges[2t], ranges[2t+1] = first and
// one-past-last position of tile t in the sorted list, found by one linear
// pass over the sorted keys.  Reading: a tile with no pairs keeps {0, 0}.
// A key whose tile id is >= num_tiles is an invalid argument.
int oracle_tile_ranges(const uint64_t* sorted_keys, uint32_t m, uint32_t num_tiles,
                       uint32_t* ranges) {
  for (uint32_t t = 0; t < num_tiles; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
  if (m == 0) return kOk;
  uint64_t prev = 0;
  for (uint32_t k = 0; k < m; ++k) {
    const uint64_t t = sorted_keys[k] >> 32;
    if (t >= num_tiles) return kInvalid;
    if (k == 0 || t != prev) {
      ranges[2 * t] = k;
      if (k > 0) ranges[2 * prev + 1] = k;
    }
    prev = t;
  }
  ranges[2 * prev + 1] = m;
  return kOk;
}

// Preprocessing (Sec. II-A "Preprocessing"; inputs Table I, outputs
// Table IV): camera transform of the mean, frustum culling, projection of
// the mean to pixels, projection of the 3D covariance to the 2D footprint
// covariance, its inverse (the conic) and the 3-sigma radius.  The paper
// names the stage, its inputs and its outputs but prints no formulas; the
// reading here is the EWA splatting projection of 3D Gaussian Splatting
// (the pipeline the paper accelerates):
//   t = R p + T                          camera-space mean (R row-major)
//   culled unless t.z > near_z
//   u = t.x / t.z, v = t.y / t.z;  x = fx u + cx,  y = fy v + cy
//   Jacobian of the perspective map at the mean, with the slopes clamped to
//   1.3 times the half field of view (lim_x = 0.65 W / fx, lim_y = 0.65 H / fy):
//     J = [[fx / t.z, 0, -fx uc / t.z], [0, fy / t.z, -fy vc / t.z]]
//   S2 = (J R) S3 (J R)^T + 0.3 I        (0.3: low-pass dilation)
//   culled unless det(S2) > 0
//   conic = (S2_yy, -S2_xy, S2_xx) / det
//   lambda = mid + sqrt(max(0.1, mid^2 - det)),  mid = (S2_xx + S2_yy) / 2
//   radius = ceil(3 sqrt(lambda))        (culled unless x, y, depth and
//                                         radius are finite; radius capped
//                                         at 2^30)
// Precision: float32, every operation rounded in the order written (the
// library computes in float32; the radius is an integer decided by float
// arithmetic, so both sides decide it in the same precision and order).
// The oracle is compiled with -ffp-contract=off (no fused multiply-add).
// A culled Gaussian gets the record {0, 0, 0, 0} and the conic {0, 0, 0, 0}.
struct G3 {  // Table I, Group 1: mean and opacity
  float x, y, z, opacity;
};
struct C3 {  // Table I, Group 2: the six entries of the symmetric 3D covariance, two texels
  float xx, xy, xz, yy, yz, zz, pad0, pad1;
};
struct Cam {
  float rot[9];    // world -> camera rotation, row-major
  float trans[3];  // camera-space translation
  float fx, fy, cx, cy, near_z;
  uint32_t width, height;
};
static_assert(sizeof(C3) == 32, "covariance is two 16-byte texels");
static_assert(sizeof(Cam) == 76, "camera block: 19 four-byte fields");

int oracle_preprocess(const G3* g, const C3* cov, uint32_t n, const Cam* cam, G2* rec,
                      float* conic_opacity) {
  if (!(cam->fx > 0.0f) || !(cam->fy > 0.0f) || cam->width == 0 || cam->height == 0) return kInvalid;
  const float* R = cam->rot;
  const float lim_x = (0.65f * static_cast<float>(cam->width)) / cam->fx;
  const float lim_y = (0.65f * static_cast<float>(cam->height)) / cam->fy;
  for (uint32_t i = 0; i < n; ++i) {
    G2 out = {0.0f, 0.0f, 0.0f, 0};
    float co[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const G3 p = g[i];
    const float tx = ((R[0] * p.x + R[1] * p.y) + R[2] * p.z) + cam->trans[0];
    const float ty = ((R[3] * p.x + R[4] * p.y) + R[5] * p.z) + cam->trans[1];
    const float tz = ((R[6] * p.x + R[7] * p.y) + R[8] * p.z) + cam->trans[2];
    bool keep = tz > cam->near_z;
    if (keep) {
      const float u = tx / tz, v = ty / tz;
      const float px = cam->fx * u + cam->cx;
      const float py = cam->fy * v + cam->cy;
      const float uc = std::fmin(lim_x, std::fmax(-lim_x, u));
      const float vc = std::fmin(lim_y, std::fmax(-lim_y, v));
      const float j00 = cam->fx / tz, j02 = -((cam->fx * uc) / tz);
      const float j11 = cam->fy / tz, j12 = -((cam->fy * vc) / tz);
      float T[2][3];
      for (int k = 0; k < 3; ++k) {
        T[0][k] = j00 * R[k] + j02 * R[6 + k];
        T[1][k] = j11 * R[3 + k] + j12 * R[6 + k];
      }
      const C3& c = cov[i];
      const float S[3][3] = {{c.xx, c.xy, c.xz}, {c.xy, c.yy, c.yz}, {c.xz, c.yz, c.zz}};
      float M[2][3];
      for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) M[r][k] = (T[r][0] * S[0][k] + T[r][1] * S[1][k]) + T[r][2] * S[2][k];
      const float a = ((M[0][0] * T[0][0] + M[0][1] * T[0][1]) + M[0][2] * T[0][2]) + 0.3f;
      const float b = (M[0][0] * T[1][0] + M[0][1] * T[1][1]) + M[0][2] * T[1][2];
      const float d = ((M[1][0] * T[1][0] + M[1][1] * T[1][1]) + M[1][2] * T[1][2]) + 0.3f;
      const float det = a * d - b * b;
      keep = det > 0.0f;
      if (keep) {
        const float mid = 0.5f * (a + d);
        const float disc = mid * mid - det;
        const float lambda = mid + std::sqrt(std::fmax(0.1f, disc));
        float r = std::ceil(3.0f * std::sqrt(lambda));
        keep = std::isfinite(px) && std::isfinite(py) && std::isfinite(tz) && std::isfinite(r);
        if (keep) {
          if (r > 1073741824.0f) r = 1073741824.0f;
          out = {px, py, tz, static_cast<int32_t>(r)};
          co[0] = d / det;
          co[1] = -(b / det);
          co[2] = a / det;
          co[3] = p.opacity;
        }
      }
    }
    rec[i] = out;
    if (conic_opacity)
      for (int k = 0; k < 4; ++k) conic_opacity[4 * static_cast<size_t>(i) + k] = co[k];
  }
  return kOk;
}

// Rendering (Sec. II-A "Rendering": alpha blending of each tile's sorted
// Gaussians per pixel; Sec. IV-C: one 16x16 tile per work group).  The
// paper names the blend without formulas; the reading is the front-to-back
// compositing of 3D Gaussian splatting.  For pixel (px, py) of tile t (the
// sample point is the pixel's integer coordinate), walking the tile's list
// sorted_values[ranges[t].start .. ranges[t].end) in order with
// transmittance T = 1 and colour C = 0:
//   d = (x - px, y - py)                      x, y: the Gaussian's 2D mean
//   power = -0.5 (a dx^2 + c dy^2) - b dx dy   (a, b, c): its conic
//   skip if power > 0
//   alpha = min(0.99, opacity exp(power)); skip if alpha < 1/255
//   T' = T (1 - alpha); stop the pixel if T' < 1e-4 (without this Gaussian)
//   C += rgb alpha T; T = T'
// and the pixel is C + T * background.  Float32 in this order (exp from
// the C library), so the GPU's result differs only through exp's last bits
// and the threshold decisions they can flip.
int oracle_render(const G2* rec, const float* conic_opacity, const float* rgb, const uint32_t* sorted_values,
                  const uint32_t* ranges, uint32_t width, uint32_t height, const float* background,
                  float* image) {
  if (width == 0 || height == 0) return kInvalid;
  const uint32_t gx = grid_dim(width);
  for (uint32_t py = 0; py < height; ++py)
    for (uint32_t px = 0; px < width; ++px) {
      const uint32_t t = (py / 16u) * gx + px / 16u;
      const float fx = static_cast<float>(px), fy = static_cast<float>(py);
      float T = 1.0f, C[3] = {0.0f, 0.0f, 0.0f};
      for (uint32_t k = ranges[2 * t]; k < ranges[2 * t + 1]; ++k) {
        const uint32_t i = sorted_values[k];
        const float* co = conic_opacity + 4 * static_cast<size_t>(i);
        const float dx = rec[i].x - fx, dy = rec[i].y - fy;
        const float power = -0.5f * (co[0] * dx * dx + co[2] * dy * dy) - co[1] * dx * dy;
        if (power > 0.0f) continue;
        const float alpha = std::fmin(0.99f, co[3] * std::exp(power));
        if (alpha < 1.0f / 255.0f) continue;
        const float test_t = T * (1.0f - alpha);
        if (test_t < 0.0001f) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * static_cast<size_t>(i) + ch] * alpha * T;
        T = test_t;
      }
      float* o = image + 3 * (static_cast<size_t>(py) * width + px);
      for (int ch = 0; ch < 3; ++ch) o[ch] = C[ch] + T * background[ch];
    }
  return kOk;
}

// The paper's 32-bit key (Sec. IV-B "key normalization"): 20 bits of tile
// number and the depth normalised to the range 2^10, so that a float-based
// sort can order by tile, then depth.  The figure that fixes the layout is
// not in the text; the reading here:
//   visible Gaussians: those with pairs (count > 0);
//   dmin, dmax: their smallest and largest depth (float32);
//   scale = 1024 / (dmax - dmin) (0 if dmax == dmin);
//   q = min(1023, floor((depth - dmin) * scale))   (float32, in this order)
//   key32 = tile << 10 | q   (bits 30 and 31 clear: the bit pattern of a
//                             positive float, so float and integer order agree)
// requiring tile < 2^20.  Pairs are emitted like oracle_duplicate (same
// order and values) and sorted stably by key32; ranges come from
// key32 >> 10.  Depths closer than 1/1024 of the range collapse to one q
// and then keep index order: the result differs from the exact 64-bit sort
// wherever that happens.
int oracle_sort_frame_normalized(const G2* g, uint32_t n, uint32_t width, uint32_t height, uint32_t* keys,
                                 uint32_t* values, uint32_t m_cap, uint32_t* m_out, uint32_t* ranges) {
  if (width == 0 || height == 0) return kInvalid;
  const int32_t gx = static_cast<int32_t>(grid_dim(width));
  const int32_t gy = static_cast<int32_t>(grid_dim(height));
  if (static_cast<uint64_t>(gx) * static_cast<uint64_t>(gy) > (1ull << 20)) return kInvalid;
  std::vector<uint32_t> counts(n);
  if (oracle_count_tiles(g, n, width, height, counts.data()) != kOk) return kInvalid;
  float dmin = 0.0f, dmax = 0.0f;
  bool any = false;
  uint64_t m = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (!counts[i]) continue;
    m += counts[i];
    if (!any || g[i].depth < dmin) dmin = g[i].depth;
    if (!any || g[i].depth > dmax) dmax = g[i].depth;
    any = true;
  }
  if (m > m_cap) return kInvalid;
  const float scale = dmax > dmin ? 1024.0f / (dmax - dmin) : 0.0f;
  std::vector<uint32_t> k0, v0;
  k0.reserve(m);
  v0.reserve(m);
  for (uint32_t i = 0; i < n; ++i) {
    if (!counts[i]) continue;
    const Rect q = tile_rect(g[i], gx, gy);
    const float f = std::floor((g[i].depth - dmin) * scale);
    const uint32_t qd = f >= 1023.0f ? 1023u : static_cast<uint32_t>(f);
    for (int32_t ty = q.y0; ty < q.y1; ++ty)
      for (int32_t tx = q.x0; tx < q.x1; ++tx) {
        const uint32_t tile = static_cast<uint32_t>(ty) * static_cast<uint32_t>(gx) + static_cast<uint32_t>(tx);
        k0.push_back((tile << 10) | qd);
        v0.push_back(i);
      }
  }
  std::vector<uint32_t> idx(m);
  for (uint32_t k = 0; k < m; ++k) idx[k] = k;
  std::stable_sort(idx.begin(), idx.end(), [&k0](uint32_t a, uint32_t b) { return k0[a] < k0[b]; });
  const uint32_t tiles = static_cast<uint32_t>(gx * gy);
  for (uint32_t t = 0; t < tiles; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
  for (uint32_t k = 0; k < m; ++k) {
    keys[k] = k0[idx[k]];
    values[k] = v0[idx[k]];
    const uint32_t t = keys[k] >> 10;
    if (k == 0 || (keys[k - 1] >> 10) != t) ranges[2 * t] = k;
    ranges[2 * t + 1] = k + 1;
  }
  *m_out = static_cast<uint32_t>(m);
  return kOk;
}

// Number of tiles and tile bits of an image (helpers for callers).
uint32_t oracle_num_tiles(uint32_t width, uint32_t height) {
  return grid_dim(width) * grid_dim(height);
}

}  // extern "C"
