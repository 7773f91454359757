// Bloom (Sec. 5.3): bright map, image pyramid, blur of every level from the second one upwards,
// the blurred levels added onto the image (then, optionally, the tone map of Sec. 5.4).
//   k_bloom_pyramid    levels 1 .. L-1 in one launch: a block reads a 64x64-pixel footprint,
//                      applies the bright test and averages 2x2 pixels into its 32x32 level-1
//                      tile, then halves the tile in shared memory level by level.  A level's
//                      clamp to the edge never reaches outside the block, because tiles are
//                      aligned to powers of two.  The full-resolution bright map is never stored.
//   k_bloom_blur       every level in one launch: a 32x16 texel tile plus an R-texel halo in shared
//                      memory, rows then columns of the separable Gaussian
//   k_bloom_composite  one 2x2 pixel quad per thread: X + s * sum_k bilinear(level k at the pixel
//                      centre), HDR store and / or the fused tone map.  On level 1 the quad's four
//                      bilinear footprints lie in a 3x3 texel block; on level k >= 2 both pixels of
//                      a row (or column) pair fall in the same texel cell, so the quad loads 2x2
//                      texels per level.  Each pixel's arithmetic is the per-pixel bilinear.
#include <string.h>

#include <cmath>

#include "shade_core.cuh"

namespace epbr {

constexpr int kBloomMaxLevels = 6, kBloomMaxR = 8;
constexpr int kBloomTX = 32, kBloomTY = 8;       // threads per block: 32 x 8
constexpr int kBlurTW = 32, kBlurTH = 16;         // blur output tile

struct BloomLevel {
  float4* pyr;  // before the blur
  float4* blr;  // after the blur
  int W, H;
};

struct BloomDev {
  BloomLevel lev[kBloomMaxLevels];  // levels 1 .. L-1
  int L, R;
  float w[2 * kBloomMaxR + 1];        // normalised Gaussian weights, w[R + d]
  int tile_start[kBloomMaxLevels + 1];  // first blur block of level k (k = 1 .. L-1), end at [L]
  int tiles_x[kBloomMaxLevels];
};

// The bright-map test: Rec. 709 luminance in FP32, each product and sum rounded on its own.
__device__ __forceinline__ bool bloom_bright(float3 c, float threshold) {
  float lum = __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, c.x), __fmul_rn(0.7152f, c.y)), __fmul_rn(0.0722f, c.z));
  return lum > threshold;
}

template <int HF>
__global__ void __launch_bounds__(kBloomTX* kBloomTY)
    k_bloom_pyramid(const void* __restrict__ hdr, long long pitch, int W, int H, float threshold, BloomDev d) {
  __shared__ float4 s_a[32 * 32];  // levels 1, 3, 5 of the block's tile
  __shared__ float4 s_b[16 * 16];  // levels 2, 4
  const int tid = threadIdx.y * kBloomTX + threadIdx.x;
  {
    const BloomLevel& l1 = d.lev[1];
    // two level-1 rows per batch: their eight HDR loads (coordinates clamped into the image, so
    // every load is valid) are issued together, then reduced in the per-texel order
#pragma unroll
    for (int r0 = 0; r0 < 4; r0 += 2) {
      float3 c[2][4];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 32 + threadIdx.y + 8 * (r0 + q);
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int a = 0; a < 2; ++a) c[q][2 * b + a] = load_hdr<HF>(hdr, pitch, min(2 * i + a, W - 1), min(2 * j + b, H - 1));
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        int li = threadIdx.x, lj = threadIdx.y + 8 * (r0 + q);
        int i = blockIdx.x * 32 + li, j = blockIdx.y * 32 + lj;
        float3 sum = f3(0, 0, 0);
        if (i < l1.W && j < l1.H) {
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (bloom_bright(c[q][t], threshold)) sum = sum + c[q][t];
          sum = 0.25f * sum;
          l1.pyr[(size_t)j * l1.W + i] = make_float4(sum.x, sum.y, sum.z, 0.0f);
        }
        s_a[lj * 32 + li] = make_float4(sum.x, sum.y, sum.z, 0.0f);
      }
    }
  }
#pragma unroll
  for (int k = 2; k < kBloomMaxLevels; ++k) {
    if (k >= d.L) break;
    __syncthreads();  // level k-1 of the tile is in shared memory
    const float4* src = (k & 1) ? s_b : s_a;
    float4* dst = (k & 1) ? s_a : s_b;
    const int side = 32 >> (k - 1), sside = 2 * side;  // tile side of level k and of level k-1
    const BloomLevel& ls = d.lev[k - 1];
    const BloomLevel& lv = d.lev[k];
    if (tid < side * side) {
      int li = tid % side, lj = tid / side;
      int i = blockIdx.x * side + li, j = blockIdx.y * side + lj;
      float3 sum = f3(0, 0, 0);
      if (i < lv.W && j < lv.H) {
        // source texels clamped to level k-1's edge, as local indices of the block's tile
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            int si = min(2 * i + a, ls.W - 1) - blockIdx.x * sside, sj = min(2 * j + b, ls.H - 1) - blockIdx.y * sside;
            sum = sum + xyz(src[sj * sside + si]);
          }
        sum = 0.25f * sum;
        lv.pyr[(size_t)j * lv.W + i] = make_float4(sum.x, sum.y, sum.z, 0.0f);
      }
      dst[lj * side + li] = make_float4(sum.x, sum.y, sum.z, 0.0f);
    }
  }
}

__global__ void __launch_bounds__(kBloomTX* kBloomTY) k_bloom_blur(BloomDev d) {
  constexpr int TW = kBlurTW + 2 * kBloomMaxR, TH = kBlurTH + 2 * kBloomMaxR;
  __shared__ float4 s_in[TH][TW];
  __shared__ float4 s_row[TH][kBlurTW];
  __shared__ float s_w[2 * kBloomMaxR + 1];
  const int tid = threadIdx.y * kBloomTX + threadIdx.x;
  const int R = d.R;
  if (tid <= 2 * R) s_w[tid] = d.w[tid];
  int b = blockIdx.x, k = 1;
#pragma unroll
  for (int q = 2; q < kBloomMaxLevels; ++q)
    if (q < d.L && b >= d.tile_start[q]) k = q;
  BloomLevel lv = d.lev[1];
  int tiles_x = d.tiles_x[1];
#pragma unroll
  for (int q = 2; q < kBloomMaxLevels; ++q)
    if (q == k) lv = d.lev[q], tiles_x = d.tiles_x[q];
  b -= d.tile_start[k];
  const int by = b / tiles_x;
  const int x0 = (b - by * tiles_x) * kBlurTW, y0 = by * kBlurTH;
  const int tw = kBlurTW + 2 * R, th = kBlurTH + 2 * R;
  for (int ty = threadIdx.y; ty < th; ty += kBloomTY) {
    const float4* row = lv.pyr + (size_t)min(max(y0 - R + ty, 0), lv.H - 1) * lv.W;
    for (int tx = threadIdx.x; tx < tw; tx += kBloomTX) s_in[ty][tx] = __ldg(row + min(max(x0 - R + tx, 0), lv.W - 1));
  }
  __syncthreads();
  for (int ty = threadIdx.y; ty < th; ty += kBloomTY) {
    float3 sum = f3(0, 0, 0);
#pragma unroll
    for (int t = 0; t <= 2 * kBloomMaxR; ++t) {
      if (t > 2 * R) break;
      sum = sum + s_w[t] * xyz(s_in[ty][threadIdx.x + t]);
    }
    s_row[ty][threadIdx.x] = make_float4(sum.x, sum.y, sum.z, 0.0f);
  }
  __syncthreads();
  const int x = x0 + threadIdx.x;
#pragma unroll
  for (int r = 0; r < kBlurTH / kBloomTY; ++r) {
    const int ly = threadIdx.y + r * kBloomTY, y = y0 + ly;
    if (x >= lv.W || y >= lv.H) continue;
    float3 sum = f3(0, 0, 0);
#pragma unroll
    for (int t = 0; t <= 2 * kBloomMaxR; ++t) {
      if (t > 2 * R) break;
      sum = sum + s_w[t] * xyz(s_row[ly + t][threadIdx.x]);
    }
    lv.blr[(size_t)y * lv.W + x] = make_float4(sum.x, sum.y, sum.z, 0.0f);
  }
}

__device__ __forceinline__ float3 lerp3(float3 a, float3 b, float t) { return a + t * (b - a); }

// The bilinear value at fractions (fx, fy) of the texel cell with corners a (top left), b (top
// right), p (bottom left), q (bottom right).
__device__ __forceinline__ float3 bilerp(float3 a, float3 b, float3 p, float3 q, float fx, float fy) {
  float3 top = lerp3(a, b, fx), bot = lerp3(p, q, fx);
  return lerp3(top, bot, fy);
}

// Adds s * sum_k (level k sampled bilinearly at the pixel centre) to the quad's four pixels
// c[b][a] = pixel (2 qi + a, 2 qj + b).  Pixel x lies at texel coordinate u = (x + 1/2) 2^-k - 1/2
// of level k, exact in FP32 for the admitted sizes.
__device__ __forceinline__ void bloom_add_quad(const BloomDev& d, float strength, int qi, int qj, float3 (&c)[2][2]) {
  float3 add[2][2] = {{f3(0, 0, 0), f3(0, 0, 0)}, {f3(0, 0, 0), f3(0, 0, 0)}};
  {
    // level 1: pixel 2 qi sits at u = qi - 1/4 (cell qi-1, fraction 3/4), pixel 2 qi + 1 at
    // qi + 1/4 (cell qi, fraction 1/4): the footprints span texels qi-1 .. qi+1
    const BloomLevel& lv = d.lev[1];
    int ci[3], cj[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      ci[t] = min(max(qi - 1 + t, 0), lv.W - 1);
      cj[t] = min(max(qj - 1 + t, 0), lv.H - 1);
    }
    float3 T[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float4* row = lv.blr + (size_t)cj[r] * lv.W;
#pragma unroll
      for (int t = 0; t < 3; ++t) T[r][t] = xyz(__ldg(row + ci[t]));
    }
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a)
        add[b][a] = add[b][a] + bilerp(T[b][a], T[b][a + 1], T[b + 1][a], T[b + 1][a + 1], a ? 0.25f : 0.75f,
                                       b ? 0.25f : 0.75f);
  }
#pragma unroll
  for (int k = 2; k < kBloomMaxLevels; ++k) {
    if (k >= d.L) break;
    // both pixels of a pair share floor(u) on this level (the pair's coordinates differ by
    // 2^(1-k) <= 1/2 and no integer lies between them), so the quad reads one texel cell
    const BloomLevel& lv = d.lev[k];
    const float sc = __int_as_float((127 - k) << 23);  // 2^-k
    float u[2], v[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      u[a] = fmaf((float)(2 * qi + a) + 0.5f, sc, -0.5f);
      v[a] = fmaf((float)(2 * qj + a) + 0.5f, sc, -0.5f);
    }
    const float fu = floorf(u[0]), fv = floorf(v[0]);
    const int iu = (int)fu, iv = (int)fv;
    const int i0 = min(max(iu, 0), lv.W - 1), i1 = min(max(iu + 1, 0), lv.W - 1);
    const int j0 = min(max(iv, 0), lv.H - 1), j1 = min(max(iv + 1, 0), lv.H - 1);
    const float4* r0 = lv.blr + (size_t)j0 * lv.W;
    const float4* r1 = lv.blr + (size_t)j1 * lv.W;
    float3 A = xyz(__ldg(r0 + i0)), B = xyz(__ldg(r0 + i1)), P = xyz(__ldg(r1 + i0)), Q = xyz(__ldg(r1 + i1));
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) add[b][a] = add[b][a] + bilerp(A, B, P, Q, u[a] - fu, v[b] - fv);
  }
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int a = 0; a < 2; ++a) c[b][a] = c[b][a] + strength * add[b][a];
}

template <int HF, int OF, bool LDR>
__global__ void __launch_bounds__(kBloomTX* kBloomTY)
    k_bloom_composite(const void* __restrict__ hdr, long long pitch, int W, int H, BloomDev d, float strength,
                      void* out, long long out_pitch, float exposure, int op, uint8_t* ldr, long long ldr_pitch) {
  const int qi = blockIdx.x * kBloomTX + threadIdx.x, qj = blockIdx.y * kBloomTY + threadIdx.y;
  if (2 * qi >= W || 2 * qj >= H) return;
  float3 c[2][2];
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int a = 0; a < 2; ++a) c[b][a] = load_hdr<HF>(hdr, pitch, min(2 * qi + a, W - 1), min(2 * qj + b, H - 1));
  bloom_add_quad(d, strength, qi, qj, c);
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      int x = 2 * qi + a, y = 2 * qj + b;
      if (x >= W || y >= H) continue;
      if (out) store_hdr<OF>(out, out_pitch, x, y, c[b][a]);
      if (LDR) ((unsigned*)(ldr + (size_t)y * ldr_pitch))[x] = pack_rgba8(c[b][a], exposure, op);
    }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static epbr_status bloom_layout(int W, int H, const epbr_bloom_params* p, char* base, BloomDev* d, size_t* bytes) {
  if (!p) return fail(EPBR_ERR_INVALID_ARG, "bloom params is NULL");
  if (W < 1 || H < 1 || W > (1 << 15) || H > (1 << 15))
    return fail(EPBR_ERR_INVALID_ARG, "bloom image %dx%d outside [1, 32768]", W, H);
  if (p->levels < 2 || p->levels > kBloomMaxLevels || p->radius < 0 || p->radius > kBloomMaxR ||
      !(p->sigma > 0.0f) || !std::isfinite(p->sigma) || !std::isfinite(p->threshold) || !(p->strength >= 0.0f) ||
      !std::isfinite(p->strength))
    return fail(EPBR_ERR_INVALID_ARG, "bloom params: levels 2..%d, radius 0..%d, sigma > 0, finite threshold, "
                "strength >= 0 required", kBloomMaxLevels, kBloomMaxR);
  size_t off = 0;
  int w = W, h = H;
  for (int k = 1; k < p->levels; ++k) {
    w = (w + 1) / 2;
    h = (h + 1) / 2;
    size_t n = (size_t)w * h * sizeof(float4);
    if (d) {
      d->lev[k] = BloomLevel{(float4*)(base + off), (float4*)(base + off + align256(n)), w, h};
    }
    off += 2 * align256(n);
  }
  *bytes = off;
  return EPBR_OK;
}

}  // namespace epbr

using namespace epbr;

extern "C" epbr_status epbr_bloom_workspace_size(int32_t width, int32_t height, const epbr_bloom_params* params,
                                                 size_t* bytes) {
  if (!bytes) return fail(EPBR_ERR_INVALID_ARG, "bytes is NULL");
  epbr_status st = bloom_layout(width, height, params, nullptr, nullptr, bytes);
  return st ? st : ok();
}

template <int HF, int OF>
static void launch_composite(dim3 g, dim3 b, cudaStream_t s, const void* hdr, long long hp, int W, int H,
                             const BloomDev& d, float strength, void* out, long long op_, float exposure, int op,
                             uint8_t* ldr, long long lp) {
  if (ldr)
    k_bloom_composite<HF, OF, true><<<g, b, 0, s>>>(hdr, hp, W, H, d, strength, out, op_, exposure, op, ldr, lp);
  else
    k_bloom_composite<HF, OF, false><<<g, b, 0, s>>>(hdr, hp, W, H, d, strength, out, op_, exposure, op, ldr, lp);
}

extern "C" epbr_status epbr_bloom(const void* hdr, int32_t hdr_format, int64_t hdr_pitch, int32_t width,
                                  int32_t height, const epbr_bloom_params* params, void* workspace,
                                  size_t workspace_bytes, void* out_hdr, int32_t out_format, int64_t out_pitch,
                                  const epbr_tonemap_params* tonemap, uint8_t* ldr, int64_t ldr_pitch,
                                  void* stream) {
  BloomDev d;
  memset(&d, 0, sizeof(d));
  size_t need = 0;
  epbr_status st = bloom_layout(width, height, params, (char*)workspace, &d, &need);
  if (st) return st;
  if (!hdr) return fail(EPBR_ERR_INVALID_ARG, "bloom: hdr is NULL");
  if (hdr_format != EPBR_HDR_RGBA32F && hdr_format != EPBR_HDR_RGBA16F)
    return fail(EPBR_ERR_INVALID_ARG, "bloom: hdr_format %d unknown", hdr_format);
  int bpp = hdr_format == EPBR_HDR_RGBA32F ? 16 : 8;
  if ((uintptr_t)hdr % bpp || hdr_pitch < (int64_t)bpp * width || hdr_pitch % bpp)
    return fail(EPBR_ERR_INVALID_ARG, "bloom: hdr misaligned or pitch too small");
  if (!workspace || (uintptr_t)workspace % 16 || workspace_bytes < need)
    return fail(EPBR_ERR_INVALID_ARG, "bloom: workspace NULL, misaligned or below %zu bytes", need);
  if (!out_hdr && !ldr) return fail(EPBR_ERR_INVALID_ARG, "bloom: no output");
  if (out_hdr) {
    if (out_format != EPBR_HDR_RGBA32F && out_format != EPBR_HDR_RGBA16F)
      return fail(EPBR_ERR_INVALID_ARG, "bloom: out_format %d unknown", out_format);
    int ob = out_format == EPBR_HDR_RGBA32F ? 16 : 8;
    if ((uintptr_t)out_hdr % ob || out_pitch < (int64_t)ob * width || out_pitch % ob)
      return fail(EPBR_ERR_INVALID_ARG, "bloom: out_hdr misaligned or pitch too small");
    if (out_hdr == hdr && (out_format != hdr_format || out_pitch != hdr_pitch))
      return fail(EPBR_ERR_INVALID_ARG, "bloom: in place needs the same format and pitch");
  }
  if (ldr) {
    if ((uintptr_t)ldr % 4 || ldr_pitch < (int64_t)4 * width || ldr_pitch % 4)
      return fail(EPBR_ERR_INVALID_ARG, "bloom: ldr misaligned or pitch too small");
    if (!tonemap || !(tonemap->exposure >= 0.0f) ||
        (tonemap->op != EPBR_TONEMAP_ACES && tonemap->op != EPBR_TONEMAP_REINHARD))
      return fail(EPBR_ERR_INVALID_ARG, "bloom: tonemap params invalid");
  }
  const int L = params->levels, R = params->radius;
  d.L = L;
  d.R = R;
  double wsum = 0.0, wd[2 * kBloomMaxR + 1];
  for (int t = -R; t <= R; ++t) wsum += (wd[t + R] = std::exp(-(double)(t * t) / (2.0 * params->sigma * params->sigma)));
  for (int t = 0; t <= 2 * R; ++t) d.w[t] = (float)(wd[t] / wsum);
  int tiles = 0;
  for (int k = 1; k < L; ++k) {
    d.tile_start[k] = tiles;
    d.tiles_x[k] = (d.lev[k].W + kBlurTW - 1) / kBlurTW;
    tiles += d.tiles_x[k] * ((d.lev[k].H + kBlurTH - 1) / kBlurTH);
  }
  d.tile_start[L] = tiles;
  cudaStream_t s = (cudaStream_t)stream;
  dim3 blk(kBloomTX, kBloomTY);
  auto grid_of = [](int w, int h) { return dim3((w + kBloomTX - 1) / kBloomTX, (h + kBloomTY - 1) / kBloomTY); };
  // pyramid blocks: one per 32x32 tile of level 1 (64x64 pixels)
  dim3 gp((d.lev[1].W + 31) / 32, (d.lev[1].H + 31) / 32);
  if (hdr_format == EPBR_HDR_RGBA32F)
    k_bloom_pyramid<EPBR_HDR_RGBA32F><<<gp, blk, 0, s>>>(hdr, hdr_pitch, width, height, params->threshold, d);
  else
    k_bloom_pyramid<EPBR_HDR_RGBA16F><<<gp, blk, 0, s>>>(hdr, hdr_pitch, width, height, params->threshold, d);
  k_bloom_blur<<<tiles, blk, 0, s>>>(d);
  float exposure = tonemap ? tonemap->exposure : 1.0f;
  int op = tonemap ? tonemap->op : 0;
  dim3 g = grid_of((width + 1) / 2, (height + 1) / 2);  // one thread per 2x2 pixel quad
  bool in32 = hdr_format == EPBR_HDR_RGBA32F, out32 = !out_hdr || out_format == EPBR_HDR_RGBA32F;
  if (in32 && out32)
    launch_composite<EPBR_HDR_RGBA32F, EPBR_HDR_RGBA32F>(g, blk, s, hdr, hdr_pitch, width, height, d, params->strength,
                                                         out_hdr, out_pitch, exposure, op, ldr, ldr_pitch);
  else if (in32)
    launch_composite<EPBR_HDR_RGBA32F, EPBR_HDR_RGBA16F>(g, blk, s, hdr, hdr_pitch, width, height, d, params->strength,
                                                         out_hdr, out_pitch, exposure, op, ldr, ldr_pitch);
  else if (out32)
    launch_composite<EPBR_HDR_RGBA16F, EPBR_HDR_RGBA32F>(g, blk, s, hdr, hdr_pitch, width, height, d, params->strength,
                                                         out_hdr, out_pitch, exposure, op, ldr, ldr_pitch);
  else
    launch_composite<EPBR_HDR_RGBA16F, EPBR_HDR_RGBA16F>(g, blk, s, hdr, hdr_pitch, width, height, d, params->strength,
                                                         out_hdr, out_pitch, exposure, op, ldr, ldr_pitch);
  if ((st = check_launch("bloom"))) return st;
  return ok();
}
