// Bloom (Sec. 5.3): bright map, image pyramid, blur of every level from the second one upwards,
// the blurred levels added onto the image (then, optionally, the tone map of Sec. 5.4).
//   k_bloom_bright_down  level 1 straight from the HDR image: each thread applies the bright test
//                        to its 2x2 pixels and averages them (the full-resolution bright map,
//                        level 0, is never stored)
//   k_bloom_down         level k from level k-1, 2x2 box average, clamped to the edge
//   k_bloom_blur         every level 1 .. L-1 in one launch: a 32x8 texel tile plus an R-texel halo
//                        in shared memory, rows then columns of the separable Gaussian
//   k_bloom_composite    per pixel: X + s * sum_k bilinear(level k at the pixel centre), HDR store
//                        and / or the fused tone map
#include <string.h>

#include <cmath>

#include "shade_core.cuh"

namespace epbr {

constexpr int kBloomMaxLevels = 6, kBloomMaxR = 8;
constexpr int kBloomTX = 32, kBloomTY = 8;

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
    k_bloom_bright_down(const void* __restrict__ hdr, long long pitch, int W, int H, float threshold,
                        float4* __restrict__ p1, int W1, int H1) {
  int i = blockIdx.x * kBloomTX + threadIdx.x, j = blockIdx.y * kBloomTY + threadIdx.y;
  if (i >= W1 || j >= H1) return;
  float3 sum = f3(0, 0, 0);
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      float3 c = load_hdr<HF>(hdr, pitch, min(2 * i + a, W - 1), min(2 * j + b, H - 1));
      if (bloom_bright(c, threshold)) sum = sum + c;
    }
  p1[(size_t)j * W1 + i] = make_float4(0.25f * sum.x, 0.25f * sum.y, 0.25f * sum.z, 0.0f);
}

__global__ void __launch_bounds__(kBloomTX* kBloomTY)
    k_bloom_down(const float4* __restrict__ src, int Ws, int Hs, float4* __restrict__ dst, int Wd, int Hd) {
  int i = blockIdx.x * kBloomTX + threadIdx.x, j = blockIdx.y * kBloomTY + threadIdx.y;
  if (i >= Wd || j >= Hd) return;
  float3 sum = f3(0, 0, 0);
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int a = 0; a < 2; ++a) sum = sum + xyz(__ldg(src + (size_t)min(2 * j + b, Hs - 1) * Ws + min(2 * i + a, Ws - 1)));
  dst[(size_t)j * Wd + i] = make_float4(0.25f * sum.x, 0.25f * sum.y, 0.25f * sum.z, 0.0f);
}

__global__ void __launch_bounds__(kBloomTX* kBloomTY) k_bloom_blur(BloomDev d) {
  constexpr int TW = kBloomTX + 2 * kBloomMaxR, TH = kBloomTY + 2 * kBloomMaxR;
  __shared__ float4 s_in[TH][TW];
  __shared__ float4 s_row[TH][kBloomTX];
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
  const int x0 = (b % tiles_x) * kBloomTX, y0 = (b / tiles_x) * kBloomTY;
  const int tw = kBloomTX + 2 * R, th = kBloomTY + 2 * R;
  for (int q = tid; q < tw * th; q += kBloomTX * kBloomTY) {
    int ty = q / tw, tx = q - ty * tw;
    int x = min(max(x0 - R + tx, 0), lv.W - 1), y = min(max(y0 - R + ty, 0), lv.H - 1);
    s_in[ty][tx] = __ldg(lv.pyr + (size_t)y * lv.W + x);
  }
  __syncthreads();
  for (int q = tid; q < th * kBloomTX; q += kBloomTX * kBloomTY) {
    int ty = q / kBloomTX, tx = q - ty * kBloomTX;
    float3 sum = f3(0, 0, 0);
    for (int t = 0; t <= 2 * R; ++t) sum = sum + s_w[t] * xyz(s_in[ty][tx + t]);
    s_row[ty][tx] = make_float4(sum.x, sum.y, sum.z, 0.0f);
  }
  __syncthreads();
  int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  if (x >= lv.W || y >= lv.H) return;
  float3 sum = f3(0, 0, 0);
  for (int t = 0; t <= 2 * R; ++t) sum = sum + s_w[t] * xyz(s_row[threadIdx.y + t][threadIdx.x]);
  lv.blr[(size_t)y * lv.W + x] = make_float4(sum.x, sum.y, sum.z, 0.0f);
}

// Level k sampled bilinearly at the centre of pixel (x, y): texel coordinate (x + 1/2) 2^-k - 1/2,
// exact in FP32 for the admitted image sizes.
__device__ __forceinline__ float3 bloom_sample(const BloomLevel& lv, int k, int x, int y) {
  float s = __int_as_float((127 - k) << 23);  // 2^-k
  float u = fmaf((float)x + 0.5f, s, -0.5f), v = fmaf((float)y + 0.5f, s, -0.5f);
  float fu = floorf(u), fv = floorf(v);
  float fx = u - fu, fy = v - fv;
  int iu = (int)fu, iv = (int)fv;
  int i0 = min(max(iu, 0), lv.W - 1), i1 = min(max(iu + 1, 0), lv.W - 1);
  int j0 = min(max(iv, 0), lv.H - 1), j1 = min(max(iv + 1, 0), lv.H - 1);
  const float4* r0 = lv.blr + (size_t)j0 * lv.W;
  const float4* r1 = lv.blr + (size_t)j1 * lv.W;
  float3 a = xyz(__ldg(r0 + i0)), b = xyz(__ldg(r0 + i1)), p = xyz(__ldg(r1 + i0)), q = xyz(__ldg(r1 + i1));
  float3 top = a + fx * (b - a), bot = p + fx * (q - p);
  return top + fy * (bot - top);
}

template <int HF, int OF, bool LDR>
__global__ void __launch_bounds__(kBloomTX* kBloomTY)
    k_bloom_composite(const void* __restrict__ hdr, long long pitch, int W, int H, BloomDev d, float strength,
                      void* out, long long out_pitch, float exposure, int op, uint8_t* ldr, long long ldr_pitch) {
  int x = blockIdx.x * kBloomTX + threadIdx.x, y = blockIdx.y * kBloomTY + threadIdx.y;
  if (x >= W || y >= H) return;
  float3 X = load_hdr<HF>(hdr, pitch, x, y);
  float3 add = f3(0, 0, 0);
#pragma unroll
  for (int k = 1; k < kBloomMaxLevels; ++k)
    if (k < d.L) add = add + bloom_sample(d.lev[k], k, x, y);
  float3 Y = X + strength * add;
  if (out) store_hdr<OF>(out, out_pitch, x, y, Y);
  if (LDR) ((unsigned*)(ldr + (size_t)y * ldr_pitch))[x] = pack_rgba8(Y, exposure, op);
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
    d.tiles_x[k] = (d.lev[k].W + kBloomTX - 1) / kBloomTX;
    tiles += d.tiles_x[k] * ((d.lev[k].H + kBloomTY - 1) / kBloomTY);
  }
  d.tile_start[L] = tiles;
  cudaStream_t s = (cudaStream_t)stream;
  dim3 blk(kBloomTX, kBloomTY);
  auto grid_of = [](int w, int h) { return dim3((w + kBloomTX - 1) / kBloomTX, (h + kBloomTY - 1) / kBloomTY); };
  const BloomLevel& l1 = d.lev[1];
  if (hdr_format == EPBR_HDR_RGBA32F)
    k_bloom_bright_down<EPBR_HDR_RGBA32F><<<grid_of(l1.W, l1.H), blk, 0, s>>>(hdr, hdr_pitch, width, height,
                                                                              params->threshold, l1.pyr, l1.W, l1.H);
  else
    k_bloom_bright_down<EPBR_HDR_RGBA16F><<<grid_of(l1.W, l1.H), blk, 0, s>>>(hdr, hdr_pitch, width, height,
                                                                              params->threshold, l1.pyr, l1.W, l1.H);
  for (int k = 2; k < L; ++k)
    k_bloom_down<<<grid_of(d.lev[k].W, d.lev[k].H), blk, 0, s>>>(d.lev[k - 1].pyr, d.lev[k - 1].W, d.lev[k - 1].H,
                                                                 d.lev[k].pyr, d.lev[k].W, d.lev[k].H);
  k_bloom_blur<<<tiles, blk, 0, s>>>(d);
  float exposure = tonemap ? tonemap->exposure : 1.0f;
  int op = tonemap ? tonemap->op : 0;
  dim3 g = grid_of(width, height);
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
