// Eye-dome lighting for point clouds (Sec. 4.2; Boucheny 2009): shading from the depth map alone.
//   k_edl  32x16 pixels per block (two rows per thread); the block's log2 depths plus an r-pixel halo are staged in
//          shared memory (one logarithm per texel; +inf for background and off-image texels, so
//          their max(0, .) terms vanish), then each pixel sums its N neighbours' log-depth drops,
//          shades its colour by exp(-A w), optionally times AO, and stores HDR and / or the
//          tone-mapped 8-bit image.
#include <string.h>

#include <cmath>

#include "shade_core.cuh"

namespace epbr {

constexpr int kEdlBX = 32, kEdlBY = 8, kEdlTileH = 2 * kEdlBY, kEdlMaxR = 8, kEdlMaxN = 16;

struct EdlDev {
  float minus_a_log2e;  // -A / ln 2: exp(-A w) = 2^(minus_a_log2e w)
  float inv_n;
  int R, N;
  signed char dx[kEdlMaxN], dy[kEdlMaxN];
  const float* ao;
  long long ao_pitch;
  float ao_inv;  // 1 / ao_scale
};

template <int FMT>
__device__ __forceinline__ float3 edl_colour(const GbufDev& g, int x, int y) {
  if (FMT == EPBR_GBUFFER_FP32) return xyz(__ldg((const float4*)(g.rt[0] + (size_t)y * g.pitch[0]) + x));
  unsigned a = __ldg((const unsigned*)(g.rt[0] + (size_t)y * g.pitch[0]) + x);
  return f3(c_srgb8[a & 255u], c_srgb8[(a >> 8) & 255u], c_srgb8[(a >> 16) & 255u]);
}

template <int FMT, int HDR, bool LDR, int NT>
__global__ void __launch_bounds__(kEdlBX* kEdlBY)
    k_edl(GbufDev g, EdlDev p, void* hdr, long long hdr_pitch, float exposure, int op, uint8_t* ldr,
          long long ldr_pitch) {
  constexpr int TW = kEdlBX + 2 * kEdlMaxR, TH = kEdlTileH + 2 * kEdlMaxR;
  __shared__ float s_l[TH * TW];
  __shared__ int s_off[kEdlMaxN];  // neighbour k as an offset into the flat tile
  const int R = p.R, tw = kEdlBX + 2 * R, th = kEdlTileH + 2 * R;
  const int N = NT > 0 ? NT : p.N;  // NT > 0: the direction count fixed at compile time
  {
    const int tid = threadIdx.y * kEdlBX + threadIdx.x;
    if (tid < N) {
      int dx = 0, dy = 0;
#pragma unroll
      for (int k = 0; k < kEdlMaxN; ++k)
        if (k == tid) dx = p.dx[k], dy = p.dy[k];
      s_off[tid] = dy * TW + dx;
    }
  }
  const int x0 = blockIdx.x * kEdlBX, y0 = blockIdx.y * kEdlTileH;
  const float inf = __int_as_float(0x7f800000);
  for (int ty = threadIdx.y; ty < th; ty += kEdlBY)
    for (int tx = threadIdx.x; tx < tw; tx += kEdlBX) {
      int x = x0 - R + tx, y = y0 - R + ty;
      float l = inf;
      if (x >= 0 && y >= 0 && x < g.W && y < g.H) {
        float e = gb_depth(g, x, y);
        if (is_surface(e)) l = lg2_ftz(e);
      }
      s_l[ty * TW + tx] = l;
    }
  __syncthreads();
  int off[NT > 0 ? NT : 1];
  if (NT > 0) {
#pragma unroll
    for (int k = 0; k < (NT > 0 ? NT : 1); ++k) off[k] = s_off[k];
  }
  const int x = x0 + threadIdx.x;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int ly = threadIdx.y + h * kEdlBY, y = y0 + ly;
    if (x >= g.W || y >= g.H) continue;
    const int centre = (ly + R) * TW + threadIdx.x + R;
    const float lp = s_l[centre];
    float3 c = f3(0, 0, 0);
    if (lp != inf) {
      float w = 0.0f;
      if (NT > 0) {
#pragma unroll
        for (int k = 0; k < (NT > 0 ? NT : 1); ++k) w += fmaxf(lp - s_l[centre + off[k]], 0.0f);
      } else {
        for (int k = 0; k < N; ++k) w += fmaxf(lp - s_l[centre + s_off[k]], 0.0f);
      }
      float shade = ex2_ftz(p.minus_a_log2e * (w * p.inv_n));
      if (p.ao)
        shade *= __ldg((const float*)((const char*)p.ao + (size_t)__float2int_rd(((float)y + 0.5f) * p.ao_inv) *
                                                              p.ao_pitch) +
                       __float2int_rd(((float)x + 0.5f) * p.ao_inv));
      c = edl_colour<FMT>(g, x, y) * shade;
    }
    if (hdr) store_hdr<HDR>(hdr, hdr_pitch, x, y, c);
    if (LDR) ((unsigned*)(ldr + (size_t)y * ldr_pitch))[x] = pack_rgba8(c, exposure, op);
  }
}

template <int FMT, int HDR>
static void launch_edl(dim3 grd, dim3 blk, cudaStream_t s, const GbufDev& g, const EdlDev& p, void* hdr,
                       long long hp, float exposure, int op, uint8_t* ldr, long long lp) {
  if (p.N == 8) {  // the usual eight directions: neighbour loop unrolled
    if (ldr)
      k_edl<FMT, HDR, true, 8><<<grd, blk, 0, s>>>(g, p, hdr, hp, exposure, op, ldr, lp);
    else
      k_edl<FMT, HDR, false, 8><<<grd, blk, 0, s>>>(g, p, hdr, hp, exposure, op, ldr, lp);
  } else {
    if (ldr)
      k_edl<FMT, HDR, true, 0><<<grd, blk, 0, s>>>(g, p, hdr, hp, exposure, op, ldr, lp);
    else
      k_edl<FMT, HDR, false, 0><<<grd, blk, 0, s>>>(g, p, hdr, hp, exposure, op, ldr, lp);
  }
}

}  // namespace epbr

using namespace epbr;

extern "C" epbr_status epbr_edl(const epbr_gbuffer* g, const epbr_edl_params* params, const float* ao, int64_t ao_pitch,
                                int32_t ao_scale, void* hdr, int32_t hdr_format, int64_t hdr_pitch,
                                const epbr_tonemap_params* tp, uint8_t* ldr, int64_t ldr_pitch, void* stream) {
  if (!g) return fail(EPBR_ERR_INVALID_ARG, "edl: gbuffer is NULL");
  if (g->width < 1 || g->height < 1 || g->width > (1 << 15) || g->height > (1 << 15))
    return fail(EPBR_ERR_INVALID_ARG, "edl: gbuffer size %dx%d outside [1, 32768]", g->width, g->height);
  if (g->format != EPBR_GBUFFER_FP32 && g->format != EPBR_GBUFFER_COMPACT)
    return fail(EPBR_ERR_INVALID_ARG, "edl: gbuffer format %d unknown", g->format);
  const int cb = g->format == EPBR_GBUFFER_FP32 ? 16 : 4;  // bytes per colour texel
  if (!g->rt[0] || (uintptr_t)g->rt[0] % cb || g->pitch[0] < (int64_t)cb * g->width || g->pitch[0] % cb)
    return fail(EPBR_ERR_INVALID_ARG, "edl: colour plane rt[0] NULL, misaligned or pitch too small");
  if (!g->rt[3] || (uintptr_t)g->rt[3] % 4 || g->pitch[3] < (int64_t)4 * g->width || g->pitch[3] % 4)
    return fail(EPBR_ERR_INVALID_ARG, "edl: depth plane rt[3] NULL, misaligned or pitch too small");
  if (!params || !(params->strength >= 0.0f) || !std::isfinite(params->strength) || params->radius < 1 ||
      params->radius > kEdlMaxR || params->directions < 1 || params->directions > kEdlMaxN)
    return fail(EPBR_ERR_INVALID_ARG, "edl: strength >= 0, radius 1..%d, directions 1..%d required", kEdlMaxR,
                kEdlMaxN);
  if (hdr_format != EPBR_HDR_RGBA32F && hdr_format != EPBR_HDR_RGBA16F)
    return fail(EPBR_ERR_INVALID_ARG, "edl: hdr_format %d unknown", hdr_format);
  const int bpp = hdr_format == EPBR_HDR_RGBA32F ? 16 : 8;
  if (hdr && ((uintptr_t)hdr % bpp || hdr_pitch < (int64_t)bpp * g->width || hdr_pitch % bpp))
    return fail(EPBR_ERR_INVALID_ARG, "edl: hdr misaligned or pitch too small");
  if (!hdr && !ldr) return fail(EPBR_ERR_INVALID_ARG, "edl: no output");
  if (ldr && ((uintptr_t)ldr % 4 || ldr_pitch < (int64_t)4 * g->width || ldr_pitch % 4))
    return fail(EPBR_ERR_INVALID_ARG, "edl: ldr misaligned or pitch too small");
  if (ldr && (!tp || !(tp->exposure >= 0.0f) || (tp->op != EPBR_TONEMAP_ACES && tp->op != EPBR_TONEMAP_REINHARD)))
    return fail(EPBR_ERR_INVALID_ARG, "edl: tonemap params invalid");
  EdlDev p;
  memset(&p, 0, sizeof(p));
  if (ao) {
    int s = ao_scale < 1 ? 1 : ao_scale;
    int Wa = (g->width + s - 1) / s;
    if (ao_scale > 8 || (uintptr_t)ao % 4 || ao_pitch < (int64_t)Wa * 4 || ao_pitch % 4)
      return fail(EPBR_ERR_INVALID_ARG, "edl: ao misaligned, pitch too small or scale > 8");
    p.ao = ao;
    p.ao_pitch = ao_pitch;
    p.ao_inv = 1.0f / (float)s;
  }
  p.R = params->radius;
  p.N = params->directions;
  p.inv_n = 1.0f / (float)p.N;
  p.minus_a_log2e = (float)(-(double)params->strength / std::log(2.0));
  for (int k = 0; k < p.N; ++k) {
    double t = 2.0 * 3.14159265358979323846 * k / p.N;
    p.dx[k] = (signed char)std::lround(params->radius * std::cos(t));
    p.dy[k] = (signed char)std::lround(params->radius * std::sin(t));
  }
  GbufDev gd = make_gbuf(*g);
  dim3 blk(kEdlBX, kEdlBY), grd((g->width + kEdlBX - 1) / kEdlBX, (g->height + kEdlTileH - 1) / kEdlTileH);
  cudaStream_t s = (cudaStream_t)stream;
  float exposure = tp ? tp->exposure : 1.0f;
  int op = tp ? tp->op : 0;
  if (g->format == EPBR_GBUFFER_FP32) {
    if (hdr_format == EPBR_HDR_RGBA32F)
      launch_edl<EPBR_GBUFFER_FP32, EPBR_HDR_RGBA32F>(grd, blk, s, gd, p, hdr, hdr_pitch, exposure, op, ldr, ldr_pitch);
    else
      launch_edl<EPBR_GBUFFER_FP32, EPBR_HDR_RGBA16F>(grd, blk, s, gd, p, hdr, hdr_pitch, exposure, op, ldr, ldr_pitch);
  } else {
    if (hdr_format == EPBR_HDR_RGBA32F)
      launch_edl<EPBR_GBUFFER_COMPACT, EPBR_HDR_RGBA32F>(grd, blk, s, gd, p, hdr, hdr_pitch, exposure, op, ldr, ldr_pitch);
    else
      launch_edl<EPBR_GBUFFER_COMPACT, EPBR_HDR_RGBA16F>(grd, blk, s, gd, p, hdr, hdr_pitch, exposure, op, ldr, ldr_pitch);
  }
  epbr_status st = check_launch("k_edl");
  return st ? st : ok();
}
