// Deferred compose and tone mapping of one view.
//   k_shade    two pixels per thread in 32x8 blocks (32x16 pixel tiles): G-buffer decode,
//              Cook-Torrance over the point lights (a list of up to 256 copied into shared
//              memory by a TMA bulk copy, longer lists staged in chunks of 256 by plain loads;
//              monochrome chunks in packed FP32x2 arithmetic), split-sum IBL times AO,
//              background from the environment; optional fused tone-map epilogue (Sec. 5.4).
//              The per-pixel arithmetic lives in shade_core.cuh.
//   k_tonemap  ACES / Reinhard + sRGB transfer, 8-bit output
#include <string.h>

#include <algorithm>

#include "shade_core.cuh"
#include "tma.cuh"

namespace epbr {

#ifndef EPBR_SHADE_BY
#define EPBR_SHADE_BY 8  // block rows of threads (block = 32 x EPBR_SHADE_BY threads, two pixels each)
#endif
constexpr int kShadeBX = 32, kShadeBY = EPBR_SHADE_BY;
constexpr int kShadeTileH = 2 * kShadeBY;  // pixel rows per block
#ifndef EPBR_SHADE_MIN_BLOCKS
#define EPBR_SHADE_MIN_BLOCKS 2  // resident blocks per SM the register budget targets
#endif

// Compose blocks whose wait for the TMA copy of their light list ran out (they read the list from
// global memory instead: the same values); read and cleared by epbr_shade_light_timeouts.  The
// second flag records a block whose drain wait before exiting ran out as well.
__device__ unsigned int g_light_stage_timeouts;
__device__ unsigned int g_light_stage_lost;

// Two vertically adjacent pixels per thread, a 32 x 2*EPBR_SHADE_BY tile per block.  A list of at
// most 256 lights is copied into shared memory by one TMA bulk copy (issued first, completing on
// an mbarrier, bounded wait) while the G-buffer loads are in flight; the block then stages it as
// (pos, I c) and the packed loop's duplicated form.  Longer lists are staged in chunks of 256 by
// plain loads.  A chunk whose lights are all monochrome takes the packed two-pixel loop
// (px_direct_mono2), any other chunk the per-pixel colour loop.
template <int FMT, int HDR, bool LDR>
__global__ void __launch_bounds__(kShadeBX* kShadeBY, EPBR_SHADE_MIN_BLOCKS)
    k_shade(GbufDev g, CamDev cam, const float4* __restrict__ lights, int NL, IblDev ibl, ShadeDev p, void* hdr,
            long long hdr_pitch, uint8_t* ldr, long long ldr_pitch, unsigned long long wait_ns) {
  __shared__ float4 s_lights[2 * kLightChunk];
  __shared__ float4 s_dup[2 * kLightChunk];
  __shared__ __align__(16) float4 s_raw[2 * kLightChunk];  // the list as the bulk copy lands it
  __shared__ __align__(8) unsigned long long s_bar;
  constexpr int kThreads = kShadeBX * kShadeBY;
  int tid = threadIdx.y * kShadeBX + threadIdx.x;
  const bool tma = NL > 0 && NL <= kLightChunk;  // launch-uniform
  if (tma && tid == 0) tma_load_bulk(s_raw, lights, smem_addr(&s_bar), (unsigned)NL * 32u);
  // Rows are dispatched bottom-up: the costliest tiles (ground and objects) usually fill the
  // bottom of a view and the cheap background the top, so the expensive work starts first and
  // the tail of the launch is short.  Any order gives the same image.
  int by = gridDim.y - 1 - blockIdx.y;
  int x = blockIdx.x * kShadeBX + threadIdx.x;
  int yy[2] = {by * kShadeTileH + 2 * (int)threadIdx.y, by * kShadeTileH + 2 * (int)threadIdx.y + 1};
  bool in[2] = {x < g.W && yy[0] < g.H, x < g.W && yy[1] < g.H};
  PxRaw raw[2];
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (in[h]) raw[h] = px_load<FMT>(g, x, yy[h]);
  bool mono = false, staged = true;
  if (tma) {
    __syncthreads();  // orders the mbarrier's initialisation before every thread's wait
    // wait_ns = 0 gives up at once (the fallback path, exercised by a test)
    staged = __syncthreads_and(wait_ns != 0 && mbar_wait_bounded(smem_addr(&s_bar), 0, wait_ns));
    if (!staged && tid == 0) atomicAdd(&g_light_stage_timeouts, 1u);
    mono = __syncthreads_and(staged ? stage_lights<true>(s_lights, s_raw, 0, NL, tid, kThreads, s_dup)
                                    : stage_lights(s_lights, lights, 0, NL, tid, kThreads, s_dup));
  } else if (NL == 0) {
    mono = true;
  }
  Px s[2];
  bool act[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (in[h]) s[h] = px_decode<FMT>(raw[h], cam, x, yy[h]);
    act[h] = in[h] && s[h].surface;
  }
  shade_lights(s, act, NL, p.flags, lights, s_lights, s_dup, kLightChunk, NL <= kLightChunk, mono, tid, kThreads);
  // Launched early (EPBR_SHADE_EARLY_START), the kernel before this one on the stream may still be
  // running up to here: the AO it writes is read, and the outputs written, only after it ends.
  griddep_wait();
  float ao[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) ao[h] = act[h] ? ao_at(p, x, yy[h]) : 1.0f;
  // Both pixels' lookups are issued before either is stored.
  float3 c[2];
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (in[h]) c[h] = px_finish(s[h], ibl, p.flags, ao[h]);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!in[h]) continue;
    if (hdr) store_hdr<HDR>(hdr, hdr_pitch, x, yy[h], c[h]);
    if (LDR) ((unsigned*)(ldr + (size_t)yy[h] * ldr_pitch))[x] = pack_rgba8(c[h], p.exposure, p.op);
  }
  // a copy that had not landed is waited for once more (bounded) before the block's shared memory
  // can go to another block; if that wait runs out too, the launch is flagged
  if (tma && !staged && !mbar_wait_bounded(smem_addr(&s_bar), 0, kTmaWaitNs) && tid == 0)
    atomicOr(&g_light_stage_lost, 1u);
}

template <int HDR>
__global__ void k_tonemap(const void* __restrict__ hdr, long long hdr_pitch, int W, int H, float exposure, int op,
                          uint8_t* __restrict__ out, long long out_pitch) {
  int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  float3 c = load_hdr<HDR>(hdr, hdr_pitch, x, y);
  ((unsigned*)(out + (size_t)y * out_pitch))[x] = pack_rgba8(c, exposure, op);
}

static epbr_status make_ibl_dev(const epbr_ibl* ibl, IblDev* d) {
  if (!ibl) return fail(EPBR_ERR_INVALID_ARG, "shade: EPBR_SHADE_IBL set but ibl is NULL");
  if (!ibl->irradiance || !ibl->lut || ibl->irr_width < 1 || ibl->irr_height < 1 || ibl->lut_size < 1 ||
      ibl->num_levels < 1 || ibl->num_levels > EPBR_MAX_LEVELS)
    return fail(EPBR_ERR_INVALID_ARG, "shade: ibl incomplete");
  d->irr = MapDev{(const float4*)ibl->irradiance, ibl->irr_width, ibl->irr_height};
  for (int m = 0; m < EPBR_MAX_LEVELS; ++m) {
    if (m < ibl->num_levels) {
      if (!ibl->level[m] || ibl->level_width[m] < 1 || ibl->level_height[m] < 1)
        return fail(EPBR_ERR_INVALID_ARG, "shade: ibl level %d invalid", m);
      d->lev[m] = MapDev{(const float4*)ibl->level[m], ibl->level_width[m], ibl->level_height[m]};
    } else {
      d->lev[m] = MapDev{nullptr, 1, 1};
    }
  }
  d->lut = (const float2*)ibl->lut;
  d->S = ibl->lut_size;
  d->M = ibl->num_levels;
  return EPBR_OK;
}

template <int FMT, int HDR>
static cudaError_t launch_shade(dim3 grd, dim3 blk, cudaStream_t s, const GbufDev& g, const CamDev& c, const float4* L,
                         int NL, const IblDev& ibl, const ShadeDev& p, void* hdr, long long hp, uint8_t* ldr,
                         long long lp) {
  const unsigned long long w = tma_first_wait_ns();
  const bool early = (p.flags & EPBR_SHADE_EARLY_START) != 0;
  cudaError_t e = launch_kernel(ldr ? k_shade<FMT, HDR, true> : k_shade<FMT, HDR, false>, grd, blk, 0, s, early, g, c, L,
                                NL, ibl, p, hdr, hp, ldr, lp, w);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

static epbr_status shade_common(const epbr_gbuffer* g, const epbr_camera* cam, const epbr_light* lights,
                                int32_t NL, const epbr_ibl* ibl, const epbr_shade_params* sp, void* hdr,
                                int32_t hdr_format, int64_t hdr_pitch, const epbr_tonemap_params* tp,
                                uint8_t* ldr, int64_t ldr_pitch, void* stream, bool shadowed = false,
                                const epbr_shadows* shadows = nullptr) {
  epbr_status st = validate_gbuffer(g, true);
  if (st) return st;
  if ((st = validate_camera(cam, g))) return st;
  if (!sp) return fail(EPBR_ERR_INVALID_ARG, "shade params is NULL");
  if (sp->flags & ~(unsigned)(EPBR_SHADE_DIRECT | EPBR_SHADE_IBL | EPBR_SHADE_MULTISCATTER | EPBR_SHADE_DIFFUSE_ONLY |
                              EPBR_SHADE_EARLY_START))
    return fail(EPBR_ERR_INVALID_ARG, "shade flags 0x%x has unknown bits", sp->flags);
  if (NL < 0 || NL > 65536) return fail(EPBR_ERR_INVALID_ARG, "num_lights %d outside [0, 65536]", NL);
  if (NL > 0 && (sp->flags & EPBR_SHADE_DIRECT) && (!lights || (uintptr_t)lights % 16))
    return fail(EPBR_ERR_INVALID_ARG, "lights NULL or not 16-byte aligned");
  if (hdr_format != EPBR_HDR_RGBA32F && hdr_format != EPBR_HDR_RGBA16F)
    return fail(EPBR_ERR_INVALID_ARG, "hdr_format %d unknown", hdr_format);
  int bpp = hdr_format == EPBR_HDR_RGBA32F ? 16 : 8;
  if (hdr && ((uintptr_t)hdr % bpp || hdr_pitch < (int64_t)bpp * g->width || hdr_pitch % bpp))
    return fail(EPBR_ERR_INVALID_ARG, "hdr buffer misaligned or pitch too small");
  if (!hdr && !ldr) return fail(EPBR_ERR_INVALID_ARG, "no output buffer");
  if (ldr && ((uintptr_t)ldr % 4 || ldr_pitch < (int64_t)4 * g->width || ldr_pitch % 4))
    return fail(EPBR_ERR_INVALID_ARG, "ldr buffer misaligned or pitch too small");
  if (ldr && (!tp || !(tp->exposure >= 0.0f) || (tp->op != EPBR_TONEMAP_ACES && tp->op != EPBR_TONEMAP_REINHARD)))
    return fail(EPBR_ERR_INVALID_ARG, "tonemap params invalid");
  ShadeDev p;
  p.flags = sp->flags;
  p.ao = sp->ao;
  p.ao_pitch = sp->ao_pitch;
  p.ao_scale = sp->ao_scale < 1 ? 1 : sp->ao_scale;
  p.ao_inv = 1.0f / (float)p.ao_scale;
  p.exposure = tp ? tp->exposure : 1.0f;
  p.op = tp ? tp->op : 0;
  if (sp->ao) {
    int Wa = (g->width + p.ao_scale - 1) / p.ao_scale;
    if ((uintptr_t)sp->ao % 4 || sp->ao_pitch < (int64_t)Wa * 4 || sp->ao_pitch % 4 || sp->ao_scale > 8)
      return fail(EPBR_ERR_INVALID_ARG, "ao buffer misaligned, pitch too small or scale > 8");
  }
  IblDev ib;
  memset(&ib, 0, sizeof(ib));
  if (sp->flags & EPBR_SHADE_IBL) {
    if ((st = make_ibl_dev(ibl, &ib))) return st;
  } else {
    for (int m = 0; m < EPBR_MAX_LEVELS; ++m) ib.lev[m] = MapDev{nullptr, 1, 1};
    ib.irr = MapDev{nullptr, 1, 1};
    ib.S = ib.M = 1;
  }
  GbufDev gd = make_gbuf(*g);
  CamDev cd = make_cam(*cam);
  dim3 blk(kShadeBX, kShadeBY), grd((g->width + kShadeBX - 1) / kShadeBX, (g->height + kShadeTileH - 1) / kShadeTileH);
  cudaStream_t s = (cudaStream_t)stream;
  const float4* L = (const float4*)lights;
  int nl = (sp->flags & EPBR_SHADE_DIRECT) ? NL : 0;
  if (shadowed) {
    if ((st = launch_shade_shadows(gd, cd, g->format, L, nl, ib, p, shadows, hdr, hdr_format, hdr_pitch, ldr, ldr_pitch,
                                   s)))
      return st;
    return ok();
  }
  cudaError_t e;
  if (g->format == EPBR_GBUFFER_FP32) {
    if (hdr_format == EPBR_HDR_RGBA32F)
      e = launch_shade<EPBR_GBUFFER_FP32, EPBR_HDR_RGBA32F>(grd, blk, s, gd, cd, L, nl, ib, p, hdr, hdr_pitch, ldr,
                                                            ldr_pitch);
    else
      e = launch_shade<EPBR_GBUFFER_FP32, EPBR_HDR_RGBA16F>(grd, blk, s, gd, cd, L, nl, ib, p, hdr, hdr_pitch, ldr,
                                                            ldr_pitch);
  } else {
    if (hdr_format == EPBR_HDR_RGBA32F)
      e = launch_shade<EPBR_GBUFFER_COMPACT, EPBR_HDR_RGBA32F>(grd, blk, s, gd, cd, L, nl, ib, p, hdr, hdr_pitch, ldr,
                                                               ldr_pitch);
    else
      e = launch_shade<EPBR_GBUFFER_COMPACT, EPBR_HDR_RGBA16F>(grd, blk, s, gd, cd, L, nl, ib, p, hdr, hdr_pitch, ldr,
                                                               ldr_pitch);
  }
  if (e != cudaSuccess) return fail(EPBR_ERR_CUDA, "k_shade: %s", cudaGetErrorString(e));
  if ((st = check_launch("k_shade"))) return st;
  return ok();
}

}  // namespace epbr

using namespace epbr;

extern "C" epbr_status epbr_shade(const epbr_gbuffer* g, const epbr_camera* cam, const epbr_light* lights, int32_t NL,
                                  const epbr_ibl* ibl, const epbr_shade_params* sp, void* hdr, int32_t hdr_format,
                                  int64_t hdr_pitch, void* stream) {
  if (!hdr) return fail(EPBR_ERR_INVALID_ARG, "hdr is NULL");
  return shade_common(g, cam, lights, NL, ibl, sp, hdr, hdr_format, hdr_pitch, nullptr, nullptr, 0, stream);
}

extern "C" epbr_status epbr_shade_tonemap(const epbr_gbuffer* g, const epbr_camera* cam, const epbr_light* lights,
                                          int32_t NL, const epbr_ibl* ibl, const epbr_shade_params* sp, void* hdr,
                                          int32_t hdr_format, int64_t hdr_pitch, const epbr_tonemap_params* tp,
                                          uint8_t* ldr, int64_t ldr_pitch, void* stream) {
  if (!ldr) return fail(EPBR_ERR_INVALID_ARG, "ldr is NULL");
  return shade_common(g, cam, lights, NL, ibl, sp, hdr, hdr_format, hdr_pitch, tp, ldr, ldr_pitch, stream);
}

extern "C" epbr_status epbr_shade_light_timeouts(uint32_t* count) {
  if (!count) return fail(EPBR_ERR_INVALID_ARG, "count is NULL");
  unsigned v = 0, lost = 0;
  const unsigned zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_light_stage_timeouts, sizeof(v)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_light_stage_timeouts, &zero, sizeof(zero)) != cudaSuccess ||
      cudaMemcpyFromSymbol(&lost, g_light_stage_lost, sizeof(lost)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_light_stage_lost, &zero, sizeof(zero)) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "shade_light_timeouts: %s", cudaGetErrorString(cudaGetLastError()));
  *count = v;
  if (lost)
    return fail(EPBR_ERR_DEVICE_STATUS,
                "shade_light_timeouts: a block's light-list copy did not complete within two waits of %llu ms; "
                "the results of launches since the last call are suspect",
                (unsigned long long)(kTmaWaitNs / 1000000));
  return ok();
}

extern "C" epbr_status epbr_tonemap(const void* hdr, int32_t hdr_format, int32_t W, int32_t H, int64_t hdr_pitch,
                                    const epbr_tonemap_params* tp, uint8_t* out, int64_t out_pitch, void* stream) {
  if (!hdr || !out || !tp) return fail(EPBR_ERR_INVALID_ARG, "tonemap: NULL argument");
  if (W < 1 || H < 1 || W > (1 << 15) || H > (1 << 15)) return fail(EPBR_ERR_INVALID_ARG, "tonemap: size invalid");
  if (hdr_format != EPBR_HDR_RGBA32F && hdr_format != EPBR_HDR_RGBA16F)
    return fail(EPBR_ERR_INVALID_ARG, "tonemap: hdr_format %d unknown", hdr_format);
  int bpp = hdr_format == EPBR_HDR_RGBA32F ? 16 : 8;
  if ((uintptr_t)hdr % bpp || hdr_pitch < (int64_t)bpp * W || hdr_pitch % bpp)
    return fail(EPBR_ERR_INVALID_ARG, "tonemap: hdr misaligned or pitch too small");
  if ((uintptr_t)out % 4 || out_pitch < (int64_t)4 * W || out_pitch % 4)
    return fail(EPBR_ERR_INVALID_ARG, "tonemap: out misaligned or pitch too small");
  if (!(tp->exposure >= 0.0f) || (tp->op != EPBR_TONEMAP_ACES && tp->op != EPBR_TONEMAP_REINHARD))
    return fail(EPBR_ERR_INVALID_ARG, "tonemap: params invalid");
  dim3 blk(256), grd((W + 255) / 256, H);
  cudaStream_t s = (cudaStream_t)stream;
  if (hdr_format == EPBR_HDR_RGBA32F)
    k_tonemap<EPBR_HDR_RGBA32F><<<grd, blk, 0, s>>>(hdr, hdr_pitch, W, H, tp->exposure, tp->op, out, out_pitch);
  else
    k_tonemap<EPBR_HDR_RGBA16F><<<grd, blk, 0, s>>>(hdr, hdr_pitch, W, H, tp->exposure, tp->op, out, out_pitch);
  epbr_status st = check_launch("k_tonemap");
  return st ? st : ok();
}

extern "C" epbr_status epbr_shade_shadows(const epbr_gbuffer* g, const epbr_camera* cam, const epbr_light* lights,
                                          int32_t NL, const epbr_ibl* ibl, const epbr_shade_params* sp,
                                          const epbr_shadows* shadows, void* hdr, int32_t hdr_format,
                                          int64_t hdr_pitch, const epbr_tonemap_params* tp, uint8_t* ldr,
                                          int64_t ldr_pitch, void* stream) {
  return shade_common(g, cam, lights, NL, ibl, sp, hdr, hdr_format, hdr_pitch, tp, ldr, ldr_pitch, stream, true,
                      shadows);
}
