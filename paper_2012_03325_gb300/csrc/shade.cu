// Deferred compose and tone mapping.
//   k_shade    per pixel: G-buffer decode (Table 1 layouts; position from depth, Sec. 4),
//              Cook-Torrance over the point lights (Sec. 3 Eq. 1, UE4 model), split-sum IBL
//              with multiple-scattering compensation (Sec. 3.1) times AO, background from the
//              environment; optional fused tone-map epilogue (Sec. 5.4)
//   k_tonemap  ACES / Reinhard + sRGB transfer, 8-bit output
//
// Direct-light arithmetic avoids normalising the half vector: with s = l + v,
//   n.h = n.s / |s|,  1 - (n.h)^2 = |n x s|^2 / |s|^2,  |s|^2 = 2 + 2 l.v,  v.h = |s| / 2,
// so D = alpha^2 |s|^4 / (pi ((n.s)^2 alpha^2 + |n x s|^2)^2), which is the GGX distribution
// written without the 1 - (n.h)^2 cancellation that loses all precision at alpha^2 ~ 4e-6.
#include <string.h>

#include "epbr_internal.cuh"

namespace epbr {

__constant__ float c_srgb8[256] = {
#include "srgb8_table.inc"
};

constexpr int kLightChunk = 256;
constexpr int kShadeBX = 32, kShadeBY = 8;

struct IblDev {
  MapDev irr;
  MapDev lev[EPBR_MAX_LEVELS];
  const float2* lut;
  int S, M;
};

struct ShadeDev {
  unsigned flags;
  int ao_scale;
  const float* ao;
  long long ao_pitch;
  float exposure;
  int op;
};

// Tone map one channel: clamp exposure * x to [0, 1e6], ACES fit (Narkowicz 2015) or Reinhard,
// clamp to [0, 1], sRGB transfer (IEC 61966-2-1), round half up to 8 bits.
__device__ __forceinline__ unsigned tonemap_channel(float x, float exposure, int op) {
  x = fminf(fmaxf(x * exposure, 0.0f), 1e6f);
  float y = (op == EPBR_TONEMAP_REINHARD) ? x / (1.0f + x)
                                          : x * fmaf(2.51f, x, 0.03f) / fmaf(x, fmaf(2.43f, x, 0.59f), 0.14f);
  y = clamp01(y);
  float s = y <= 0.0031308f ? 12.92f * y : fmaf(1.055f, powf(y, 1.0f / 2.4f), -0.055f);
  return (unsigned)floorf(fmaf(255.0f, s, 0.5f));
}

__device__ __forceinline__ unsigned pack_rgba8(float3 c, float exposure, int op) {
  return tonemap_channel(c.x, exposure, op) | (tonemap_channel(c.y, exposure, op) << 8) |
         (tonemap_channel(c.z, exposure, op) << 16) | (255u << 24);
}

__device__ __forceinline__ float sat_half(float x) { return fminf(fmaxf(x, -65504.0f), 65504.0f); }

template <int HDR>
__device__ __forceinline__ void store_hdr(void* hdr, long long pitch, int x, int y, float3 c) {
  char* row = (char*)hdr + (size_t)y * pitch;
  if (HDR == EPBR_HDR_RGBA32F) {
    ((float4*)row)[x] = make_float4(c.x, c.y, c.z, 1.0f);
  } else {
    __half2 a = __floats2half2_rn(sat_half(c.x), sat_half(c.y));
    __half2 b = __floats2half2_rn(sat_half(c.z), 1.0f);
    uint2 u;
    u.x = *reinterpret_cast<unsigned*>(&a);
    u.y = *reinterpret_cast<unsigned*>(&b);
    ((uint2*)row)[x] = u;
  }
}

template <int HDR>
__device__ __forceinline__ float3 load_hdr(const void* hdr, long long pitch, int x, int y) {
  const char* row = (const char*)hdr + (size_t)y * pitch;
  if (HDR == EPBR_HDR_RGBA32F) {
    float4 v = __ldg((const float4*)row + x);
    return xyz(v);
  } else {
    uint2 u = __ldg((const uint2*)row + x);
    float2 a = __half22float2(*reinterpret_cast<__half2*>(&u.x));
    float2 b = __half22float2(*reinterpret_cast<__half2*>(&u.y));
    return f3(a.x, a.y, b.x);
  }
}

struct Material {
  float3 albedo;
  float metal, rough;
};

template <int FMT>
__device__ __forceinline__ Material gb_material(const GbufDev& g, int x, int y) {
  Material m;
  if (FMT == EPBR_GBUFFER_FP32) {
    float4 a = __ldg((const float4*)(g.rt[0] + (size_t)y * g.pitch[0]) + x);
    float r = __ldg((const float4*)(g.rt[1] + (size_t)y * g.pitch[1]) + x).w;
    m.albedo = xyz(a);
    m.metal = a.w;
    m.rough = r;
  } else {
    uchar4 a = __ldg((const uchar4*)(g.rt[0] + (size_t)y * g.pitch[0]) + x);
    uchar2 mr = __ldg((const uchar2*)(g.rt[2] + (size_t)y * g.pitch[2]) + x);
    m.albedo = f3(c_srgb8[a.x], c_srgb8[a.y], c_srgb8[a.z]);
    m.metal = mr.x * (1.0f / 255.0f);
    m.rough = mr.y * (1.0f / 255.0f);
  }
  m.metal = clamp01(m.metal);
  m.rough = fminf(fmaxf(m.rough, kRoughMin), 1.0f);
  return m;
}

// Bilinear read of the BRDF table, clamp to edge.
__device__ __forceinline__ float2 lut_bilinear(const float2* lut, int S, float mu, float r) {
  float x = fmaf(mu, (float)S, -0.5f), y = fmaf(r, (float)S, -0.5f);
  float x0 = floorf(x), y0 = floorf(y), fx = x - x0, fy = y - y0;
  int i0 = min(max((int)x0, 0), S - 1), i1 = min(max((int)x0 + 1, 0), S - 1);
  int j0 = min(max((int)y0, 0), S - 1), j1 = min(max((int)y0 + 1, 0), S - 1);
  float2 a = __ldg(lut + j0 * S + i0), b = __ldg(lut + j0 * S + i1);
  float2 p = __ldg(lut + j1 * S + i0), q = __ldg(lut + j1 * S + i1);
  float tx = fmaf(fx, b.x - a.x, a.x), ty = fmaf(fx, b.y - a.y, a.y);
  float bx = fmaf(fx, q.x - p.x, p.x), by = fmaf(fx, q.y - p.y, p.y);
  return make_float2(fmaf(fy, bx - tx, tx), fmaf(fy, by - ty, ty));
}

// Everything one pixel needs; returns linear HDR radiance.
template <int FMT>
__device__ __forceinline__ float3 shade_pixel(const GbufDev& g, const CamDev& cam, const float4* s_lights,
                                              int NL, const float4* __restrict__ lights_g, const IblDev& ibl,
                                              const ShadeDev& p, int x, int y, bool staged) {
  float e = gb_depth(g, x, y);
  float3 r = view_ray(cam, x, y);
  float3 dw = rot(cam, r);
  if (!is_surface(e)) {
    if (p.flags & EPBR_SHADE_IBL) return equirect_lookup(ibl.lev[0], dw);
    return f3(0, 0, 0);
  }
  float3 eye = f3(cam.eye[0], cam.eye[1], cam.eye[2]);
  float3 P = eye + e * dw;
  float3 v = normalize3(dw) * -1.0f;
  float3 n = gb_normal<FMT>(g, x, y);
  Material m = gb_material<FMT>(g, x, y);
  float nv_raw = dot3(n, v);
  float nv = fmaxf(nv_raw, kNvMin);
  bool diffuse_only = (p.flags & EPBR_SHADE_DIFFUSE_ONLY) != 0;
  float3 F0 = f3(fmaf(m.metal, m.albedo.x - 0.04f, 0.04f), fmaf(m.metal, m.albedo.y - 0.04f, 0.04f),
                 fmaf(m.metal, m.albedo.z - 0.04f, 0.04f));
  float3 cdiff = m.albedo * (1.0f - m.metal);
  float3 acc = f3(0, 0, 0);
  if (p.flags & EPBR_SHADE_DIRECT) {
    float alpha = m.rough * m.rough, a2 = alpha * alpha;
    float k = (m.rough + 1.0f) * (m.rough + 1.0f) * 0.125f, omk = 1.0f - k;
    float vv = 1.0f / (4.0f * kPi * fmaf(nv, omk, k));  // G1(v) / (4 pi n.v)
    float3 cdpi = diffuse_only ? m.albedo * kInvPi : cdiff * kInvPi;
    float3 omF0 = f3(1.0f - F0.x, 1.0f - F0.y, 1.0f - F0.z);
    for (int i = 0; i < NL; ++i) {
      float4 la = staged ? s_lights[2 * i] : __ldg(lights_g + 2 * i);
      float4 lc = staged ? s_lights[2 * i + 1] : __ldg(lights_g + 2 * i + 1);
      float3 L = xyz(la) - P;
      float d2 = dot3(L, L);
      float rs = rsqrtf(d2);
      float nl = dot3(n, L) * rs;
      if (nl > 0.0f) {
        float3 rad = xyz(lc) * (la.w * rs * rs * nl);  // I c / d^2 (n.l)
        if (diffuse_only) {
          acc = acc + mul3(cdpi, rad);
          continue;
        }
        float lv = dot3(v, L) * rs;
        float3 s = L * rs + v;
        float3 c = cross3(n, s);
        float c2 = dot3(c, c);
        float ns = nl + nv_raw;
        float hh = fmaxf(fmaf(2.0f, lv, 2.0f), 1e-30f);
        float den = fmaf(ns * ns, a2, c2);
        float vh = 0.5f * hh * rsqrtf(hh);
        float xx = 1.0f - vh, x2 = xx * xx, fc = x2 * x2 * xx;
        float spec = a2 * hh * hh * vv / fmaxf(den * den * fmaf(nl, omk, k), 1e-37f);
        float3 F = f3(fmaf(omF0.x, fc, F0.x), fmaf(omF0.y, fc, F0.y), fmaf(omF0.z, fc, F0.z));
        acc.x = fmaf(fmaf(F.x, spec - cdpi.x, cdpi.x), rad.x, acc.x);
        acc.y = fmaf(fmaf(F.y, spec - cdpi.y, cdpi.y), rad.y, acc.y);
        acc.z = fmaf(fmaf(F.z, spec - cdpi.z, cdpi.z), rad.z, acc.z);
      }
    }
  }
  if (p.flags & EPBR_SHADE_IBL) {
    float ao = 1.0f;
    if (p.ao) ao = __ldg((const float*)((const char*)p.ao + (size_t)(y / p.ao_scale) * p.ao_pitch) + x / p.ao_scale);
    float3 irr = equirect_lookup(ibl.irr, n);
    if (diffuse_only) {
      acc = acc + mul3(m.albedo, irr) * ao;
    } else {
      float3 R = n * (2.0f * nv_raw) - v;
      float lod = m.rough * (float)(ibl.M - 1);
      int l0 = min((int)floorf(lod), ibl.M - 1);
      int l1 = min(l0 + 1, ibl.M - 1);
      float tl = lod - (float)l0;
      float u, vv2;
      dir_to_uv(R, u, vv2);
      float3 p0 = equirect_bilinear(ibl.lev[l0], u, vv2);
      float3 p1 = equirect_bilinear(ibl.lev[l1], u, vv2);
      float3 pref = p0 + tl * (p1 - p0);
      float2 AB = lut_bilinear(ibl.lut, ibl.S, clamp01(nv), m.rough);
      float xv = 1.0f - nv, xv2 = xv * xv, fcv = xv2 * xv2 * xv;
      float Fr_base = 1.0f - m.rough;
      float F0a[3] = {F0.x, F0.y, F0.z}, cd[3] = {cdiff.x, cdiff.y, cdiff.z};
      float pr[3] = {pref.x, pref.y, pref.z}, ir[3] = {irr.x, irr.y, irr.z}, la[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        float Fr = fmaxf(Fr_base, F0a[q]) - F0a[q];
        float kS = fmaf(Fr, fcv, F0a[q]);
        if (p.flags & EPBR_SHADE_MULTISCATTER) {
          float FssEss = fmaf(kS, AB.x, AB.y);
          float Ess = AB.x + AB.y, Ems = 1.0f - Ess;
          float Favg = F0a[q] + (1.0f - F0a[q]) * (1.0f / 21.0f);
          float Fms = FssEss * Favg / (1.0f - Ems * Favg);
          float kD = cd[q] * (1.0f - FssEss - Fms * Ems);
          la[q] = fmaf(FssEss, pr[q], (Fms * Ems + kD) * ir[q]);
        } else {
          la[q] = fmaf((1.0f - kS) * cd[q], ir[q], fmaf(kS, AB.x, AB.y) * pr[q]);
        }
      }
      acc = acc + f3(la[0], la[1], la[2]) * ao;
    }
  }
  return acc;
}

template <int FMT, int HDR, bool LDR>
__global__ void __launch_bounds__(kShadeBX* kShadeBY) k_shade(GbufDev g, CamDev cam, const float4* __restrict__ lights,
                                                              int NL, IblDev ibl, ShadeDev p, void* hdr,
                                                              long long hdr_pitch, uint8_t* ldr, long long ldr_pitch) {
  __shared__ float4 s_lights[2 * kLightChunk];
  int tid = threadIdx.y * kShadeBX + threadIdx.x;
  bool staged = NL <= kLightChunk;
  if (staged && (p.flags & EPBR_SHADE_DIRECT)) {
    for (int q = tid; q < 2 * NL; q += kShadeBX * kShadeBY) s_lights[q] = __ldg(lights + q);
  }
  __syncthreads();
  int x = blockIdx.x * kShadeBX + threadIdx.x, y = blockIdx.y * kShadeBY + threadIdx.y;
  if (x >= g.W || y >= g.H) return;
  float3 c = shade_pixel<FMT>(g, cam, s_lights, NL, lights, ibl, p, x, y, staged);
  if (hdr) store_hdr<HDR>(hdr, hdr_pitch, x, y, c);
  if (LDR) {
    unsigned v = pack_rgba8(c, p.exposure, p.op);
    ((unsigned*)(ldr + (size_t)y * ldr_pitch))[x] = v;
  }
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
static void launch_shade(dim3 grd, dim3 blk, cudaStream_t s, const GbufDev& g, const CamDev& c, const float4* L,
                         int NL, const IblDev& ibl, const ShadeDev& p, void* hdr, long long hp, uint8_t* ldr,
                         long long lp) {
  if (ldr)
    k_shade<FMT, HDR, true><<<grd, blk, 0, s>>>(g, c, L, NL, ibl, p, hdr, hp, ldr, lp);
  else
    k_shade<FMT, HDR, false><<<grd, blk, 0, s>>>(g, c, L, NL, ibl, p, hdr, hp, ldr, lp);
}

static epbr_status shade_common(const epbr_gbuffer* g, const epbr_camera* cam, const epbr_light* lights,
                                int32_t NL, const epbr_ibl* ibl, const epbr_shade_params* sp, void* hdr,
                                int32_t hdr_format, int64_t hdr_pitch, const epbr_tonemap_params* tp,
                                uint8_t* ldr, int64_t ldr_pitch, void* stream) {
  epbr_status st = validate_gbuffer(g, true);
  if (st) return st;
  if ((st = validate_camera(cam, g))) return st;
  if (!sp) return fail(EPBR_ERR_INVALID_ARG, "shade params is NULL");
  if (sp->flags & ~(unsigned)(EPBR_SHADE_DIRECT | EPBR_SHADE_IBL | EPBR_SHADE_MULTISCATTER | EPBR_SHADE_DIFFUSE_ONLY))
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
  dim3 blk(kShadeBX, kShadeBY), grd((g->width + kShadeBX - 1) / kShadeBX, (g->height + kShadeBY - 1) / kShadeBY);
  cudaStream_t s = (cudaStream_t)stream;
  const float4* L = (const float4*)lights;
  int nl = (sp->flags & EPBR_SHADE_DIRECT) ? NL : 0;
  if (g->format == EPBR_GBUFFER_FP32) {
    if (hdr_format == EPBR_HDR_RGBA32F)
      launch_shade<EPBR_GBUFFER_FP32, EPBR_HDR_RGBA32F>(grd, blk, s, gd, cd, L, nl, ib, p, hdr, hdr_pitch, ldr, ldr_pitch);
    else
      launch_shade<EPBR_GBUFFER_FP32, EPBR_HDR_RGBA16F>(grd, blk, s, gd, cd, L, nl, ib, p, hdr, hdr_pitch, ldr, ldr_pitch);
  } else {
    if (hdr_format == EPBR_HDR_RGBA32F)
      launch_shade<EPBR_GBUFFER_COMPACT, EPBR_HDR_RGBA32F>(grd, blk, s, gd, cd, L, nl, ib, p, hdr, hdr_pitch, ldr, ldr_pitch);
    else
      launch_shade<EPBR_GBUFFER_COMPACT, EPBR_HDR_RGBA16F>(grd, blk, s, gd, cd, L, nl, ib, p, hdr, hdr_pitch, ldr, ldr_pitch);
  }
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
