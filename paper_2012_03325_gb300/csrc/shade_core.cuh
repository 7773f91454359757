// Per-pixel compose as device functions, shared by the per-view kernel (shade.cu) and the fused
// multi-view kernel (batch.cu):
//   px_setup     G-buffer decode (Table 1 layouts), position from depth (Sec. 4), material terms
//   px_direct    Cook-Torrance over a chunk of point lights staged in shared memory (Sec. 3,
//                Eq. 1 with the UE4 model)
//   px_ambient   split-sum IBL with multiple-scattering compensation, times AO (Sec. 3.1)
//   tonemap      ACES / Reinhard + sRGB transfer (Sec. 5.4)
//
// Direct-light arithmetic avoids normalising the half vector: with s = l + v,
//   n.h = n.s / |s|,  1 - (n.h)^2 = |n x s|^2 / |s|^2,  |s|^2 = 2 + 2 l.v,  v.h = |s| / 2,
// so D = alpha^2 |s|^4 / (pi ((n.s)^2 alpha^2 + |n x s|^2)^2): the GGX distribution written
// without the 1 - (n.h)^2 cancellation that loses all precision at alpha^2 ~ 4e-6.  The light
// loop is branch-free: n.l is clamped at 0, which makes the contribution of a light below the
// horizon exactly 0 (every factor stays finite), as Eq. 1 integrates only n.l > 0.
#pragma once

#include "epbr_internal.cuh"

namespace epbr {

__constant__ float c_srgb8[256] = {
#include "srgb8_table.inc"
};

constexpr int kLightChunk = 256;
#ifndef EPBR_LIGHT_UNROLL
#define EPBR_LIGHT_UNROLL 8
#endif
constexpr int kLightUnroll = EPBR_LIGHT_UNROLL;  // light-loop unrolling of the monochrome loop

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
  float y = (op == EPBR_TONEMAP_REINHARD) ? x * rcp_ftz(1.0f + x)
                                          : x * fmaf(2.51f, x, 0.03f) * rcp_ftz(fmaf(x, fmaf(2.43f, x, 0.59f), 0.14f));
  y = clamp01(y);
  // y^(1/2.4) as 2^(log2(y) / 2.4) (relative error ~1e-6, i.e. < 3e-4 of an 8-bit step)
  float s = y <= 0.0031308f ? 12.92f * y : fmaf(1.055f, ex2_ftz(lg2_ftz(y) * (1.0f / 2.4f)), -0.055f);
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

// State of one pixel through the compose.
struct Px {
  float3 P, n, v, albedo, acc;
  float nv_raw, nv, metal, rough;
  bool surface;
};

// Raw G-buffer texel of one pixel, loaded before it is decoded (lets the loads of a block be in
// flight while its lights are staged).
struct PxRaw {
  float e;
  float4 a, b;  // FP32: rt0, rt1.  COMPACT: a.x = rt0 bits, a.y = rt1 bits, a.z = rt2 bits
};

template <int FMT>
__device__ __forceinline__ PxRaw px_load(const GbufDev& g, int x, int y) {
  PxRaw r;
  r.e = gb_depth(g, x, y);
  if (FMT == EPBR_GBUFFER_FP32) {
    r.a = __ldg((const float4*)(g.rt[0] + (size_t)y * g.pitch[0]) + x);
    r.b = __ldg((const float4*)(g.rt[1] + (size_t)y * g.pitch[1]) + x);
  } else {
    r.a.x = __uint_as_float(__ldg((const unsigned*)(g.rt[0] + (size_t)y * g.pitch[0]) + x));
    r.a.y = __uint_as_float(__ldg((const unsigned*)(g.rt[1] + (size_t)y * g.pitch[1]) + x));
    r.a.z = __uint_as_float((unsigned)__ldg((const unsigned short*)(g.rt[2] + (size_t)y * g.pitch[2]) + x));
  }
  return r;
}

template <int FMT>
__device__ __forceinline__ Px px_decode(const PxRaw& r, const CamDev& cam, int x, int y) {
  Px s;
  float3 dw = rot(cam, view_ray(cam, x, y));
  s.acc = f3(0, 0, 0);
  s.surface = is_surface(r.e);
  s.v = dw * -rsqrt_ftz(dot3(dw, dw));  // v = (eye - P) / |eye - P| with P = eye + e * dw
  if (!s.surface) {
    s.P = dw;  // background: keep the view ray for the environment lookup
    return s;
  }
  s.P = f3(cam.eye[0], cam.eye[1], cam.eye[2]) + r.e * dw;
  if (FMT == EPBR_GBUFFER_FP32) {
    s.n = normalize3(xyz(r.b));
    s.albedo = xyz(r.a);
    s.metal = r.a.w;
    s.rough = r.b.w;
  } else {
    unsigned a = __float_as_uint(r.a.x), nb = __float_as_uint(r.a.y), mr = __float_as_uint(r.a.z);
    s.n = oct_decode(*reinterpret_cast<const __half2*>(&nb));
    s.albedo = f3(c_srgb8[a & 255u], c_srgb8[(a >> 8) & 255u], c_srgb8[(a >> 16) & 255u]);
    s.metal = (mr & 255u) * (1.0f / 255.0f);
    s.rough = (mr >> 8) * (1.0f / 255.0f);
  }
  s.metal = clamp01(s.metal);
  s.rough = fminf(fmaxf(s.rough, kRoughMin), 1.0f);
  s.nv_raw = dot3(s.n, s.v);
  s.nv = fmaxf(s.nv_raw, kNvMin);
  return s;
}

template <int FMT>
__device__ __forceinline__ Px px_setup(const GbufDev& g, const CamDev& cam, int x, int y) {
  return px_decode<FMT>(px_load<FMT>(g, x, y), cam, x, y);
}

// Lights staged in shared memory as pairs (pos.xyz, Ic.r), (Ic.rgb, -) with Ic = intensity *
// colour, so a monochrome light needs only the first float4.  Returns
// whether every light this thread staged is monochrome (equal colour channels); callers combine
// the flags with __syncthreads_and to pick the monochrome loop for the chunk.
__device__ __forceinline__ bool stage_lights(float4* s_lights, const float4* __restrict__ lights, int first,
                                             int cnt, int tid, int nthreads) {
  bool mono = true;
  for (int q = tid; q < cnt; q += nthreads) {
    float4 a = __ldg(lights + 2 * (first + q));
    float4 c = __ldg(lights + 2 * (first + q) + 1);
    float4 ic = make_float4(a.w * c.x, a.w * c.y, a.w * c.z, 0.0f);
    s_lights[2 * q] = make_float4(a.x, a.y, a.z, ic.x);  // .w: Ic of a monochrome light
    s_lights[2 * q + 1] = ic;
    mono = mono && ic.x == ic.y && ic.y == ic.z;
  }
  return mono;
}

// Direct light of one pixel, accumulated over chunks of staged lights.  With
//   F_c = F0_c + (1 - F0_c) fc,  1 - F_c = (1 - F0_c)(1 - fc),
// the contribution w Ic_c [cdiff_c/pi (1 - F_c) + spec F_c] of a light (w = (n.l)/d^2) is
//   Ic_c [K_c (w (1 - fc)) + F0_c (w spec) + (1 - F0_c)(w spec fc)],  K_c = cdiff_c/pi (1 - F0_c),
// so the loop keeps three sums per channel of Ic_c times light scalars and the per-channel
// material factors are applied once per pixel (px_direct_end).  spec is accumulated without
// its per-pixel factor alpha^2 G1(v) / (4 pi n.v), applied at the end as well.  For a chunk of
// monochrome lights (Ic_r = Ic_g = Ic_b) the three channels share one sum each.
struct Direct {
  float3 sa, sb, sbf;  // sums of Ic w (1 - fc), Ic w spec', Ic w spec' fc
  float3 nxv;          // n x v: n x (l + v) = (n x L) / |L| + n x v
  float a2vv, alpha, nva, k, omk;  // nva = alpha n.v: alpha (n.l + n.v) = fma(n.l, alpha, nva)
};

__device__ __forceinline__ Direct px_direct_begin(const Px& s) {
  Direct d;
  d.sa = d.sb = d.sbf = f3(0, 0, 0);
  float alpha = s.rough * s.rough;
  d.alpha = alpha;
  d.nva = alpha * s.nv_raw;
  d.k = (s.rough + 1.0f) * (s.rough + 1.0f) * 0.125f;
  d.omk = 1.0f - d.k;
  d.a2vv = alpha * alpha * rcp_ftz(4.0f * kPi * fmaf(s.nv, d.omk, d.k));  // alpha^2 G1(v) / (4 pi n.v)
  d.nxv = cross3(s.n, s.v);
  return d;
}

// Scalar light terms shared by both loops.  Guards are folded into existing FMAs: |L|^2 + 1e-30
// (a light at P contributes 0), |n x s|^2 + 1e-18 (keeps the GGX denominator normal when
// l = -v), and |l + v|^2 biased by 1e-6 (>= 0 under rounding); each changes a result by less
// than 1e-12 relative.
struct LightTerms {
  float a, b, bf;
};

__device__ __forceinline__ LightTerms light_terms(const Px& s, const Direct& d, float4 lp) {
  float3 L = xyz(lp) - s.P;
  float d2 = fmaf(L.x, L.x, fmaf(L.y, L.y, fmaf(L.z, L.z, 1e-30f)));
  float rs = rsqrt_ftz(d2);
  float3 l = L * rs;
  float nl = dot3(s.n, l);
  float nlc = fmaxf(nl, 0.0f);
  float lv = dot3(s.v, l);
  // n x (l + v) = n x l + n x v, accumulated onto the per-pixel n x v
  float3 c = f3(fmaf(s.n.y, l.z, fmaf(-s.n.z, l.y, d.nxv.x)), fmaf(s.n.z, l.x, fmaf(-s.n.x, l.z, d.nxv.y)),
                fmaf(s.n.x, l.y, fmaf(-s.n.y, l.x, d.nxv.z)));
  float c2 = fmaf(c.x, c.x, fmaf(c.y, c.y, fmaf(c.z, c.z, 1e-18f)));
  float nsa = fmaf(nl, d.alpha, d.nva);  // alpha n.(l + v)
  float hh = fmaf(2.0f, lv, 2.000001f);  // |l + v|^2
  float den = fmaf(nsa, nsa, c2);
  float xx = fmaf(-0.5f, sqrt_ftz(hh), 1.0f);  // 1 - v.h, v.h = |l + v| / 2
#ifdef EPBR_FC_POW5
  float x2 = xx * xx, fc = x2 * x2 * xx;
#else
  float fc = ex2_ftz(5.0f * lg2_ftz(fabsf(xx)));  // (1 - v.h)^5 (|xx|: v.h may round above 1)
#endif
  float w = rs * rs * nlc;  // (n.l) / d^2
  float spec = hh * hh * rcp_ftz(den * den * fmaf(nlc, d.omk, d.k));
  LightTerms t;
  t.a = fmaf(-w, fc, w);
  t.b = w * spec;
  t.bf = t.b * fc;
  return t;
}

// Adds `cnt` staged lights with arbitrary colours.
__device__ __forceinline__ void px_direct(const Px& s, Direct& d, const float4* s_lights, int cnt) {
  float3 sa = d.sa, sb = d.sb, sbf = d.sbf;
#pragma unroll 4
  for (int i = 0; i < cnt; ++i) {
    float4 lc = s_lights[2 * i + 1];
    LightTerms t = light_terms(s, d, s_lights[2 * i]);
    sa.x = fmaf(lc.x, t.a, sa.x);
    sa.y = fmaf(lc.y, t.a, sa.y);
    sa.z = fmaf(lc.z, t.a, sa.z);
    sb.x = fmaf(lc.x, t.b, sb.x);
    sb.y = fmaf(lc.y, t.b, sb.y);
    sb.z = fmaf(lc.z, t.b, sb.z);
    sbf.x = fmaf(lc.x, t.bf, sbf.x);
    sbf.y = fmaf(lc.y, t.bf, sbf.y);
    sbf.z = fmaf(lc.z, t.bf, sbf.z);
  }
  d.sa = sa;
  d.sb = sb;
  d.sbf = sbf;
}

// Adds `cnt` staged monochrome lights (Ic_r = Ic_g = Ic_b).
__device__ __forceinline__ void px_direct_mono(const Px& s, Direct& d, const float4* s_lights, int cnt) {
  float sa = 0.0f, sb = 0.0f, sbf = 0.0f;
#pragma unroll(kLightUnroll)
  for (int i = 0; i < cnt; ++i) {
    float4 lp = s_lights[2 * i];
    float ic = lp.w;
    LightTerms t = light_terms(s, d, lp);
    sa = fmaf(ic, t.a, sa);
    sb = fmaf(ic, t.b, sb);
    sbf = fmaf(ic, t.bf, sbf);
  }
  d.sa = d.sa + f3(sa, sa, sa);
  d.sb = d.sb + f3(sb, sb, sb);
  d.sbf = d.sbf + f3(sbf, sbf, sbf);
}

__device__ __forceinline__ void px_direct_end(Px& s, const Direct& d) {
  float3 F0 = f3(fmaf(s.metal, s.albedo.x - 0.04f, 0.04f), fmaf(s.metal, s.albedo.y - 0.04f, 0.04f),
                 fmaf(s.metal, s.albedo.z - 0.04f, 0.04f));
  float3 omF0 = f3(1.0f - F0.x, 1.0f - F0.y, 1.0f - F0.z);
  float3 K = mul3(s.albedo * ((1.0f - s.metal) * kInvPi), omF0);
  float3 sb = d.sb * d.a2vv, sbf = d.sbf * d.a2vv;
  s.acc.x += fmaf(K.x, d.sa.x, fmaf(F0.x, sb.x, omF0.x * sbf.x));
  s.acc.y += fmaf(K.y, d.sa.y, fmaf(F0.y, sb.y, omF0.y * sbf.y));
  s.acc.z += fmaf(K.z, d.sa.z, fmaf(F0.z, sb.z, omF0.z * sbf.z));
}

// Diffuse-only variant: sum of Ic (n.l)/d^2, times albedo/pi at the end.
__device__ __forceinline__ void px_direct_diffuse(const Px& s, Direct& d, const float4* s_lights, int cnt) {
  float3 sa = d.sa;
#pragma unroll 4
  for (int i = 0; i < cnt; ++i) {
    float4 lp = s_lights[2 * i], lc = s_lights[2 * i + 1];
    float3 L = xyz(lp) - s.P;
    float rs = rsqrt_ftz(fmaf(L.x, L.x, fmaf(L.y, L.y, fmaf(L.z, L.z, 1e-30f))));
    float w = rs * rs * fmaxf(dot3(s.n, L) * rs, 0.0f);
    sa.x = fmaf(lc.x, w, sa.x);
    sa.y = fmaf(lc.y, w, sa.y);
    sa.z = fmaf(lc.z, w, sa.z);
  }
  d.sa = sa;
}

__device__ __forceinline__ void px_direct_diffuse_end(Px& s, const Direct& d) {
  s.acc = s.acc + mul3(s.albedo * kInvPi, d.sa);
}

// Adds the split-sum ambient term (times AO) to s.acc.
__device__ __forceinline__ void px_ambient(Px& s, const IblDev& ibl, unsigned flags, float ao) {
  float3 irr = equirect_lookup(ibl.irr, s.n);
  if (flags & EPBR_SHADE_DIFFUSE_ONLY) {
    s.acc = s.acc + mul3(s.albedo, irr) * ao;
    return;
  }
  float3 F0 = f3(fmaf(s.metal, s.albedo.x - 0.04f, 0.04f), fmaf(s.metal, s.albedo.y - 0.04f, 0.04f),
                 fmaf(s.metal, s.albedo.z - 0.04f, 0.04f));
  float3 cdiff = s.albedo * (1.0f - s.metal);
  float3 R = s.n * (2.0f * s.nv_raw) - s.v;
  float lod = s.rough * (float)(ibl.M - 1);
  int l0 = min((int)floorf(lod), ibl.M - 1);
  int l1 = min(l0 + 1, ibl.M - 1);
  float tl = lod - (float)l0;
  float u, vv;
  dir_to_uv(R, u, vv);
  float3 p0 = equirect_bilinear(ibl.lev[l0], u, vv);
  float3 p1 = equirect_bilinear(ibl.lev[l1], u, vv);
  float3 pref = p0 + tl * (p1 - p0);
  float2 AB = lut_bilinear(ibl.lut, ibl.S, clamp01(s.nv), s.rough);
  float xv = 1.0f - s.nv, xv2 = xv * xv, fcv = xv2 * xv2 * xv;
  float Fr_base = 1.0f - s.rough;
  float F0a[3] = {F0.x, F0.y, F0.z}, cd[3] = {cdiff.x, cdiff.y, cdiff.z};
  float pr[3] = {pref.x, pref.y, pref.z}, ir[3] = {irr.x, irr.y, irr.z}, la[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float Fr = fmaxf(Fr_base, F0a[q]) - F0a[q];
    float kS = fmaf(Fr, fcv, F0a[q]);
    if (flags & EPBR_SHADE_MULTISCATTER) {
      // Fdez-Aguera 2019: single-scatter energy plus the series of further bounces
      float FssEss = fmaf(kS, AB.x, AB.y);
      float Ess = AB.x + AB.y, Ems = 1.0f - Ess;
      float Favg = F0a[q] + (1.0f - F0a[q]) * (1.0f / 21.0f);
      float Fms = FssEss * Favg * rcp_ftz(fmaf(-Ems, Favg, 1.0f));
      float kD = cd[q] * (1.0f - FssEss - Fms * Ems);
      la[q] = fmaf(FssEss, pr[q], (Fms * Ems + kD) * ir[q]);
    } else {
      la[q] = fmaf((1.0f - kS) * cd[q], ir[q], fmaf(kS, AB.x, AB.y) * pr[q]);
    }
  }
  s.acc = s.acc + f3(la[0], la[1], la[2]) * ao;
}

// Final radiance of a pixel after px_direct: ambient, or the environment for background.
__device__ __forceinline__ float3 px_finish(Px& s, const IblDev& ibl, unsigned flags, float ao) {
  if (!s.surface) return (flags & EPBR_SHADE_IBL) ? equirect_lookup(ibl.lev[0], s.P) : f3(0, 0, 0);
  if (flags & EPBR_SHADE_IBL) px_ambient(s, ibl, flags, ao);
  return s.acc;
}

}  // namespace epbr
