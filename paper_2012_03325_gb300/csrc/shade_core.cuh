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
  float ao_inv;  // 1 / ao_scale
  const float* ao;
  long long ao_pitch;
  float exposure;
  int op;
};

// AO texel of pixel (x, y): texel (floor(x / scale), floor(y / scale)), the quotients taken as
// floor((x + 1/2) / scale) in FP32, exact for x < 2^15 and scale <= 8 (the fraction stays at
// least 1/16 away from an integer while the rounding error is below 2^-8).
__device__ __forceinline__ float ao_at(const ShadeDev& p, int x, int y) {
  if (!p.ao) return 1.0f;
  int ax = __float2int_rd(((float)x + 0.5f) * p.ao_inv), ay = __float2int_rd(((float)y + 0.5f) * p.ao_inv);
  return __ldg((const float*)((const char*)p.ao + (size_t)ay * p.ao_pitch) + ax);
}

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
// the flags with __syncthreads_and to pick the monochrome loop for the chunk.  With s_dup, each
// light is also written as (x, x, y, y), (z, z, Ic, Ic): the operands of the two-pixel packed
// loop (px_direct_mono2), each coordinate already duplicated into both halves of a pair.
// FROM_SMEM: `lights` is a copy of the list in shared memory (staged by a TMA bulk copy).
template <bool FROM_SMEM = false>
__device__ __forceinline__ bool stage_lights(float4* s_lights, const float4* __restrict__ lights, int first,
                                             int cnt, int tid, int nthreads, float4* s_dup = nullptr) {
  bool mono = true;
  for (int q = tid; q < cnt; q += nthreads) {
    float4 a = FROM_SMEM ? lights[2 * (first + q)] : __ldg(lights + 2 * (first + q));
    float4 c = FROM_SMEM ? lights[2 * (first + q) + 1] : __ldg(lights + 2 * (first + q) + 1);
    float4 ic = make_float4(a.w * c.x, a.w * c.y, a.w * c.z, 0.0f);
    s_lights[2 * q] = make_float4(a.x, a.y, a.z, ic.x);  // .w: Ic of a monochrome light
    s_lights[2 * q + 1] = ic;
    if (s_dup) {
      s_dup[2 * q] = make_float4(a.x, a.x, a.y, a.y);
      s_dup[2 * q + 1] = make_float4(a.z, a.z, ic.x, ic.x);
    }
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
  return d;
}

// Scalar light terms shared by both loops.  Guards are folded into existing FMAs: |L|^2 + 1e-30
// (a light at P contributes 0) and |n x s|^2 + 1e-18 (keeps the GGX denominator normal when
// l = -v) change a result by < 1e-12 relative.  The half vector s = l + v is formed explicitly,
// so |s|^2 is a sum of squares (never negative) and needs no bias, also for a light behind a
// grazing view (l ~ -v, where 2 + 2 l.v would cancel).
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
  float3 h = f3(fmaf(L.x, rs, s.v.x), fmaf(L.y, rs, s.v.y), fmaf(L.z, rs, s.v.z));  // s = l + v
  float3 c = cross3(s.n, h);                                                        // n x s
  float c2 = fmaf(c.x, c.x, fmaf(c.y, c.y, fmaf(c.z, c.z, 1e-18f)));
  float nsa = fmaf(nl, d.alpha, d.nva);  // alpha n.(l + v)
  float hh = fmaf(h.x, h.x, fmaf(h.y, h.y, h.z * h.z));  // |s|^2
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

// alpha^2 G1(v) / (4 pi n.v): the per-pixel factor of the specular sums.
__device__ __forceinline__ float spec_factor(const Px& s) {
  float alpha = s.rough * s.rough, k = (s.rough + 1.0f) * (s.rough + 1.0f) * 0.125f;
  return alpha * alpha * rcp_ftz(4.0f * kPi * fmaf(s.nv, 1.0f - k, k));
}

// Adds K sa + F0 sb a2vv + (1 - F0) sbf a2vv to s.acc (the per-channel material factors of the
// three light sums).
__device__ __forceinline__ void px_direct_fold(Px& s, float3 sa, float3 sb, float3 sbf, float a2vv) {
  float3 F0 = f3(fmaf(s.metal, s.albedo.x - 0.04f, 0.04f), fmaf(s.metal, s.albedo.y - 0.04f, 0.04f),
                 fmaf(s.metal, s.albedo.z - 0.04f, 0.04f));
  float3 omF0 = f3(1.0f - F0.x, 1.0f - F0.y, 1.0f - F0.z);
  float3 K = mul3(s.albedo * ((1.0f - s.metal) * kInvPi), omF0);
  sb = sb * a2vv;
  sbf = sbf * a2vv;
  s.acc.x += fmaf(K.x, sa.x, fmaf(F0.x, sb.x, omF0.x * sbf.x));
  s.acc.y += fmaf(K.y, sa.y, fmaf(F0.y, sb.y, omF0.y * sbf.y));
  s.acc.z += fmaf(K.z, sa.z, fmaf(F0.z, sb.z, omF0.z * sbf.z));
}

__device__ __forceinline__ void px_direct_end(Px& s, const Direct& d) { px_direct_fold(s, d.sa, d.sb, d.sbf, d.a2vv); }

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

// ---- Two pixels per thread: the monochrome light loop in packed FP32x2 instructions ----------
//
// Each thread shades two pixels; every per-pixel quantity of the light loop is a float2 whose
// halves belong to the two pixels, and each arithmetic step is one fma/mul/add.f32x2 for both.
// The loop runs in a per-pixel tangent frame (t, b, n) (Duff et al. ONB around n), where with
// L = R (p_light - P) = R p_light + q (q = -R P) and v = (v_t, v_b, n.v):
//   n.L = L_z,  s = L / |L| + v,  |n x s|^2 = s_x^2 + s_y^2,  n.s = s_z,  |s|^2 = |n x s|^2 + s_z^2,
// i.e. the quantities of the direct-light terms above without any cross or dot product per light.
// The loop keeps four sums per pixel: Ic w, Ic w fc, Ic w spec', Ic w spec' fc, so
// sa = (Ic w) - (Ic w fc), sb = Ic w spec', sbf = Ic w spec' fc of the scalar loop.

__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Per-pixel constants of the packed loop for two pixels.
struct Frame2 {
  float2 tx, ty, tz, bx, by, bz, nx, ny, nz;  // rows of R = (t; b; n)
  float2 qx, qy, qz;                          // q = -R P
  float2 vx, vy, vz;                          // R v
  float2 al, k, omk;                          // alpha, Smith-Schlick k, 1 - k
};

struct Sums2 {
  float2 w, wf, b, bf;  // sums of Ic w, Ic w fc, Ic w spec', Ic w spec' fc
};

struct FrameHalf {
  float t[3], b[3], n[3], q[3], v[3], al, k, omk;
};

__device__ __forceinline__ FrameHalf frame_half(const Px& s, bool active) {
  FrameHalf h;
  if (!active) {  // an inactive half computes finite values that are never used
#pragma unroll
    for (int i = 0; i < 3; ++i) h.t[i] = h.b[i] = h.n[i] = h.q[i] = h.v[i] = 0.0f;
    h.al = h.k = h.omk = 1.0f;
    return h;
  }
  float3 t, b;
  onb(s.n, t, b);
  h.t[0] = t.x, h.t[1] = t.y, h.t[2] = t.z;
  h.b[0] = b.x, h.b[1] = b.y, h.b[2] = b.z;
  h.n[0] = s.n.x, h.n[1] = s.n.y, h.n[2] = s.n.z;
  h.q[0] = -dot3(t, s.P), h.q[1] = -dot3(b, s.P), h.q[2] = -dot3(s.n, s.P);
  h.v[0] = dot3(t, s.v), h.v[1] = dot3(b, s.v), h.v[2] = s.nv_raw;
  h.al = s.rough * s.rough;
  h.k = (s.rough + 1.0f) * (s.rough + 1.0f) * 0.125f;
  h.omk = 1.0f - h.k;
  return h;
}

__device__ __forceinline__ Frame2 make_frame2(const Px& s0, bool a0, const Px& s1, bool a1) {
  FrameHalf h0 = frame_half(s0, a0), h1 = frame_half(s1, a1);
  Frame2 f;
  f.tx = make_float2(h0.t[0], h1.t[0]), f.ty = make_float2(h0.t[1], h1.t[1]), f.tz = make_float2(h0.t[2], h1.t[2]);
  f.bx = make_float2(h0.b[0], h1.b[0]), f.by = make_float2(h0.b[1], h1.b[1]), f.bz = make_float2(h0.b[2], h1.b[2]);
  f.nx = make_float2(h0.n[0], h1.n[0]), f.ny = make_float2(h0.n[1], h1.n[1]), f.nz = make_float2(h0.n[2], h1.n[2]);
  f.qx = make_float2(h0.q[0], h1.q[0]), f.qy = make_float2(h0.q[1], h1.q[1]), f.qz = make_float2(h0.q[2], h1.q[2]);
  f.vx = make_float2(h0.v[0], h1.v[0]), f.vy = make_float2(h0.v[1], h1.v[1]), f.vz = make_float2(h0.v[2], h1.v[2]);
  f.al = make_float2(h0.al, h1.al), f.k = make_float2(h0.k, h1.k), f.omk = make_float2(h0.omk, h1.omk);
  return f;
}

// Adds `cnt` monochrome lights staged as (x, x, y, y), (z, z, Ic, Ic) to the sums of both pixels.
// Guards as in light_terms: |L|^2 + 1e-30, |n x s|^2 + 1e-18.
__device__ __forceinline__ void px_direct_mono2(const Frame2& f, Sums2& S, const float4* s_dup, int cnt) {
  float2 sw = S.w, swf = S.wf, sb = S.b, sbf = S.bf;
  const float2 e30 = dup2(1e-30f), e18 = dup2(1e-18f), mhalf = dup2(-0.5f), one = dup2(1.0f);
#pragma unroll(kLightUnroll)
  for (int i = 0; i < cnt; ++i) {
    float4 u = s_dup[2 * i], z = s_dup[2 * i + 1];
    float2 X = make_float2(u.x, u.y), Y = make_float2(u.z, u.w), Z = make_float2(z.x, z.y), IC = make_float2(z.z, z.w);
    float2 Lx = pfma(f.tx, X, pfma(f.ty, Y, pfma(f.tz, Z, f.qx)));
    float2 Ly = pfma(f.bx, X, pfma(f.by, Y, pfma(f.bz, Z, f.qy)));
    float2 Lz = pfma(f.nx, X, pfma(f.ny, Y, pfma(f.nz, Z, f.qz)));
    float2 d2 = pfma(Lx, Lx, pfma(Ly, Ly, pfma(Lz, Lz, e30)));
    float2 rs = make_float2(rsqrt_ftz(d2.x), rsqrt_ftz(d2.y));
    float2 sx = pfma(Lx, rs, f.vx), sy = pfma(Ly, rs, f.vy), sz = pfma(Lz, rs, f.vz);
    float2 c2 = pfma(sx, sx, pfma(sy, sy, e18));  // |n x s|^2
    float2 hh = pfma(sz, sz, c2);                 // |s|^2
    float2 nsa = pmul(sz, f.al);                  // alpha n.s
    float2 den = pfma(nsa, nsa, c2);
    float2 nlc = pmul(make_float2(fmaxf(Lz.x, 0.0f), fmaxf(Lz.y, 0.0f)), rs);  // max(n.l, 0)
    float2 xx = pfma(mhalf, make_float2(sqrt_ftz(hh.x), sqrt_ftz(hh.y)), one);  // 1 - v.h
    float2 x2 = pmul(xx, xx);
    float2 fc = pmul(pmul(x2, x2), xx);  // (1 - v.h)^5 in the FMA pipe (as ex2(5 lg2) the MUFU pipe would be the bound)
    // Ic (n.l) / d^2, with 1 / d^2 from the MUFU pipe (which has room here) instead of rs * rs
    float2 icw = pmul(pmul(IC, make_float2(rcp_ftz(d2.x), rcp_ftz(d2.y))), nlc);
    float2 q = pmul(pmul(den, den), pfma(nlc, f.omk, f.k));
    float2 icb = pmul(icw, pmul(pmul(hh, hh), make_float2(rcp_ftz(q.x), rcp_ftz(q.y))));
    sw = padd(sw, icw);
    swf = pfma(icw, fc, swf);
    sb = padd(sb, icb);
    sbf = pfma(icb, fc, sbf);
  }
  S.w = sw, S.wf = swf, S.b = sb, S.bf = sbf;
}

// Folds half `h` (0 or 1) of the packed sums into pixel s.
__device__ __forceinline__ void px_direct_fold2(Px& s, const Sums2& S, int h) {
  float w = h ? S.w.y : S.w.x, wf = h ? S.wf.y : S.wf.x, b = h ? S.b.y : S.b.x, bf = h ? S.bf.y : S.bf.x;
  float sa = w - wf;
  px_direct_fold(s, f3(sa, sa, sa), f3(b, b, b), f3(bf, bf, bf), spec_factor(s));
}

// Direct light of a pixel pair summed over all NL lights, in chunks of `chunk` lights staged in
// shared memory (s_lights, and s_dup for the packed loop).  With `prestaged` the block has staged
// all lights already (NL <= chunk) and `mono` is their block vote; otherwise every chunk is staged
// here, so every thread of the block must call this with the same NL, chunk and prestaged.
// Monochrome chunks take the packed loop; other chunks, and the diffuse-only mode, the per-pixel
// loops, whose sums are folded into s[h].acc chunk by chunk.
__device__ __forceinline__ void shade_lights(Px (&s)[2], const bool (&act)[2], int NL, unsigned flags,
                                             const float4* __restrict__ lights, float4* s_lights, float4* s_dup,
                                             int chunk, bool prestaged, bool mono, int tid, int nthreads) {
  const bool diffuse_only = (flags & EPBR_SHADE_DIFFUSE_ONLY) != 0;
  Frame2 fr;
  Sums2 sums;
  sums.w = sums.wf = sums.b = sums.bf = make_float2(0.0f, 0.0f);
  if (NL > 0 && !diffuse_only && (act[0] || act[1])) fr = make_frame2(s[0], act[0], s[1], act[1]);
  for (int base = 0; base < NL; base += chunk) {
    int cnt = prestaged ? NL : min(chunk, NL - base);
    bool m = mono;
    if (!prestaged) {
      __syncthreads();  // the previous chunk has been read by every thread
      m = __syncthreads_and(stage_lights(s_lights, lights, base, cnt, tid, nthreads, s_dup));
    }
    if (!(act[0] || act[1])) continue;
    if (!diffuse_only && m) {
      px_direct_mono2(fr, sums, s_dup, cnt);
      continue;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!act[h]) continue;
      Direct d = px_direct_begin(s[h]);
      if (diffuse_only) {
        px_direct_diffuse(s[h], d, s_lights, cnt);
        px_direct_diffuse_end(s[h], d);
      } else {
        px_direct(s[h], d, s_lights, cnt);
        px_direct_end(s[h], d);
      }
    }
  }
  if (NL > 0 && !diffuse_only) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (act[h]) px_direct_fold2(s[h], sums, h);
  }
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

// Host: launches the shadowed compose (shadow.cu) after shade.cu has validated the common
// arguments; validates `shadows`.
epbr_status launch_shade_shadows(const GbufDev& g, const CamDev& c, int fmt, const float4* L, int NL,
                                 const IblDev& ibl, const ShadeDev& p, const epbr_shadows* shadows, void* hdr,
                                 int hdr_format, long long hp, uint8_t* ldr, long long lp, cudaStream_t st);

}  // namespace epbr
