// SSAO per-texel arithmetic (paper Sec. 5.2, normal-oriented hemisphere of Bavoil & Sainz
// 2008): ssao_texel is the one-texel form of the fused multi-view kernel (batch.cu), which the
// per-view k_ssao_raw (ssao.cu) restates for two texels in packed arithmetic; the blur is shared.
#pragma once

#include "epbr_internal.cuh"

namespace epbr {

constexpr int kMaxSsaoSamples = 256;
#ifndef EPBR_SSAO_UNROLL
#define EPBR_SSAO_UNROLL 8
#endif
constexpr int kSsaoUnroll = EPBR_SSAO_UNROLL;  // samples whose depth taps are in flight together

struct SsaoDev {
  int K, scale, R;
  float radius, bias, sigma_s, sigma_z;
  const float4* kernel;
  const float2* noise;
  float inv_k;    // 1 / K
  float blur_ks;  // -log2(e) / (2 sigma_s^2): the spatial exponent per squared texel distance
};

__host__ inline SsaoDev make_ssao(const epbr_ssao_params& p) {
  SsaoDev d;
  d.K = p.num_samples;
  d.scale = p.scale;
  d.R = p.blur_radius;
  d.radius = p.radius;
  d.bias = p.bias;
  d.sigma_s = p.sigma_s;
  d.sigma_z = p.sigma_z;
  d.kernel = (const float4*)p.kernel;
  d.noise = (const float2*)p.noise;
  d.inv_k = (float)(1.0 / p.num_samples);
  d.blur_ks = (float)(-1.4426950408889634 / (2.0 * (double)p.sigma_s * (double)p.sigma_s));
  return d;
}

__device__ __forceinline__ float smoothstep01(float x) {
  x = clamp01(x);
  return x * x * (3.0f - 2.0f * x);
}

// Unblurred AO of AO texel (i, j), which uses full-resolution pixel (scale i, scale j), as
// (AO, depth of that pixel); background pixels (depth +inf) have AO 1.  `s_kernel` holds the K
// hemisphere offsets.
template <int FMT>
__device__ __forceinline__ float2 ssao_texel(const GbufDev& g, const CamDev& cam, const SsaoDev& p,
                                             const float4* s_kernel, int i, int j) {
  int X0 = p.scale * i, Y0 = p.scale * j;
  float e = gb_depth(g, X0, Y0);
  if (!is_surface(e)) return make_float2(1.0f, e);
  float3 P = e * view_ray(cam, X0, Y0);
  float3 n = rot_t(cam, gb_normal<FMT>(g, X0, Y0));
  float2 nz = __ldg(p.noise + ((j & 3) * 4 + (i & 3)));
  float3 rv = f3(nz.x, nz.y, 0.0f);
  float3 t = rv - n * dot3(rv, n), b;
  float tt = dot3(t, t);
  if (tt < 1e-8f) {  // |t| < 1e-4
    onb(n, t, b);
  } else {
    t = t * rsqrt_ftz(tt);
    b = cross3(n, t);
  }
  const float ix_scale = cam.ix_scale, iy_scale = cam.iy_scale, hw = 0.5f * cam.W, hh = 0.5f * cam.H;
  const float3 rt = t * p.radius, rb = b * p.radius, rn = n * p.radius;
  float occ = 0.0f;
  // Branch-free so that the depth taps of several samples are in flight together: an invalid
  // sample (behind the camera or off-screen) reads pixel (0, 0) and is masked out.  The pixel of
  // a sample is (floor(x), floor(y)); 0 <= x < W is tested as 0 <= floor(x) < W, one unsigned
  // compare (a negative or saturated conversion is out of range).
#pragma unroll(kSsaoUnroll)
  for (int k = 0; k < p.K; ++k) {
    float4 ks = s_kernel[k];
    float3 S = f3(fmaf(rt.x, ks.x, fmaf(rb.x, ks.y, fmaf(rn.x, ks.z, P.x))),
                  fmaf(rt.y, ks.x, fmaf(rb.y, ks.y, fmaf(rn.y, ks.z, P.y))),
                  fmaf(rt.z, ks.x, fmaf(rb.z, ks.y, fmaf(rn.z, ks.z, P.z))));
    float eS = -S.z;
    float inv = rcp_ftz(eS);
    int ix = __float2int_rd(fmaf(S.x * inv, ix_scale, hw));
    int iy = __float2int_rd(fmaf(-S.y * inv, iy_scale, hh));
    bool valid = eS > 0.0f && (unsigned)ix < (unsigned)cam.W && (unsigned)iy < (unsigned)cam.H;
    float eb = gb_depth(g, valid ? ix : 0, valid ? iy : 0);
    // eb <= eS - bias (finite) already excludes a background tap at +inf
    bool hit = valid && eb > 0.0f && eb <= eS - p.bias;
    occ += hit ? smoothstep01(p.radius * rcp_ftz(fabsf(e - eb))) : 0.0f;
  }
  return make_float2(fmaf(-occ, p.inv_k, 1.0f), e);
}

// Depth-aware blur of one AO texel from shared-memory tiles: `ao` and `ed` point at the
// centre texel inside row-major tiles of row pitch `tp` that hold R texels around it (taps
// outside the image staged as background: AO 0, depth +inf).  Weight
//   w = exp(-(dx^2 + dy^2) / (2 sigma_s^2)) * exp(-|e_q - e_p| / (sigma_z e_p))
// as one base-2 exponential; a background tap has |e_q - e_p| = +inf and so weight exactly 0.
// Background centre texels return 1.  RT > 0 fixes the radius at compile time (R = RT).
template <int RT>
__device__ __forceinline__ float ssao_blur_texel_r(const SsaoDev& p, const float* ao, const float* ed, int tp) {
  float ep = ed[0];
  if (!is_surface(ep)) return 1.0f;
  const int R = RT > 0 ? RT : p.R;
  const float ks = p.blur_ks;
  float kz = -1.4426950408889634f * rcp_ftz(p.sigma_z * ep);
  float num = 0.0f, den = 0.0f;
#pragma unroll
  for (int dy = -R; dy <= R; ++dy) {
    const float* ra = ao + dy * tp;
    const float* re = ed + dy * tp;
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      float w = ex2_ftz(fmaf(fabsf(re[dx] - ep), kz, (float)(dx * dx + dy * dy) * ks));
      num = fmaf(w, ra[dx], num);
      den += w;
    }
  }
  return num * rcp_ftz(den);  // den >= 1: the centre tap has weight 2^0
}

__device__ __forceinline__ float ssao_blur_texel(const SsaoDev& p, const float* ao, const float* ed, int tp) {
  return p.R == 3 ? ssao_blur_texel_r<3>(p, ao, ed, tp) : ssao_blur_texel_r<0>(p, ao, ed, tp);
}

}  // namespace epbr
