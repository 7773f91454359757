// Shadow maps with 3x3 percentage-closer filtering for the point lights (Sec. 5.1; Williams
// 1978, Reeves et al. 1987), evaluated inside the compose's light loop.
//   k_shade_shadow  one pixel per thread in 32x8 blocks, lights and their shadow cameras staged
//                   in shared memory in chunks of 128; per light the direct terms of Eq. 1 and,
//                   when the light reaches the pixel (n.l > 0), its PCF visibility: the fragment
//                   projected into the light's map and the 3x3 block of depths around its texel
//                   compared with z - b0 - b1 z.  Ambient, background and tone map as k_shade.
#include <cmath>

#include "shade_core.cuh"

namespace epbr {

constexpr int kShadowChunk = 128;

struct ShadowDev {
  const float* maps;
  const float4* cams;  // 4 float4 per light: rows 0..2 of world -> light view, (f, -, -, -)
  long long map_texels;  // S * S
  int S;
  float b0, b1;
};

// Lit share of the 3x3 block of map texels around the projection of P (a tap outside the map,
// or P behind the light, counts as lit).
__device__ __forceinline__ float shadow_visibility(const float4* cam, float3 P, const float* __restrict__ map, int S,
                                                   float b0, float b1) {
  float4 r0 = cam[0], r1 = cam[1], r2 = cam[2];
  float f = cam[3].x;
  float qx = fmaf(r0.x, P.x, fmaf(r0.y, P.y, fmaf(r0.z, P.z, r0.w)));
  float qy = fmaf(r1.x, P.x, fmaf(r1.y, P.y, fmaf(r1.z, P.z, r1.w)));
  float z = -fmaf(r2.x, P.x, fmaf(r2.y, P.y, fmaf(r2.z, P.z, r2.w)));
  if (!(z > 0.0f)) return 1.0f;
  float half = 0.5f * (float)S, k = f * rcp_ftz(z);
  float s = fmaf(qx * k, half, half), t = fmaf(-qy * k, half, half);
  if (!(fabsf(s) < 1e9f && fabsf(t) < 1e9f)) return 1.0f;  // far outside the frustum
  int i0 = __float2int_rd(s), j0 = __float2int_rd(t);
  float thr = fmaf(-b1, z, z) - b0;  // lit when d >= z - b1 z - b0
  // the whole block inside (1 <= i0, j0 < S - 1, one unsigned compare each; none for S <= 2): no
  // per-tap bounds
  const unsigned inner = (unsigned)max(S - 2, 0);
  if ((unsigned)(i0 - 1) < inner && (unsigned)(j0 - 1) < inner) {
    // the lit taps counted in FP32 (sums of 0 and 1, exact): a compare-and-set and an FP32 add per
    // tap instead of an integer select and add, fewer instructions for the integer pipe, the busier
    // one in this kernel; the offset within the map fits 32 bits (S <= 8192)
    const float* p0 = map + ((j0 - 1) * S + (i0 - 1));
    float lit = 0.0f;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy, p0 += S)
      lit += ((__ldg(p0) >= thr) ? 1.0f : 0.0f) + ((__ldg(p0 + 1) >= thr) ? 1.0f : 0.0f) +
             ((__ldg(p0 + 2) >= thr) ? 1.0f : 0.0f);
    return lit * (1.0f / 9.0f);
  }
  int lit = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    int j = j0 + dy;
    bool jin = (unsigned)j < (unsigned)S;
    const float* row = map + (size_t)(jin ? j : 0) * S;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      int i = i0 + dx;
      bool in = jin && (unsigned)i < (unsigned)S;
      lit += in ? (__ldg(row + (in ? i : 0)) >= thr) : 1;
    }
  }
  return (float)lit * (1.0f / 9.0f);
}

template <int FMT, int HDR, bool LDR>
__global__ void __launch_bounds__(256, 4)
    k_shade_shadow(GbufDev g, CamDev cam, const float4* __restrict__ lights, int NL, IblDev ibl, ShadeDev p,
                   ShadowDev sh, void* hdr, long long hdr_pitch, uint8_t* ldr, long long ldr_pitch) {
  __shared__ float4 s_lights[2 * kShadowChunk];
  __shared__ float4 s_cams[4 * kShadowChunk];
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int by = gridDim.y - 1 - blockIdx.y;  // costliest rows first, as k_shade
  const int x = blockIdx.x * 32 + threadIdx.x, y = by * 8 + threadIdx.y;
  const bool inside = x < g.W && y < g.H;
  Px s;
  if (inside) s = px_setup<FMT>(g, cam, x, y);
  const bool active = inside && s.surface;
  const bool diffuse_only = (p.flags & EPBR_SHADE_DIFFUSE_ONLY) != 0;
  Direct d;
  if (active) d = px_direct_begin(s);
  for (int base = 0; base < NL; base += kShadowChunk) {
    const int cnt = min(kShadowChunk, NL - base);
    __syncthreads();  // the previous chunk has been read
    for (int q = tid; q < 4 * cnt; q += 256) s_cams[q] = __ldg(sh.cams + 4 * (size_t)base + q);
    // a chunk of monochrome lights keeps one sum per kind (each channel's sum would be the same)
    const bool mono = __syncthreads_and(stage_lights(s_lights, lights, base, cnt, tid, 256));
    if (!active) continue;
    if (mono && !diffuse_only) {
      float sa = 0.0f, sb = 0.0f, sbf = 0.0f;
      const float* map = sh.maps + (size_t)base * sh.map_texels;
      for (int i = 0; i < cnt; ++i, map += sh.map_texels) {
        const float4 lp = s_lights[2 * i];
        LightTerms t = light_terms(s, d, lp);
        if (t.a > 0.0f || t.b > 0.0f) {
          const float v = shadow_visibility(s_cams + 4 * i, s.P, map, sh.S, sh.b0, sh.b1);
          t.a *= v;
          t.b *= v;
          t.bf *= v;
        }
        sa = sa + lp.w * t.a;  // lp.w: the light's Ic
        sb = sb + lp.w * t.b;
        sbf = sbf + lp.w * t.bf;
      }
      d.sa = d.sa + f3(sa, sa, sa);
      d.sb = d.sb + f3(sb, sb, sb);
      d.sbf = d.sbf + f3(sbf, sbf, sbf);
      continue;
    }
    float3 sa = d.sa, sb = d.sb, sbf = d.sbf;
    for (int i = 0; i < cnt; ++i) {
      float4 lp = s_lights[2 * i], lc = s_lights[2 * i + 1];
      const float* map = sh.maps + (size_t)(base + i) * sh.map_texels;
      if (diffuse_only) {
        float3 L = xyz(lp) - s.P;
        float rs = rsqrt_ftz(fmaf(L.x, L.x, fmaf(L.y, L.y, fmaf(L.z, L.z, 1e-30f))));
        float w = rs * rs * fmaxf(dot3(s.n, L) * rs, 0.0f);
        if (w > 0.0f) w *= shadow_visibility(s_cams + 4 * i, s.P, map, sh.S, sh.b0, sh.b1);
        sa = sa + xyz(lc) * w;
        continue;
      }
      LightTerms t = light_terms(s, d, lp);
      if (t.a > 0.0f || t.b > 0.0f) {
        float v = shadow_visibility(s_cams + 4 * i, s.P, map, sh.S, sh.b0, sh.b1);
        t.a *= v;
        t.b *= v;
        t.bf *= v;
      }
      sa = sa + xyz(lc) * t.a;
      sb = sb + xyz(lc) * t.b;
      sbf = sbf + xyz(lc) * t.bf;
    }
    d.sa = sa;
    d.sb = sb;
    d.sbf = sbf;
  }
  if (!inside) return;
  if (active && NL > 0) {
    if (diffuse_only)
      px_direct_diffuse_end(s, d);
    else
      px_direct_end(s, d);
  }
  // Launched early (EPBR_SHADE_EARLY_START), the kernel before this one on the stream may still be
  // running up to here: the AO it writes is read, and the outputs written, only after it ends.
  griddep_wait();
  const float ao = active ? ao_at(p, x, y) : 1.0f;
  float3 c = px_finish(s, ibl, p.flags, ao);
  if (hdr) store_hdr<HDR>(hdr, hdr_pitch, x, y, c);
  if (LDR) ((unsigned*)(ldr + (size_t)y * ldr_pitch))[x] = pack_rgba8(c, p.exposure, p.op);
}

template <int FMT, int HDR>
static cudaError_t launch_shadow(dim3 grd, dim3 blk, cudaStream_t st, const GbufDev& g, const CamDev& c,
                                 const float4* L, int NL, const IblDev& ibl, const ShadeDev& p, const ShadowDev& sh,
                                 void* hdr, long long hp, uint8_t* ldr, long long lp) {
  const bool early = (p.flags & EPBR_SHADE_EARLY_START) != 0;
  cudaError_t e = launch_kernel(ldr ? k_shade_shadow<FMT, HDR, true> : k_shade_shadow<FMT, HDR, false>, grd, blk, 0, st,
                                early, g, c, L, NL, ibl, p, sh, hdr, hp, ldr, lp);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

epbr_status launch_shade_shadows(const GbufDev& g, const CamDev& c, int fmt, const float4* L, int NL,
                                 const IblDev& ibl, const ShadeDev& p, const epbr_shadows* shadows, void* hdr,
                                 int hdr_format, long long hp, uint8_t* ldr, long long lp, cudaStream_t st) {
  const epbr_shadows* s = shadows;
  if (!s || !s->maps || !s->cameras || (uintptr_t)s->maps % 4 || (uintptr_t)s->cameras % 16 || s->size < 1 ||
      s->size > 8192 || !(s->bias_const >= 0.0f) || !(s->bias_slope >= 0.0f) || !std::isfinite(s->bias_const) ||
      !std::isfinite(s->bias_slope))
    return fail(EPBR_ERR_INVALID_ARG, "shadows: maps / cameras NULL or misaligned, size outside [1, 8192] or "
                "negative / non-finite bias");
  ShadowDev sh{s->maps, (const float4*)s->cameras, (long long)s->size * s->size, s->size, s->bias_const,
               s->bias_slope};
  dim3 blk(32, 8), grd((g.W + 31) / 32, (g.H + 7) / 8);
  cudaError_t e;
  if (fmt == EPBR_GBUFFER_FP32) {
    if (hdr_format == EPBR_HDR_RGBA32F)
      e = launch_shadow<EPBR_GBUFFER_FP32, EPBR_HDR_RGBA32F>(grd, blk, st, g, c, L, NL, ibl, p, sh, hdr, hp, ldr, lp);
    else
      e = launch_shadow<EPBR_GBUFFER_FP32, EPBR_HDR_RGBA16F>(grd, blk, st, g, c, L, NL, ibl, p, sh, hdr, hp, ldr, lp);
  } else {
    if (hdr_format == EPBR_HDR_RGBA32F)
      e = launch_shadow<EPBR_GBUFFER_COMPACT, EPBR_HDR_RGBA32F>(grd, blk, st, g, c, L, NL, ibl, p, sh, hdr, hp, ldr,
                                                                lp);
    else
      e = launch_shadow<EPBR_GBUFFER_COMPACT, EPBR_HDR_RGBA16F>(grd, blk, st, g, c, L, NL, ibl, p, sh, hdr, hp, ldr,
                                                                lp);
  }
  if (e != cudaSuccess) return fail(EPBR_ERR_CUDA, "k_shade_shadow: %s", cudaGetErrorString(e));
  return check_launch("k_shade_shadow");
}

}  // namespace epbr
