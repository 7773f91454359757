// Screen-space ambient occlusion (paper Sec. 5.2: normal-oriented hemisphere of Bavoil &
// Sainz 2008, at half resolution, then a bilateral blur).
//   k_ssao_raw   two AO texels per thread, the sample loop in packed FP32x2 arithmetic; the K
//                kernel offsets sit in shared memory.  TILED: the block's depth footprint plus a
//                kSsaoHalo-pixel halo is copied into shared memory by one TMA tile load
//                (cp.async.bulk.tensor, completion on an mbarrier) while the texels' frames are
//                set up; a warp whose samples all project inside the tile reads its depth taps
//                from it, any other warp (12% of the surface warps of the 1080p scene) and the
//                untiled form read the depth plane through the read-only cache
//   k_ssao_blur  one thread per AO texel; (2R+1)^2 depth-aware taps read from a shared-memory
//                tile of AO values and depths with an R-texel halo
//   k_ssao_blur2 the same for R = 3 with two vertically adjacent texels per thread sharing their
//                tap rows
#include <cuda.h>  // CUtensorMap and its encoder's enums (the encoder is fetched at run time)
#include <string.h>


#include "ssao_core.cuh"
#include "tma.cuh"

namespace epbr {

#ifndef EPBR_SSAO_MIN_BLOCKS
#define EPBR_SSAO_MIN_BLOCKS 4  // resident 256-thread blocks per SM the register budget targets
#endif
#ifndef EPBR_SSAO_TILED_MIN_BLOCKS
#define EPBR_SSAO_TILED_MIN_BLOCKS 3  // the same for the tiled form (48 KB of tile per block)
#endif


// Two AO texels per thread, (i, j) and (i, j + 8) of a 32 x 16 texel tile.  Per texel the
// hemisphere frame is set up as in ssao_texel, then pre-scaled so that a sample k gives its pixel
// coordinates as X / eS + W/2, Y / eS + H/2 with X = ix_scale S.x, Y = -iy_scale S.y, eS = -S.z,
// each three FMAs of the kernel offset; the sample loop runs for both texels in packed FP32x2
// arithmetic.  Depth taps are addressed by a 32-bit texel index (the depth plane holds at most
// 2^32 texels of its pitch, checked on the host).
struct SsaoRows {
  float x[4], y[4], z[4];  // coefficients of (k.x, k.y, k.z, 1)
};

template <int FMT>
__device__ __forceinline__ float ssao_rows(const GbufDev& g, const CamDev& cam, const SsaoDev& p, int i, int j,
                                           bool in, SsaoRows& r) {
#pragma unroll
  for (int q = 0; q < 4; ++q) r.x[q] = r.y[q] = r.z[q] = 0.0f;  // an unused half projects nowhere
  if (!in) return __int_as_float(0x7f800000);
  const int X0 = p.scale * i, Y0 = p.scale * j;
  const float e = gb_depth(g, X0, Y0);
  if (!is_surface(e)) return e;
  const float3 P = e * view_ray(cam, X0, Y0);
  const float3 n = rot_t(cam, gb_normal<FMT>(g, X0, Y0));
  const float2 nz = __ldg(p.noise + ((j & 3) * 4 + (i & 3)));
  const float3 rv = f3(nz.x, nz.y, 0.0f);
  float3 t = rv - n * dot3(rv, n), b;
  const float tt = dot3(t, t);
  if (tt < 1e-8f) {  // |t| < 1e-4
    onb(n, t, b);
  } else {
    t = t * rsqrt_ftz(tt);
    b = cross3(n, t);
  }
  const float3 rt = t * p.radius, rb = b * p.radius, rn = n * p.radius;
  const float sx = cam.ix_scale, sy = -cam.iy_scale;
  r.x[0] = rt.x * sx, r.x[1] = rb.x * sx, r.x[2] = rn.x * sx, r.x[3] = P.x * sx;
  r.y[0] = rt.y * sy, r.y[1] = rb.y * sy, r.y[2] = rn.y * sy, r.y[3] = P.y * sy;
  r.z[0] = -rt.z, r.z[1] = -rb.z, r.z[2] = -rn.z, r.z[3] = -P.z;
  return e;
}

__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }

// Depth tile of the TILED form: the block's 64 x 32 pixel footprint (32 x 16 AO texels at scale
// 2) plus kSsaoHalo pixels on every side, 48 KB of dynamic shared memory.  The halo is a multiple
// of 4 so that the tile's x origin 64 bx - kSsaoHalo is a multiple of 16 bytes, as a tiled TMA
// copy requires; the origin may lie left of or above the image (the copy fills zeros there, and
// such texels never decide a sample: a tap counts only when its pixel lies inside the image).
constexpr int kSsaoHalo = 32;
constexpr int kSsaoTileW = 64 + 2 * kSsaoHalo, kSsaoTileH = 32 + 2 * kSsaoHalo;
constexpr unsigned kSsaoTileN = kSsaoTileW * kSsaoTileH;
constexpr unsigned kSsaoTileBytes = kSsaoTileN * 4;

// Warps of k_ssao_raw<TILED> whose first wait for their tile copy ran out (their taps then all
// read the depth plane, so the AO is unaffected); read and cleared by epbr_ssao_tile_timeouts.
__device__ unsigned int g_ssao_tile_timeouts;
// Set when a block's second (drain) wait ran out too, so that it exited with its copy possibly
// still in flight towards shared memory another block may reuse: the AO of such a launch is
// suspect.  Read and cleared by epbr_ssao_tile_timeouts, which then reports an error.
__device__ unsigned int g_ssao_tile_lost;

// floor(x) as an unsigned pixel index without the conversion unit: x + 1.5 * 2^23 rounded down
// lies on the float grid of spacing 1, so for |x| < 2^22 it is exactly floor(x) + 1.5 * 2^23 and
// its bit pattern minus that of 1.5 * 2^23 is floor(x) (two's complement for negative x).  Any
// other x (|x| >= 2^22, inf, NaN) gives a value >= 2^22 as unsigned, which the on-screen test
// (width and height <= 2^15) rejects, as it rejects the wrapped negative floors.
__device__ __forceinline__ unsigned floor_px(float x) {
  return (unsigned)__float_as_int(__fadd_rd(x, 12582912.0f)) - 0x4B400000u;
}

// Whether every sample of a texel projects inside the tile: each sample point lies within
// Rb = radius * max_k |kernel[k]| of P, so in the pre-scaled coordinates (X, Y, eS) of
// ssao_rows it lies in the box [X_P -+ sx Rb] x [Y_P -+ sy Rb] x [e -+ Rb]; with e - Rb > 0 the
// pixel coordinates X / eS + W/2, Y / eS + H/2 take their extremes at the box's corners.  The
// bounds are widened by 2 pixels, far beyond the FP32 rounding of either computation.
__device__ __forceinline__ bool samples_in_tile(const SsaoRows& r, float e, float Rb, float sx, float sy, float hw,
                                                float hh, int tx0, int ty0) {
  const float dlo = e - Rb, dhi = e + Rb;
  if (!(dlo > 0.0f)) return false;
  const float ilo = 1.0f / dlo, ihi = 1.0f / dhi;
  const float xa = r.x[3] - sx * Rb, xb = r.x[3] + sx * Rb;
  const float ya = r.y[3] - sy * Rb, yb = r.y[3] + sy * Rb;
  const float x0 = floorf(fminf(xa * ilo, xa * ihi) + hw) - 2.0f, x1 = floorf(fmaxf(xb * ilo, xb * ihi) + hw) + 2.0f;
  const float y0 = floorf(fminf(ya * ilo, ya * ihi) + hh) - 2.0f, y1 = floorf(fmaxf(yb * ilo, yb * ihi) + hh) + 2.0f;
  return x0 >= (float)tx0 && x1 < (float)(tx0 + kSsaoTileW) && y0 >= (float)ty0 && y1 < (float)(ty0 + kSsaoTileH);
}

// The sample loop for two texels (packed FP32x2).  FROM_TILE: every tap reads the shared-memory
// tile (the caller has checked that every sample of the warp's texels projects inside it; the
// index is clamped to the tile all the same); otherwise taps read the depth plane.  Branch-free
// as in ssao_texel: an invalid sample (behind the camera or off-screen) reads some in-range texel
// and is masked out.
template <bool FROM_TILE>
__device__ __forceinline__ float2 ssao_samples(const SsaoRows& a, const SsaoRows& b, float e0, float e1,
                                               const float4* s_kernel, const SsaoDev& p, const CamDev& cam,
                                               const GbufDev& g, const float* s_dep, unsigned tbase) {
  const float2 tx = pk(a.x[0], b.x[0]), bx = pk(a.x[1], b.x[1]), nx = pk(a.x[2], b.x[2]), px = pk(a.x[3], b.x[3]);
  const float2 ty = pk(a.y[0], b.y[0]), by = pk(a.y[1], b.y[1]), ny = pk(a.y[2], b.y[2]), py = pk(a.y[3], b.y[3]);
  const float2 tz = pk(a.z[0], b.z[0]), bz = pk(a.z[1], b.z[1]), nz = pk(a.z[2], b.z[2]), pz = pk(a.z[3], b.z[3]);
  const float2 hw = pk(0.5f * cam.W, 0.5f * cam.W), hh = pk(0.5f * cam.H, 0.5f * cam.H);
  const float2 m2 = pk(-2.0f, -2.0f), c3 = pk(3.0f, 3.0f);
  const float* dep = (const float*)g.rt[3];
  const unsigned dp = (unsigned)(g.pitch[3] >> 2);
  const unsigned W = (unsigned)cam.W, H = (unsigned)cam.H;
  float2 occ = pk(0.0f, 0.0f);
#pragma unroll(kSsaoUnroll)
  for (int k = 0; k < p.K; ++k) {
    const float4 ks = s_kernel[k];
    const float2 KX = pk(ks.x, ks.x), KY = pk(ks.y, ks.y), KZ = pk(ks.z, ks.z);
    const float2 X = __ffma2_rn(tx, KX, __ffma2_rn(bx, KY, __ffma2_rn(nx, KZ, px)));
    const float2 Y = __ffma2_rn(ty, KX, __ffma2_rn(by, KY, __ffma2_rn(ny, KZ, py)));
    const float2 Z = __ffma2_rn(tz, KX, __ffma2_rn(bz, KY, __ffma2_rn(nz, KZ, pz)));  // eS
    const float2 inv = pk(rcp_ftz(Z.x), rcp_ftz(Z.y));
    const float2 fx = __ffma2_rn(X, inv, hw), fy = __ffma2_rn(Y, inv, hh);
    const unsigned ix0 = floor_px(fx.x), iy0 = floor_px(fy.x);
    const unsigned ix1 = floor_px(fx.y), iy1 = floor_px(fy.y);
    // From the tile no test is needed: a tap outside the image reads the zeros the copy filled in
    // (0 never passes eb > 0), and a warp reads the tile only when its samples lie in front of
    // the camera (were Z <= 0 after rounding, Z - bias < 0 <= eb would reject the tap anyway).
    const bool v0 = FROM_TILE || (Z.x > 0.0f && ix0 < W && iy0 < H);
    const bool v1 = FROM_TILE || (Z.y > 0.0f && ix1 < W && iy1 < H);
    float eb0, eb1;
    if (FROM_TILE) {
      eb0 = s_dep[min(iy0 * (unsigned)kSsaoTileW + ix0 - tbase, kSsaoTileN - 1)];
      eb1 = s_dep[min(iy1 * (unsigned)kSsaoTileW + ix1 - tbase, kSsaoTileN - 1)];
    } else {
      eb0 = __ldg(dep + (v0 ? iy0 * dp + ix0 : 0u));
      eb1 = __ldg(dep + (v1 ? iy1 * dp + ix1 : 0u));
    }
    // eb <= eS - bias (finite) already excludes a background tap at +inf
    const bool h0 = v0 && eb0 > 0.0f && eb0 <= Z.x - p.bias;
    const bool h1 = v1 && eb1 > 0.0f && eb1 <= Z.y - p.bias;
    const float2 x = pk(__saturatef(p.radius * rcp_ftz(fabsf(e0 - eb0))),
                        __saturatef(p.radius * rcp_ftz(fabsf(e1 - eb1))));
    const float2 sm = __fmul2_rn(__fmul2_rn(x, x), __ffma2_rn(m2, x, c3));  // smoothstep
    occ = __fadd2_rn(occ, pk(h0 ? sm.x : 0.0f, h1 ? sm.y : 0.0f));
  }
  return occ;
}

template <int FMT, bool TILED>
__global__ void __launch_bounds__(256, TILED ? EPBR_SSAO_TILED_MIN_BLOCKS : EPBR_SSAO_MIN_BLOCKS)
    k_ssao_raw(const __grid_constant__ CUtensorMap depth_map, GbufDev g, CamDev cam, SsaoDev p,
               float* __restrict__ ao, long long ao_pitch, int Wa, int Ha, unsigned long long wait_ns) {
  __shared__ float4 s_kernel[kMaxSsaoSamples];
  __shared__ __align__(8) unsigned long long s_bar;
  extern __shared__ __align__(128) float s_dep[];  // TILED: kSsaoTileH x kSsaoTileW depths
  // a blur launched early after this kernel may put its blocks on the SMs this grid's last wave
  // leaves free; it waits for this grid before it reads the AO
  griddep_launch_dependents();
  const int tid = threadIdx.y * 32 + threadIdx.x;
  // tile origin in pixels (a scale-2 block covers pixels [64 bx, 64 bx + 64) x [32 by, 32 by + 32))
  const int tx0 = (int)blockIdx.x * 64 - kSsaoHalo, ty0 = (int)blockIdx.y * 32 - kSsaoHalo;
  if (TILED && tid == 0) tma_load_tile_2d(&depth_map, s_dep, smem_addr(&s_bar), tx0, ty0, kSsaoTileBytes);
  for (int k = tid; k < p.K; k += 256) s_kernel[k] = __ldg(p.kernel + k);
  const int i = blockIdx.x * 32 + threadIdx.x, j0 = blockIdx.y * 16 + threadIdx.y, j1 = j0 + 8;
  const bool in0 = i < Wa && j0 < Ha, in1 = i < Wa && j1 < Ha;
  SsaoRows a, b;
  const float e0 = ssao_rows<FMT>(g, cam, p, i, j0, in0, a);
  const float e1 = ssao_rows<FMT>(g, cam, p, i, j1, in1, b);
  __syncthreads();  // also orders the mbarrier's initialisation before every thread's wait
  const bool s0 = in0 && is_surface(e0), s1 = in1 && is_surface(e1);
  bool tile_ok = false, from_tile = false;
  if (TILED) {
    // wait_ns = 0 gives up at once (the fallback path, exercised by a test)
    tile_ok = wait_ns != 0 && mbar_wait_bounded(smem_addr(&s_bar), 0, wait_ns);
    if (!tile_ok && threadIdx.x == 0) atomicAdd(&g_ssao_tile_timeouts, 1u);
    // the longest kernel offset, over the warp's lanes
    float k2 = 0.0f;
    for (int k = threadIdx.x; k < p.K; k += 32) {
      const float4 ks = s_kernel[k];
      k2 = fmaxf(k2, fmaf(ks.x, ks.x, fmaf(ks.y, ks.y, ks.z * ks.z)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) k2 = fmaxf(k2, __shfl_xor_sync(0xffffffffu, k2, o));
    const float Rb = p.radius * sqrtf(k2) * 1.0001f;
    const float sx = cam.ix_scale, sy = cam.iy_scale, hw = 0.5f * cam.W, hh = 0.5f * cam.H;
    const bool fit = (!s0 || samples_in_tile(a, e0, Rb, sx, sy, hw, hh, tx0, ty0)) &&
                     (!s1 || samples_in_tile(b, e1, Rb, sx, sy, hw, hh, tx0, ty0));
    from_tile = __all_sync(0xffffffffu, tile_ok && fit);
  }
  if (s0 || s1) {
    const unsigned tbase = (unsigned)ty0 * (unsigned)kSsaoTileW + (unsigned)tx0;
    const float2 occ = from_tile ? ssao_samples<true>(a, b, e0, e1, s_kernel, p, cam, g, s_dep, tbase)
                                 : ssao_samples<false>(a, b, e0, e1, s_kernel, p, cam, g, s_dep, tbase);
    if (s0) ((float*)((char*)ao + (size_t)j0 * ao_pitch))[i] = fmaf(-occ.x, p.inv_k, 1.0f);
    if (s1) ((float*)((char*)ao + (size_t)j1 * ao_pitch))[i] = fmaf(-occ.y, p.inv_k, 1.0f);
  }
  if (in0 && !s0) ((float*)((char*)ao + (size_t)j0 * ao_pitch))[i] = 1.0f;
  if (in1 && !s1) ((float*)((char*)ao + (size_t)j1 * ao_pitch))[i] = 1.0f;
  // A copy that had not landed is waited for once more (bounded) so that it does not write into
  // the shared memory of a block that starts on this SM after this one; if that wait runs out
  // too, the launch is flagged.
  if (TILED && !tile_ok && !mbar_wait_bounded(smem_addr(&s_bar), 0, kTmaWaitNs) && threadIdx.x == 0)
    atomicOr(&g_ssao_tile_lost, 1u);
}

// Blur tile: 32x8 AO texels plus a halo of R <= 8 texels, AO values and the depths of their
// source pixels staged in shared memory (taps outside the image are staged as background).
constexpr int kBlurBX = 32, kBlurBY = 8, kBlurMaxR = 8;
constexpr int kBlurTW = kBlurBX + 2 * kBlurMaxR, kBlurTH = kBlurBY + 2 * kBlurMaxR;

template <int FMT>
__global__ void __launch_bounds__(kBlurBX* kBlurBY) k_ssao_blur(GbufDev g, SsaoDev p, const float* __restrict__ in,
                                                                long long in_pitch, float* __restrict__ out,
                                                                long long out_pitch, int Wa, int Ha) {
  __shared__ float s_ao[kBlurTH][kBlurTW];
  __shared__ float s_e[kBlurTH][kBlurTW];
  // launched early: nothing is read before the previous kernel (the raw AO's) has finished;
  // a compose launched early after this one may start once every block is past this point
  griddep_wait();
  griddep_launch_dependents();
  const int R = p.R;
  const int tw = kBlurBX + 2 * R, th = kBlurBY + 2 * R;
  const int i0 = blockIdx.x * kBlurBX - R, j0 = blockIdx.y * kBlurBY - R;
  const float inf = __int_as_float(0x7f800000);
  for (int q = threadIdx.y * kBlurBX + threadIdx.x; q < tw * th; q += kBlurBX * kBlurBY) {
    int ty = q / tw, tx = q - ty * tw;
    int qi = i0 + tx, qj = j0 + ty;
    float a = 0.0f, e = inf;
    if (qi >= 0 && qi < Wa && qj >= 0 && qj < Ha) {
      a = __ldg((const float*)((const char*)in + (size_t)qj * in_pitch) + qi);
      e = gb_depth(g, p.scale * qi, p.scale * qj);
    }
    s_ao[ty][tx] = a;
    s_e[ty][tx] = e;
  }
  __syncthreads();
  int i = blockIdx.x * kBlurBX + threadIdx.x, j = blockIdx.y * kBlurBY + threadIdx.y;
  if (i >= Wa || j >= Ha) return;
  ((float*)((char*)out + (size_t)j * out_pitch))[i] =
      ssao_blur_texel(p, &s_ao[threadIdx.y + R][threadIdx.x + R], &s_e[threadIdx.y + R][threadIdx.x + R], kBlurTW);
}

// The 7x7 blur (R = 3) with two vertically adjacent AO texels per thread, (i, 2 ty') and
// (i, 2 ty' + 1) of a 32 x 16 texel tile: the (AO, depth) pairs of the tile and its 3-texel halo sit
// in shared memory as float2, and the 8 rows x 7 columns a thread reads serve both texels (6 of the
// 7 rows are shared), 56 loads instead of 2 x 2 x 49.  Each texel's sum runs over the taps in the
// order of ssao_blur_texel_r, so the result is that function's bit for bit.
constexpr int kBlur2R = 3, kBlur2TW = kBlurBX + 2 * kBlur2R, kBlur2TH = 2 * kBlurBY + 2 * kBlur2R;

template <int FMT>
__global__ void __launch_bounds__(kBlurBX* kBlurBY) k_ssao_blur2(GbufDev g, SsaoDev p, const float* __restrict__ in,
                                                                 long long in_pitch, float* __restrict__ out,
                                                                 long long out_pitch, int Wa, int Ha) {
  __shared__ float2 s_ae[kBlur2TH][kBlur2TW];
  griddep_wait();  // as k_ssao_blur
  griddep_launch_dependents();
  const int i0 = blockIdx.x * kBlurBX - kBlur2R, j0 = blockIdx.y * (2 * kBlurBY) - kBlur2R;
  const float inf = __int_as_float(0x7f800000);
  for (int q = threadIdx.y * kBlurBX + threadIdx.x; q < kBlur2TW * kBlur2TH; q += kBlurBX * kBlurBY) {
    const int ty = q / kBlur2TW, tx = q - ty * kBlur2TW;
    const int qi = i0 + tx, qj = j0 + ty;
    float a = 0.0f, e = inf;
    if (qi >= 0 && qi < Wa && qj >= 0 && qj < Ha) {
      a = __ldg((const float*)((const char*)in + (size_t)qj * in_pitch) + qi);
      e = gb_depth(g, p.scale * qi, p.scale * qj);
    }
    s_ae[ty][tx] = make_float2(a, e);
  }
  __syncthreads();
  const int i = blockIdx.x * kBlurBX + threadIdx.x, ja = blockIdx.y * (2 * kBlurBY) + 2 * threadIdx.y, jb = ja + 1;
  if (i >= Wa || ja >= Ha) return;
  // tile row 2 ty' + k holds texel row ja - 3 + k: texel a reads k = 0..6 (dy = k - 3), b k = 1..7
  const float epa = s_ae[2 * threadIdx.y + kBlur2R][threadIdx.x + kBlur2R].y;
  const float epb = s_ae[2 * threadIdx.y + kBlur2R + 1][threadIdx.x + kBlur2R].y;
  const bool sa = is_surface(epa), sb = jb < Ha && is_surface(epb);
  const float ks = p.blur_ks;
  const float kza = -1.4426950408889634f * rcp_ftz(p.sigma_z * epa);
  const float kzb = -1.4426950408889634f * rcp_ftz(p.sigma_z * epb);
  float na = 0.0f, da = 0.0f, nb = 0.0f, db = 0.0f;
#pragma unroll
  for (int k = 0; k < 2 * kBlur2R + 2; ++k) {
    const float2* row = &s_ae[2 * threadIdx.y + k][threadIdx.x];
#pragma unroll
    for (int c = 0; c < 2 * kBlur2R + 1; ++c) {
      const float2 v = row[c];
      const int dx = c - kBlur2R;
      if (k <= 2 * kBlur2R) {
        const int dy = k - kBlur2R;
        const float w = ex2_ftz(fmaf(fabsf(v.y - epa), kza, (float)(dx * dx + dy * dy) * ks));
        na = fmaf(w, v.x, na);
        da += w;
      }
      if (k >= 1) {
        const int dy = k - 1 - kBlur2R;
        const float w = ex2_ftz(fmaf(fabsf(v.y - epb), kzb, (float)(dx * dx + dy * dy) * ks));
        nb = fmaf(w, v.x, nb);
        db += w;
      }
    }
  }
  ((float*)((char*)out + (size_t)ja * out_pitch))[i] = sa ? na * rcp_ftz(da) : 1.0f;
  if (jb < Ha) ((float*)((char*)out + (size_t)jb * out_pitch))[i] = sb ? nb * rcp_ftz(db) : 1.0f;
}

static epbr_status validate_ssao(const epbr_ssao_params* p) {
  if (!p) return fail(EPBR_ERR_INVALID_ARG, "ssao params is NULL");
  if (p->num_samples < 1 || p->num_samples > kMaxSsaoSamples)
    return fail(EPBR_ERR_INVALID_ARG, "ssao num_samples %d outside [1, %d]", p->num_samples, kMaxSsaoSamples);
  if (p->scale != 1 && p->scale != 2) return fail(EPBR_ERR_INVALID_ARG, "ssao scale must be 1 or 2");
  if (!(p->radius > 0.0f) || !(p->bias >= 0.0f) || !(p->sigma_s > 0.0f) || !(p->sigma_z > 0.0f))
    return fail(EPBR_ERR_INVALID_ARG, "ssao radius/bias/sigmas invalid");
  if (p->blur_radius < 0 || p->blur_radius > 8) return fail(EPBR_ERR_INVALID_ARG, "ssao blur_radius outside [0, 8]");
  if (!p->kernel || !p->noise || (uintptr_t)p->kernel % 16 || (uintptr_t)p->noise % 8)
    return fail(EPBR_ERR_INVALID_ARG, "ssao kernel/noise NULL or misaligned");
  return EPBR_OK;
}


static void ao_dims(const epbr_gbuffer* g, const epbr_ssao_params* p, int* w, int* h) {
  *w = (g->width + p->scale - 1) / p->scale;
  *h = (g->height + p->scale - 1) / p->scale;
}

static epbr_status check_ao_buffer(const void* ao, int64_t pitch, int Wa, const char* what) {
  if (!ao || (uintptr_t)ao % 4 || pitch < (int64_t)Wa * 4 || pitch % 4)
    return fail(EPBR_ERR_INVALID_ARG, "%s: AO buffer NULL, misaligned or pitch too small", what);
  return EPBR_OK;
}


// cuTensorMapEncodeTiled, fetched from the driver once per process (the library links only the
// CUDA runtime); null when the driver does not provide it.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return (EncodeTiledFn)f;
  }();
  return fn;
}

// The TILED form applies at scale 2 to views of at most kSsaoTiledMaxRows rows when the depth
// plane meets the TMA rules (16-byte aligned base, row pitch a multiple of 16 bytes below 2^40)
// and the tensor map encodes; `map` then describes the depth plane with a kSsaoTileW x kSsaoTileH
// box.  The row limit: the samples' spread in pixels grows with the view's focal length in pixels
// (its height, at a given field of view) while the halo is fixed, so on taller views fewer warps
// fit the tile (88% of the surface warps at 1080p, 35% at 2160p on the generator's scenes) and
// the untiled form, at its higher occupancy, is used.
constexpr int kSsaoTiledMaxRows = 1536;


static bool depth_tile_map(const epbr_gbuffer* g, const epbr_ssao_params* p, CUtensorMap* map) {
  if (p->scale != 2 || g->height > kSsaoTiledMaxRows || (uintptr_t)g->rt[3] % 16 || g->pitch[3] % 16 ||
      g->pitch[3] >= (1ll << 40))
    return false;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)g->width, (cuuint64_t)g->height};
  const cuuint64_t strides[1] = {(cuuint64_t)g->pitch[3]};
  const cuuint32_t box[2] = {(cuuint32_t)kSsaoTileW, (cuuint32_t)kSsaoTileH};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)g->rt[3], dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace epbr

using namespace epbr;

extern "C" epbr_status epbr_ssao_size(const epbr_gbuffer* g, const epbr_ssao_params* p, int32_t* w, int32_t* h) {
  epbr_status st = validate_gbuffer(g, false);
  if (st) return st;
  if ((st = validate_ssao(p))) return st;
  if (!w || !h) return fail(EPBR_ERR_INVALID_ARG, "output pointers NULL");
  ao_dims(g, p, w, h);
  return ok();
}

extern "C" epbr_status epbr_ssao_workspace_size(const epbr_gbuffer* g, const epbr_ssao_params* p, size_t* bytes) {
  int w, h;
  epbr_status st = epbr_ssao_size(g, p, &w, &h);
  if (st) return st;
  if (!bytes) return fail(EPBR_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = (size_t)w * h * 4;
  return ok();
}

extern "C" epbr_status epbr_ssao_raw(const epbr_gbuffer* g, const epbr_camera* cam, const epbr_ssao_params* p,
                                     float* ao, int64_t ao_pitch, void* stream) {
  epbr_status st = validate_gbuffer(g, false);
  if (st) return st;
  if ((st = validate_camera(cam, g))) return st;
  if ((st = validate_ssao(p))) return st;
  int Wa, Ha;
  ao_dims(g, p, &Wa, &Ha);
  if ((st = check_ao_buffer(ao, ao_pitch, Wa, "ssao_raw"))) return st;
  if ((uint64_t)g->height * (uint64_t)(g->pitch[3] / 4) > 0xffffffffull)
    return fail(EPBR_ERR_UNSUPPORTED, "ssao_raw: depth plane of more than 2^32 texels (height x pitch / 4)");
  dim3 blk(32, 8), grd((Wa + 31) / 32, (Ha + 15) / 16);
  GbufDev gd = make_gbuf(*g);
  CamDev cd = make_cam(*cam);
  SsaoDev sd = make_ssao(*p);
  cudaStream_t s = (cudaStream_t)stream;
  CUtensorMap map;
  const bool tiled = depth_tile_map(g, p, &map);
  if (!tiled) memset(&map, 0, sizeof(map));  // unused by the untiled form
  const bool fp32 = g->format == EPBR_GBUFFER_FP32;
  if (tiled) {
    void (*k)(const CUtensorMap, GbufDev, CamDev, SsaoDev, float*, long long, int, int, unsigned long long) =
        fp32 ? k_ssao_raw<EPBR_GBUFFER_FP32, true> : k_ssao_raw<EPBR_GBUFFER_COMPACT, true>;
    // the 48 KB tile is above the default dynamic shared-memory limit; the attribute is per
    // function and device, and setting it again is harmless
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSsaoTileBytes) != cudaSuccess)
      return fail(EPBR_ERR_CUDA, "ssao_raw: shared-memory attribute: %s", cudaGetErrorString(cudaGetLastError()));
    k<<<grd, blk, kSsaoTileBytes, s>>>(map, gd, cd, sd, ao, ao_pitch, Wa, Ha, tma_first_wait_ns());
  } else if (fp32)
    k_ssao_raw<EPBR_GBUFFER_FP32, false><<<grd, blk, 0, s>>>(map, gd, cd, sd, ao, ao_pitch, Wa, Ha, 0ull);
  else
    k_ssao_raw<EPBR_GBUFFER_COMPACT, false><<<grd, blk, 0, s>>>(map, gd, cd, sd, ao, ao_pitch, Wa, Ha, 0ull);
  if ((st = check_launch("k_ssao_raw"))) return st;
  return ok();
}

extern "C" epbr_status epbr_ssao_tiled(const epbr_gbuffer* g, const epbr_ssao_params* p, int32_t* tiled) {
  int w, h;
  epbr_status st = epbr_ssao_size(g, p, &w, &h);
  if (st) return st;
  if (!tiled) return fail(EPBR_ERR_INVALID_ARG, "tiled is NULL");
  CUtensorMap map;
  *tiled = depth_tile_map(g, p, &map) ? 1 : 0;
  return ok();
}

extern "C" epbr_status epbr_ssao_tile_timeouts(uint32_t* count) {
  if (!count) return fail(EPBR_ERR_INVALID_ARG, "count is NULL");
  unsigned v = 0, lost = 0;
  const unsigned zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_ssao_tile_timeouts, sizeof(v)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_ssao_tile_timeouts, &zero, sizeof(zero)) != cudaSuccess ||
      cudaMemcpyFromSymbol(&lost, g_ssao_tile_lost, sizeof(lost)) != cudaSuccess ||
      cudaMemcpyToSymbol(g_ssao_tile_lost, &zero, sizeof(zero)) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "ssao_tile_timeouts: %s", cudaGetErrorString(cudaGetLastError()));
  *count = v;
  if (lost)
    return fail(EPBR_ERR_DEVICE_STATUS,
                "ssao_tile_timeouts: a block's depth-tile copy did not complete within two waits of %llu ms; "
                "the AO of launches since the last call is suspect",
                (unsigned long long)(kTmaWaitNs / 1000000));
  return ok();
}

extern "C" epbr_status epbr_ssao_set_tile_wait(uint64_t first_wait_ns, uint64_t* previous_ns) {
  if (first_wait_ns > kTmaWaitNs)
    return fail(EPBR_ERR_INVALID_ARG, "ssao_set_tile_wait: %llu ns above the default %llu ns",
                (unsigned long long)first_wait_ns, (unsigned long long)kTmaWaitNs);
  const unsigned long long prev = set_tma_first_wait_ns(first_wait_ns);
  if (previous_ns) *previous_ns = prev;
  return ok();
}

extern "C" epbr_status epbr_ssao_blur(const epbr_gbuffer* g, const epbr_ssao_params* p, const float* in,
                                      int64_t in_pitch, float* out, int64_t out_pitch, void* stream) {
  epbr_status st = validate_gbuffer(g, false);
  if (st) return st;
  if ((st = validate_ssao(p))) return st;
  int Wa, Ha;
  ao_dims(g, p, &Wa, &Ha);
  if ((st = check_ao_buffer(in, in_pitch, Wa, "ssao_blur in"))) return st;
  if ((st = check_ao_buffer(out, out_pitch, Wa, "ssao_blur out"))) return st;
  if (in == out) return fail(EPBR_ERR_INVALID_ARG, "ssao_blur: in and out must differ");
  dim3 blk(kBlurBX, kBlurBY), grd((Wa + kBlurBX - 1) / kBlurBX, (Ha + kBlurBY - 1) / kBlurBY);
  GbufDev gd = make_gbuf(*g);
  SsaoDev sd = make_ssao(*p);
  cudaStream_t s = (cudaStream_t)stream;
  // Launched early (programmatic stream serialisation): the blocks may take the SMs that the
  // previous kernel's last wave leaves free and wait there for it (griddep_wait before any read),
  // which hides the launch gap after the raw AO pass.
  const bool fp32 = g->format == EPBR_GBUFFER_FP32;
  cudaError_t e;
  if (p->blur_radius == kBlur2R) {  // the 7x7 blur: two texels per thread
    dim3 grd2((Wa + kBlurBX - 1) / kBlurBX, (Ha + 2 * kBlurBY - 1) / (2 * kBlurBY));
    e = launch_kernel(fp32 ? k_ssao_blur2<EPBR_GBUFFER_FP32> : k_ssao_blur2<EPBR_GBUFFER_COMPACT>, grd2, blk, 0, s,
                      true, gd, sd, in, (long long)in_pitch, out, (long long)out_pitch, Wa, Ha);
  } else {
    e = launch_kernel(fp32 ? k_ssao_blur<EPBR_GBUFFER_FP32> : k_ssao_blur<EPBR_GBUFFER_COMPACT>, grd, blk, 0, s, true,
                      gd, sd, in, (long long)in_pitch, out, (long long)out_pitch, Wa, Ha);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(EPBR_ERR_CUDA, "k_ssao_blur: %s", cudaGetErrorString(e));
  }
  if ((st = check_launch("k_ssao_blur"))) return st;
  return ok();
}

extern "C" epbr_status epbr_ssao(const epbr_gbuffer* g, const epbr_camera* cam, const epbr_ssao_params* p,
                                 float* ao, int64_t ao_pitch, void* ws, size_t ws_bytes, void* stream) {
  int Wa, Ha;
  epbr_status st = epbr_ssao_size(g, p, &Wa, &Ha);
  if (st) return st;
  if (p->blur_radius == 0) return epbr_ssao_raw(g, cam, p, ao, ao_pitch, stream);
  size_t need = (size_t)Wa * Ha * 4;
  if (!ws || ws_bytes < need || (uintptr_t)ws % 4)
    return fail(EPBR_ERR_NO_MEMORY, "ssao: workspace needs %zu bytes, got %zu", need, ws ? ws_bytes : (size_t)0);
  if ((st = epbr_ssao_raw(g, cam, p, (float*)ws, (int64_t)Wa * 4, stream))) return st;
  return epbr_ssao_blur(g, p, (const float*)ws, (int64_t)Wa * 4, ao, ao_pitch, stream);
}
