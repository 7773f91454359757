// Image-based lighting precompute (paper Sec. 3.1; split sum of Karis 2013):
//   k_brdf_lut          BRDF integration table (A, B), one warp per texel, Kahan + shuffles
//   k_irradiance_part   exact-quadrature irradiance, per-block partial sums over a slice of
//                       source texels staged in shared memory (packed FP32x2 over output pairs,
//                       plain sums per staged tile, Kahan across tiles)
//   k_irradiance_final  one warp per output: lanes sum the block partials, a shuffle butterfly
//                       adds the lanes (fixed order: deterministic), then the ratio
//   k_prefilter         GGX-prefiltered levels 1..M-1, one block per row of a level: the row's
//                       sample geometry computed once (the sampling frame turns with the texel
//                       about the pole axis), each texel sums its samples at shifted columns
#include <cuda.h>  // CUcontext and CUresult for the context queries (fetched at run time)

#include <algorithm>
#include <mutex>

#include "epbr_internal.cuh"

namespace epbr {

// Hammersley point k of N: (k / N, radical_inverse_2(k)).  For k < 2^24 the mirrored bits fit
// the float mantissa, so xi2 is exact.
__device__ __forceinline__ float hammersley_xi2(unsigned k) {
  return __uint2float_rn(__brev(k)) * 2.3283064365386963e-10f;
}

// GGX half vector in the frame (t, b, n): phi = 2 pi xi1, cos^2 = (1 - xi2) / d,
// sin^2 = alpha^2 xi2 / d with d = 1 + (alpha^2 - 1) xi2 (sin^2 taken directly, which avoids
// the cancellation of 1 - cos^2 near the lobe centre).
__device__ __forceinline__ float3 ggx_half(float xi1, float xi2, float a2, float3 t, float3 b, float3 n) {
  float inv = 1.0f / fmaf(a2 - 1.0f, xi2, 1.0f);
  float ct = sqrtf((1.0f - xi2) * inv);
  float st = sqrtf(a2 * xi2 * inv);
  float sp, cp;
  sincospif(2.0f * xi1, &sp, &cp);
  return t * (st * cp) + b * (st * sp) + n * ct;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------------------------------
// BRDF integration table
// ------------------------------------------------------------------------------------------
__global__ void k_brdf_lut(int S, int N, float2* __restrict__ lut) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= S * S) return;
  int i = warp % S, j = warp / S;
  float mu = (i + 0.5f) / S, r = (j + 0.5f) / S;
  float alpha = r * r, a2 = alpha * alpha, k = 0.5f * alpha;
  float3 v = f3(sqrtf(fmaf(-mu, mu, 1.0f)), 0.0f, mu);
  float nv = mu;
  float g1v = nv / fmaf(nv, 1.0f - k, k);
  Kahan A, B;
  const float3 t = f3(1, 0, 0), b = f3(0, 1, 0), n = f3(0, 0, 1);
  float invN = 1.0f / N;
  for (int s = lane; s < N; s += 32) {
    float3 h = ggx_half(s * invN, hammersley_xi2((unsigned)s), a2, t, b, n);
    float vh = dot3(v, h);
    float nl = fmaf(2.0f * vh, h.z, -v.z);
    if (nl > 0.0f) {
      float g = g1v * nl / fmaf(nl, 1.0f - k, k);
      float gvis = g * vh / (h.z * nv);
      float x = 1.0f - vh, x2 = x * x;
      float fc = x2 * x2 * x;
      A.add((1.0f - fc) * gvis);
      B.add(fc * gvis);
    }
  }
  float a = warp_sum(A.s - A.c), bb = warp_sum(B.s - B.c);
  if (lane == 0) lut[warp] = make_float2(a * invN, bb * invN);
}

// ------------------------------------------------------------------------------------------
// Irradiance: sum_t L_t max(n.d_t, 0) Omega_t / sum_t max(n.d_t, 0) Omega_t
// ------------------------------------------------------------------------------------------
constexpr int kIrrThreads = 128;
constexpr int kIrrOutPerThread = 4;  // outputs per thread and pass (two packed pairs): 512 per pass
constexpr int kIrrTile = 256;        // source texels staged per step
constexpr int kIrrTexelsPerBlock = 1024;
constexpr int kIrrMaxBlocks = 608;

int irr_blocks(int We, int He) {
  long long n = (long long)We * He;
  long long b = (n + kIrrTexelsPerBlock - 1) / kIrrTexelsPerBlock;
  return (int)std::min<long long>(std::max<long long>(b, 1), kIrrMaxBlocks);
}

size_t irr_workspace_bytes(int We, int He, int Wi, int Hi) {
  return (size_t)irr_blocks(We, He) * Wi * Hi * sizeof(float4);
}

// Unit direction of the centre of texel (i, j) of a W x H equirect map.
__device__ __forceinline__ float3 texel_dir(int i, int j, int W, int H) {
  float st, ct, sp, cp;
  sincospif((j + 0.5f) / H, &st, &ct);
  sincospif(2.0f * ((i + 0.5f) / W) - 1.0f, &sp, &cp);
  return f3(st * sp, ct, -st * cp);
}

// Each block sums over its slice of source texels for every output texel; a thread owns
// kIrrOutPerThread outputs as two pairs whose arithmetic runs in packed FP32x2 instructions.
// A source texel is staged once per tile as d Omega (max(n.d, 0) Omega = max(n.(d Omega), 0) since
// Omega > 0) and L, every value duplicated into both halves of a pair: (dx, dx, dy, dy),
// (dz, dz, Lr, Lr), (Lg, Lg, Lb, Lb).  Per tile the four sums of each output (L w and w) are
// plain FP32; the tile's sums are then added to the slice totals with Kahan compensation.
__global__ void __launch_bounds__(kIrrThreads) k_irradiance_part(const float4* __restrict__ env, int We,
                                                                 int He, int Wi, int Hi,
                                                                 float4* __restrict__ part) {
  __shared__ float4 s_src[kIrrTile][3];
  long long ntex = (long long)We * He;
  long long per = (ntex + gridDim.x - 1) / gridDim.x;
  long long t0 = per * blockIdx.x;
  long long t1 = t0 + per < ntex ? t0 + per : ntex;
  int nout = Wi * Hi;
  // Omega of row y = (2 pi / W)(cos(pi y / H) - cos(pi (y + 1) / H))
  //               = (4 pi / W) sin(pi (y + 0.5) / H) sin(pi / (2 H))   (product form)
  float row_k = 4.0f * kPi / We * sinpif(0.5f / He);
  for (int og = 0; og < nout; og += kIrrThreads * kIrrOutPerThread) {
    // pair p holds outputs og + (2p + h) * kIrrThreads + tid, h = 0, 1; an absent output has n = 0
    float2 nx[2], ny[2], nz[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      float3 a, b;
      int oa = og + (2 * p) * kIrrThreads + threadIdx.x, ob = oa + kIrrThreads;
      a = oa < nout ? texel_dir(oa % Wi, oa / Wi, Wi, Hi) : f3(0, 0, 0);
      b = ob < nout ? texel_dir(ob % Wi, ob / Wi, Wi, Hi) : f3(0, 0, 0);
      nx[p] = make_float2(a.x, b.x), ny[p] = make_float2(a.y, b.y), nz[p] = make_float2(a.z, b.z);
    }
    Kahan acc[kIrrOutPerThread][4];
    for (long long base = t0; base < t1; base += kIrrTile) {
      int cnt = (int)(t1 - base < kIrrTile ? t1 - base : kIrrTile);
      __syncthreads();
      for (int q = threadIdx.x; q < cnt; q += kIrrThreads) {
        long long t = base + q;
        int x = (int)(t % We), y = (int)(t / We);
        float3 d = texel_dir(x, y, We, He) * (row_k * sinpif((y + 0.5f) / He));
        float4 L = __ldg(env + t);
        s_src[q][0] = make_float4(d.x, d.x, d.y, d.y);
        s_src[q][1] = make_float4(d.z, d.z, L.x, L.x);
        s_src[q][2] = make_float4(L.y, L.y, L.z, L.z);
      }
      __syncthreads();
      float2 sr[2], sg[2], sb[2], sw[2];
#pragma unroll
      for (int p = 0; p < 2; ++p) sr[p] = sg[p] = sb[p] = sw[p] = make_float2(0.0f, 0.0f);
#pragma unroll 4
      for (int q = 0; q < cnt; ++q) {
        const float4 u = s_src[q][0], v = s_src[q][1], z = s_src[q][2];
        const float2 dx = make_float2(u.x, u.y), dy = make_float2(u.z, u.w), dz = make_float2(v.x, v.y);
        const float2 Lr = make_float2(v.z, v.w), Lg = make_float2(z.x, z.y), Lb = make_float2(z.z, z.w);
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          float2 w = __ffma2_rn(nx[p], dx, __ffma2_rn(ny[p], dy, __fmul2_rn(nz[p], dz)));
          w = make_float2(fmaxf(w.x, 0.0f), fmaxf(w.y, 0.0f));
          sr[p] = __ffma2_rn(Lr, w, sr[p]);
          sg[p] = __ffma2_rn(Lg, w, sg[p]);
          sb[p] = __ffma2_rn(Lb, w, sb[p]);
          sw[p] = __fadd2_rn(sw[p], w);
        }
      }
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        acc[2 * p][0].add(sr[p].x), acc[2 * p][1].add(sg[p].x), acc[2 * p][2].add(sb[p].x);
        acc[2 * p][3].add(sw[p].x);
        acc[2 * p + 1][0].add(sr[p].y), acc[2 * p + 1][1].add(sg[p].y), acc[2 * p + 1][2].add(sb[p].y);
        acc[2 * p + 1][3].add(sw[p].y);
      }
    }
#pragma unroll
    for (int r = 0; r < kIrrOutPerThread; ++r) {
      int o = og + r * kIrrThreads + threadIdx.x;
      if (o < nout)
        part[(size_t)blockIdx.x * nout + o] =
            make_float4(acc[r][0].s - acc[r][0].c, acc[r][1].s - acc[r][1].c,
                        acc[r][2].s - acc[r][2].c, acc[r][3].s - acc[r][3].c);
    }
  }
}

// One warp per output texel: lane l sums the partials of blocks l, l + 32, ... (Kahan), then the
// lanes' sums are added by a butterfly of shuffles (a fixed order: deterministic).
__global__ void k_irradiance_final(const float4* __restrict__ part, int nblocks, int nout,
                                   float4* __restrict__ out) {
  const int o = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (o >= nout) return;  // warp-uniform
  Kahan s[4];
  for (int b = lane; b < nblocks; b += 32) {
    float4 p = __ldg(part + (size_t)b * nout + o);
    s[0].add(p.x);
    s[1].add(p.y);
    s[2].add(p.z);
    s[3].add(p.w);
  }
  const float r = warp_sum(s[0].s - s[0].c), g = warp_sum(s[1].s - s[1].c);
  const float bl = warp_sum(s[2].s - s[2].c), den = warp_sum(s[3].s - s[3].c);
  if (lane != 0) return;
  float inv = den > 0.0f ? 1.0f / den : 0.0f;  // no texel centre in the hemisphere: 0
  out[o] = make_float4(r * inv, g * inv, bl * inv, 1.0f);
}

// ------------------------------------------------------------------------------------------
// Prefiltered levels 1..M-1 in one launch
// ------------------------------------------------------------------------------------------
struct ChainDev {
  int M;
  int nlev;                       // levels written: 1..M-1
  long long off[EPBR_MAX_LEVELS + 1];  // texel prefix sums over levels 1..M-1
  int W[EPBR_MAX_LEVELS], H[EPBR_MAX_LEVELS];
  float4* dst[EPBR_MAX_LEVELS];
};

// With n = v, a GGX half vector h with tangent-space components (sin t cos p, sin t sin p, cos t)
// gives l = 2 (n.h) h - n = T (2 h_z h_x) + B (2 h_z h_y) + n (2 h_z^2 - 1), n.l = 2 h_z^2 - 1:
// functions of the sample and the level only.  The frame (T, B, n) is built from the map's pole
// axis (T = y x n normalised, B = n x T), so it turns with n about that axis: the texels of one
// row of a level share every sample's polar angle, and their sample directions differ only by
// the row's azimuth step.  In the source map (level 0, W0 columns) texel i of a level-m row
// therefore reads each sample at the source coordinate of texel 0 moved right by i * W0 / Wm
// columns.  One block per (level, row): the block computes, once, every kept sample's source
// coordinate for texel 0 (the only equirect mapping in the kernel) and its bilinear weights,
// then every texel of the row sums its samples from the shifted coordinates.  Rows wider than
// kPrefilterSeg texels are split into segments, one block each.
constexpr int kPrefilterMaxSamples = 2048;
constexpr int kPrefilterThreads = 256;
constexpr int kPrefilterTexels = 2;  // texels per thread: a block shades a segment of up to 512 texels of a row
constexpr int kPrefilterSeg = kPrefilterThreads * kPrefilterTexels;

// Sample `sidx` of N for alpha^2 = a2 as (2 h_z h_x, 2 h_z h_y, n.l, -); kept iff n.l > 0.  Both
// compaction passes call this, so they agree on every decision.
__device__ __forceinline__ float4 prefilter_sample(int sidx, float a2, float invN) {
  float xi2 = hammersley_xi2((unsigned)sidx);
  float inv = 1.0f / fmaf(a2 - 1.0f, xi2, 1.0f);
  float ct = sqrtf((1.0f - xi2) * inv), st = sqrtf(a2 * xi2 * inv);
  float sp, cp;
  sincospif(2.0f * (sidx * invN), &sp, &cp);
  return make_float4(2.0f * ct * st * cp, 2.0f * ct * st * sp, fmaf(2.0f * ct, ct, -1.0f), 0.0f);
}

// Source coordinate of a sample direction l in the level-0 map: x = u W0 - 0.5, y = v H0 - 0.5.
__device__ __forceinline__ float2 prefilter_src_xy(float3 l, int W0, int H0) {
  float u, v;
  dir_to_uv(l, u, v);
  return make_float2(fmaf(u, (float)W0, -0.5f), fmaf(v, (float)H0, -0.5f));
}

// Per kept sample, for texel 0 of the row, in order of source row: INT_SHIFT (W0 a multiple of
// Wm) stores the four bilinear weights times n.l and (column, row); otherwise the two row weights
// times n.l and the source x coordinate (the column fraction then varies along the row), and the
// row.  Samples are visited in order of their source row so that consecutive samples read the
// same two rows, which stay in L1 (a deterministic bitonic sort of (row, sample) keys).
template <bool INT_SHIFT>
__global__ void __launch_bounds__(kPrefilterThreads) k_prefilter(MapDev src, ChainDev ch, int N) {
  // dynamic shared memory: N float4 weights, N int2 (column, row), N ushort sorted positions; the
  // sort keys ((source row << 16) | kept-sample index, N unsigned) occupy the weights' space
  // until the records are written
  extern __shared__ __align__(16) float4 s_pf[];
  __shared__ int s_base[kPrefilterMaxSamples / 32 + 1];
  __shared__ float s_wsum[kPrefilterThreads / 32];
  float4* s_w = s_pf;
  int2* s_xy = (int2*)(s_pf + N);
  unsigned short* s_pos = (unsigned short*)(s_xy + N);
  unsigned* s_key = (unsigned*)s_pf;
  const int m = blockIdx.y + 1;
  const int W = ch.W[m], H = ch.H[m];
  const int segs = (W + kPrefilterSeg - 1) / kPrefilterSeg;
  const int j = blockIdx.x / segs, i0 = (blockIdx.x - j * segs) * kPrefilterSeg;
  if (j >= H) return;  // block-uniform
  const int W0 = src.W, H0 = src.H;
  const float r = (float)m / (float)(ch.M - 1);
  const float a2 = r * r * r * r;
  const float invN = 1.0f / N;
  const int groups = (N + 31) / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // kept samples per group of 32, then an exclusive prefix over the groups (sample order)
  for (int gi = warp; gi < groups; gi += kPrefilterThreads / 32) {
    int sidx = gi * 32 + lane;
    bool keep = sidx < N && prefilter_sample(sidx, a2, invN).z > 0.0f;
    unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_base[gi] = __popc(bal);
  }
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int gi = 0; gi < groups; ++gi) {
      int c = s_base[gi];
      s_base[gi] = acc;
      acc += c;
    }
    s_base[groups] = acc;
  }
  __syncthreads();
  const int ns = s_base[groups];
  // the frame of texel 0 of the row: n, T = y x n / |y x n| = (-cos phi0, 0, -sin phi0), B = n x T
  const float3 n = texel_dir(0, j, W, H);
  float sp0, cp0;
  sincospif(2.0f * (0.5f / W) - 1.0f, &sp0, &cp0);
  const float3 T = f3(-cp0, 0.0f, -sp0);
  const float3 B = cross3(n, T);
  // pass A: each kept sample's source row, as a sort key
  for (int gi = warp; gi < groups; gi += kPrefilterThreads / 32) {
    int sidx = gi * 32 + lane;
    float4 e = sidx < N ? prefilter_sample(sidx, a2, invN) : make_float4(0, 0, 0, 0);
    bool keep = sidx < N && e.z > 0.0f;
    unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int q = s_base[gi] + __popc(bal & ((1u << lane) - 1u));
      const float2 xy = prefilter_src_xy(T * e.x + B * e.y + n * e.z, W0, H0);
      const int iy = min(max((int)floorf(xy.y), 0), H0 - 1);
      s_key[q] = ((unsigned)iy << 16) | (unsigned)q;
    }
  }
  int P = 1;
  while (P < ns) P <<= 1;
  for (int q = ns + tid; q < P; q += kPrefilterThreads) s_key[q] = 0xffffffffu;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int q = tid; q < P; q += kPrefilterThreads) {
        const int o = q ^ jj;
        if (o > q) {
          const unsigned a = s_key[q], b = s_key[o];
          if ((a > b) == ((q & k) == 0)) {
            s_key[q] = b;
            s_key[o] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int q = tid; q < ns; q += kPrefilterThreads) s_pos[s_key[q] & 0xffffu] = (unsigned short)q;
  __syncthreads();  // the keys are dead from here: their space takes the records
  // pass B: the records at their sorted positions; the weight sum sum_k n.l_k (the same for every
  // texel of the level), summed in sample order
  float wpart = 0.0f;
  for (int gi = warp; gi < groups; gi += kPrefilterThreads / 32) {
    int sidx = gi * 32 + lane;
    float4 e = sidx < N ? prefilter_sample(sidx, a2, invN) : make_float4(0, 0, 0, 0);
    bool keep = sidx < N && e.z > 0.0f;
    unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int q = s_base[gi] + __popc(bal & ((1u << lane) - 1u));
      const float2 xy = prefilter_src_xy(T * e.x + B * e.y + n * e.z, W0, H0);
      const float xf = floorf(xy.x), yf = floorf(xy.y);
      const float fx = xy.x - xf, fy = xy.y - yf;
      const float wt = e.z * (1.0f - fy), wb = e.z * fy;
      const int p = s_pos[q];
      if (INT_SHIFT)
        s_w[p] = make_float4(wt * (1.0f - fx), wt * fx, wb * (1.0f - fx), wb * fx);
      else
        s_w[p] = make_float4(wt, wb, xy.x, 0.0f);
      s_xy[p] = make_int2((int)xf, (int)yf);
      wpart += e.z;
    }
  }
  wpart = warp_sum(wpart);
  if (lane == 0) s_wsum[warp] = wpart;
  __syncthreads();
  float wsum = 0.0f;
#pragma unroll
  for (int w = 0; w < kPrefilterThreads / 32; ++w) wsum += s_wsum[w];
  const float inv = 1.0f / wsum;
  const int step_i = W0 / W;  // INT_SHIFT: whole source columns per texel
  const float step_f = (float)W0 / (float)W;
  if (INT_SHIFT) {
    // Lanes by tap column: lane l of warp w serves output texels i = i0 + 64 w + 16 g + (l >> 1),
    // g = 0..3, with the tap column d = l & 1 (columns x0 + s i + d), so a warp's loads of one
    // row and group are 32 consecutive texels at level 1 (s = 2); the two lanes of a texel add
    // their sums at the end.
    const int t = lane >> 1, dl = lane & 1;
    const int wbase = i0 + warp * 64;
    if (wbase >= W) return;  // warp-uniform, after the last barrier
    int col[4];
    bool ong[4];
    float3 acc[4], part[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const int i = wbase + 16 * g + t;
      ong[g] = wbase + 16 * g < W;  // warp-uniform: whether group g has texels
      col[g] = min(i, W - 1) * step_i + dl;
      acc[g] = part[g] = f3(0, 0, 0);
    }
#pragma unroll 2
    for (int q = 0; q < ns; ++q) {
      const float4 w = s_w[q];
      const int2 xy = s_xy[q];
      const int r0 = max(xy.y, 0) * W0, r1 = min(xy.y + 1, H0 - 1) * W0;
      const float wa = dl ? w.y : w.x, wb = dl ? w.w : w.z;  // this column's weights in rows r0, r1
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        if (!ong[g]) continue;
        int c = xy.x + col[g];  // in [-1, 2 W0 - 1)
        c = c < 0 ? c + W0 : (c >= W0 ? c - W0 : c);
        const float4 a = __ldg(src.texels + (r0 + c)), p = __ldg(src.texels + (r1 + c));
        part[g].x = fmaf(wa, a.x, fmaf(wb, p.x, part[g].x));
        part[g].y = fmaf(wa, a.y, fmaf(wb, p.y, part[g].y));
        part[g].z = fmaf(wa, a.z, fmaf(wb, p.z, part[g].z));
      }
      if ((q & 63) == 63) {  // fold every 64 samples' plain sums into the running sums
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          acc[g] = acc[g] + part[g];
          part[g] = f3(0, 0, 0);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (!ong[g]) continue;
      float3 v = acc[g] + part[g];
      v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
      v.z += __shfl_xor_sync(0xffffffffu, v.z, 1);
      const int i = wbase + 16 * g + t;
      if (dl == 0 && i < W) {
        const float3 o = v * inv;
        ch.dst[m][(long long)j * W + i] = make_float4(o.x, o.y, o.z, 1.0f);
      }
    }
    return;
  }
  int ii[kPrefilterTexels];
  bool on[kPrefilterTexels];  // block-uniform: whether the segment has a texel group c
  float3 acc[kPrefilterTexels], part[kPrefilterTexels];
#pragma unroll
  for (int c = 0; c < kPrefilterTexels; ++c) {
    on[c] = i0 + c * kPrefilterThreads < W;
    ii[c] = min(i0 + c * kPrefilterThreads + tid, W - 1);  // duplicates of the last texel are not stored
    acc[c] = part[c] = f3(0, 0, 0);
  }
#pragma unroll 2
  for (int q = 0; q < ns; ++q) {
    const float4 w = s_w[q];
    const int2 xy = s_xy[q];
    const int r0 = max(xy.y, 0) * W0, r1 = min(xy.y + 1, H0 - 1) * W0;
#pragma unroll
    for (int c = 0; c < kPrefilterTexels; ++c) {
      if (!on[c]) continue;
      const float x = fmaf((float)ii[c], step_f, w.z);
      const float xf = floorf(x), fx = x - xf;
      int x0 = (int)xf;
      const float4 wq = make_float4(w.x * (1.0f - fx), w.x * fx, w.y * (1.0f - fx), w.y * fx);
      x0 = x0 < 0 ? x0 + W0 : (x0 >= W0 ? x0 - W0 : x0);
      const int x1 = x0 + 1 == W0 ? 0 : x0 + 1;
      const float4 a = __ldg(src.texels + (r0 + x0)), b = __ldg(src.texels + (r0 + x1));
      const float4 p = __ldg(src.texels + (r1 + x0)), d = __ldg(src.texels + (r1 + x1));
      part[c].x = fmaf(wq.x, a.x, fmaf(wq.y, b.x, fmaf(wq.z, p.x, fmaf(wq.w, d.x, part[c].x))));
      part[c].y = fmaf(wq.x, a.y, fmaf(wq.y, b.y, fmaf(wq.z, p.y, fmaf(wq.w, d.y, part[c].y))));
      part[c].z = fmaf(wq.x, a.z, fmaf(wq.y, b.z, fmaf(wq.z, p.z, fmaf(wq.w, d.z, part[c].z))));
    }
    if ((q & 63) == 63) {  // fold every 64 samples' plain sums into the running sums
#pragma unroll
      for (int c = 0; c < kPrefilterTexels; ++c) {
        acc[c] = acc[c] + part[c];
        part[c] = f3(0, 0, 0);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kPrefilterTexels; ++c) {
    const int i = i0 + c * kPrefilterThreads + tid;
    if (on[c] && i < W) {
      const float3 o = (acc[c] + part[c]) * inv;
      ch.dst[m][(long long)j * W + i] = make_float4(o.x, o.y, o.z, 1.0f);
    }
  }
}

static epbr_status validate_ibl_for(const epbr_ibl* ibl, int We, int He) {
  if (!ibl) return fail(EPBR_ERR_INVALID_ARG, "ibl is NULL");
  if (ibl->num_levels < 1 || ibl->num_levels > EPBR_MAX_LEVELS)
    return fail(EPBR_ERR_INVALID_ARG, "ibl->num_levels %d invalid", ibl->num_levels);
  for (int m = 0; m < ibl->num_levels; ++m) {
    int w = std::max(1, We >> m), h = std::max(1, He >> m);
    if (!ibl->level[m] || ibl->level_width[m] != w || ibl->level_height[m] != h)
      return fail(EPBR_ERR_INVALID_ARG, "ibl level %d does not match the env (%dx%d expected)", m, w, h);
    if ((uintptr_t)ibl->level[m] % 16) return fail(EPBR_ERR_INVALID_ARG, "ibl level %d not 16-byte aligned", m);
  }
  return EPBR_OK;
}

}  // namespace epbr

using namespace epbr;

extern "C" epbr_status epbr_brdf_lut(int32_t S, int32_t N, float* lut, void* stream) {
  if (S < 1 || S > 4096 || N < 1 || N > (1 << 24) || !lut)
    return fail(EPBR_ERR_INVALID_ARG, "brdf_lut: size %d / samples %d / pointer invalid", S, N);
  if ((uintptr_t)lut % 8) return fail(EPBR_ERR_INVALID_ARG, "brdf_lut: lut not 8-byte aligned");
  long long threads = (long long)S * S * 32;
  int blocks = (int)((threads + 255) / 256);
  k_brdf_lut<<<blocks, 256, 0, (cudaStream_t)stream>>>(S, N, (float2*)lut);
  epbr_status st = check_launch("k_brdf_lut");
  return st ? st : ok();
}

extern "C" epbr_status epbr_precompute_ibl_workspace_size(const epbr_ibl_params* p, int32_t We,
                                                          int32_t He, size_t* bytes) {
  if (!p || !bytes) return fail(EPBR_ERR_INVALID_ARG, "params or bytes is NULL");
  if (We < 1 || He < 1 || p->irr_width < 1 || p->irr_height < 1)
    return fail(EPBR_ERR_INVALID_ARG, "sizes must be positive");
  *bytes = irr_workspace_bytes(We, He, p->irr_width, p->irr_height);
  return ok();
}

extern "C" epbr_status epbr_irradiance(const epbr_env* env, int32_t Wi, int32_t Hi, float* out,
                                       void* ws, size_t ws_bytes, void* stream) {
  epbr_status st = validate_env(env);
  if (st) return st;
  if (Wi < 1 || Hi < 1 || Wi > 4096 || Hi > 4096 || !out)
    return fail(EPBR_ERR_INVALID_ARG, "irradiance: output %dx%d or pointer invalid", Wi, Hi);
  if ((uintptr_t)out % 16) return fail(EPBR_ERR_INVALID_ARG, "irradiance: out not 16-byte aligned");
  size_t need = irr_workspace_bytes(env->width, env->height, Wi, Hi);
  if (!ws || ws_bytes < need || (uintptr_t)ws % 16)
    return fail(EPBR_ERR_NO_MEMORY, "irradiance: workspace needs %zu bytes (16-byte aligned), got %zu", need,
                ws ? ws_bytes : (size_t)0);
  int nb = irr_blocks(env->width, env->height);
  cudaStream_t s = (cudaStream_t)stream;
  k_irradiance_part<<<nb, kIrrThreads, 0, s>>>((const float4*)env->texels, env->width, env->height, Wi,
                                               Hi, (float4*)ws);
  if ((st = check_launch("k_irradiance_part"))) return st;
  int nout = Wi * Hi;
  k_irradiance_final<<<(unsigned)(((long long)nout * 32 + 255) / 256), 256, 0, s>>>((const float4*)ws, nb, nout,
                                                                                   (float4*)out);
  if ((st = check_launch("k_irradiance_final"))) return st;
  return ok();
}

// ------------------------------------------------------------------------------------------
// Irradiance for callers that cannot allocate: the per-block partial sums go to a fixed,
// library-owned device array instead of caller workspace.
// ------------------------------------------------------------------------------------------
namespace epbr {

constexpr size_t kStaticScratchBytes = (size_t)8 << 20;  // 8 MiB: 32x16 outputs over 608 blocks need 4.75 MiB
static __device__ __align__(256) float4 g_irr_scratch[kStaticScratchBytes / sizeof(float4)];

constexpr int kMaxDevices = 64;

// The array's device address is per context: a caller may run its own driver context on a
// device instead of the primary one, and a device reset gives the device a new primary context
// (with the array loaded afresh).  The cache therefore keeps, per device, the unique id of the
// context the address was looked up in (cuCtxGetId, never reused within a process) and looks
// the address up again when the current context is another one.
struct ScratchSlot {
  unsigned long long ctx_id;
  void* addr;
};
static std::mutex g_scratch_mutex;
static ScratchSlot g_scratch_slot[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

template <typename Fn>
static Fn driver_fn(const char* name) {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return (Fn)f;
}

// Unique id of the calling thread's current context (0 and false when there is none).
static bool current_ctx_id(unsigned long long* id) {
  static const CtxGetCurrentFn get_cur = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
  static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
  CUcontext ctx = nullptr;
  if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_irr_scratch in the current context.  In host code the name g_irr_scratch
// is only a host-side handle, so the address is asked from the runtime (with the device current)
// once per device and context and cached.
static epbr_status static_scratch(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(EPBR_ERR_CUDA, "irradiance_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(EPBR_ERR_UNSUPPORTED, "irradiance_noalloc: device %d", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  unsigned long long id = 0;
  bool have_id = current_ctx_id(&id);
  ScratchSlot& slot = g_scratch_slot[dev];
  if (!have_id || !slot.addr || slot.ctx_id != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_irr_scratch);  // also makes the primary context current if none is
    if (e != cudaSuccess || !p)
      return fail(EPBR_ERR_CUDA, "irradiance_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    if (!have_id && !current_ctx_id(&id))
      return fail(EPBR_ERR_CUDA, "irradiance_noalloc: no current context after the symbol lookup");
    slot.ctx_id = id;
    slot.addr = p;
  }
  *out = slot.addr;
  return EPBR_OK;
}

}  // namespace epbr

extern "C" epbr_status epbr_irradiance_noalloc(const epbr_env* env, int32_t Wi, int32_t Hi, float* out,
                                               void* stream) {
  epbr_status st = validate_env(env);
  if (st) return st;
  if (Wi < 1 || Hi < 1 || Wi > 4096 || Hi > 4096 || !out)
    return fail(EPBR_ERR_INVALID_ARG, "irradiance_noalloc: output %dx%d or pointer invalid", Wi, Hi);
  if ((uintptr_t)out % 16) return fail(EPBR_ERR_INVALID_ARG, "irradiance_noalloc: out not 16-byte aligned");
  size_t need = irr_workspace_bytes(env->width, env->height, Wi, Hi);
  if (need > kStaticScratchBytes)
    return fail(EPBR_ERR_INVALID_ARG,
                "irradiance_noalloc: a %dx%d map over a %dx%d environment needs %zu bytes of scratch; the "
                "static scratch holds %zu (use epbr_irradiance with a workspace)",
                Wi, Hi, env->width, env->height, need, kStaticScratchBytes);
  void* ws = nullptr;
  if ((st = static_scratch(&ws))) return st;
  int nb = irr_blocks(env->width, env->height);
  cudaStream_t s = (cudaStream_t)stream;
  // Every partial the final pass reads is written by the first pass, so the scratch needs no
  // clearing between calls.
  k_irradiance_part<<<nb, kIrrThreads, 0, s>>>((const float4*)env->texels, env->width, env->height, Wi, Hi,
                                               (float4*)ws);
  if ((st = check_launch("k_irradiance_part"))) return st;
  int nout = Wi * Hi;
  k_irradiance_final<<<(unsigned)(((long long)nout * 32 + 255) / 256), 256, 0, s>>>((const float4*)ws, nb, nout,
                                                                                   (float4*)out);
  if ((st = check_launch("k_irradiance_final"))) return st;
  return ok();
}

extern "C" epbr_status epbr_prefilter(const epbr_env* env, int32_t N, const epbr_ibl* ibl, void* stream) {
  epbr_status st = validate_env(env);
  if (st) return st;
  if ((st = validate_ibl_for(ibl, env->width, env->height))) return st;
  if (N < 1 || N > kPrefilterMaxSamples)
    return fail(EPBR_ERR_INVALID_ARG, "prefilter: samples %d outside [1, %d]", N, kPrefilterMaxSamples);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(ibl->level[0], env->texels, (size_t)env->width * env->height * 16,
                      cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "prefilter: level-0 copy failed: %s", cudaGetErrorString(cudaGetLastError()));
  if (ibl->num_levels < 2) return ok();
  ChainDev ch;
  ch.M = ibl->num_levels;
  ch.nlev = ibl->num_levels - 1;
  ch.off[0] = 0;
  for (int m = 0; m < EPBR_MAX_LEVELS; ++m) {
    ch.W[m] = ibl->level_width[m];
    ch.H[m] = ibl->level_height[m];
    ch.dst[m] = (float4*)ibl->level[m];
  }
  for (int li = 0; li < ch.nlev; ++li) ch.off[li + 1] = ch.off[li] + (long long)ch.W[li + 1] * ch.H[li + 1];
  MapDev src{(const float4*)env->texels, env->width, env->height};
  // one block per row of every level (level 1 has the most rows); whole-column shifts when every
  // level's width divides the source width
  bool int_shift = true;
  for (int m = 1; m < ibl->num_levels; ++m) int_shift = int_shift && env->width % ch.W[m] == 0;
  unsigned most = 0;
  for (int m = 1; m < ibl->num_levels; ++m)
    most = std::max(most, (unsigned)(ch.H[m] * ((ch.W[m] + kPrefilterSeg - 1) / kPrefilterSeg)));
  dim3 grid(most, (unsigned)ch.nlev);
  const size_t smem = (size_t)N * (sizeof(float4) + sizeof(int2) + sizeof(unsigned short));
  void (*k)(MapDev, ChainDev, int) = int_shift ? k_prefilter<true> : k_prefilter<false>;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "prefilter: shared-memory attribute: %s", cudaGetErrorString(cudaGetLastError()));
  // a small shared-memory carve-out leaves most of the SM's 256 KB to L1, which holds the source
  // rows the resident blocks read (two rows of up to 16 KB per block)
  cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 50);  // a hint; failure is harmless
  k<<<grid, kPrefilterThreads, smem, s>>>(src, ch, N);
  if ((st = check_launch("k_prefilter"))) return st;
  return ok();
}

extern "C" epbr_status epbr_precompute_ibl(const epbr_env* env, const epbr_ibl_params* p, const epbr_ibl* ibl,
                                           void* ws, size_t ws_bytes, void* stream) {
  epbr_status st = validate_env(env);
  if (st) return st;
  if (!p) return fail(EPBR_ERR_INVALID_ARG, "params is NULL");
  if ((st = validate_ibl_for(ibl, env->width, env->height))) return st;
  if (ibl->num_levels != p->num_levels || ibl->lut_size != p->lut_size || ibl->irr_width != p->irr_width ||
      ibl->irr_height != p->irr_height || !ibl->lut || !ibl->irradiance)
    return fail(EPBR_ERR_INVALID_ARG, "ibl layout does not match params");
  if ((st = epbr_brdf_lut(p->lut_size, p->lut_samples, ibl->lut, stream))) return st;
  if ((st = epbr_irradiance(env, p->irr_width, p->irr_height, ibl->irradiance, ws, ws_bytes, stream))) return st;
  if ((st = epbr_prefilter(env, p->prefilter_samples, ibl, stream))) return st;
  return ok();
}
