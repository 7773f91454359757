// The G-buffer pass of surfel rendering (Sec. 4.3): oriented elliptical disks splatted into the
// FP32 G-buffer, the surfels within a depth window of the nearest one blended.
//   k_surfel_rays     the view-space ray (u_x, u_y, -1) of every pixel column and row
//   k_surfel_setup    one thread per surfel: view-space frame (centre, unit normal, orthogonalised
//                     unit tangent, bitangent), the near rule, and the pixel box of the projected
//                     ellipse (its image conic's extent, widened by 1/8 pixel); a box of more
//                     than 1024 pixels counts as tasks of 1024 pixels (0 tasks for the others)
//   k_surfel_cover    one warp per surfel with a box of at most 1024 pixels, then one warp per
//                     task of the larger boxes (a binary search over the scanned task counts finds
//                     its surfel), the lanes walking the pixels in row order: the ellipse test
//                     multiplied through by (n^.d)^2 (no quotient), the ray-plane depth only for a
//                     covered pixel; pass 0 keeps the smallest depth per pixel (atomicMin on its
//                     bits), pass 1 adds the attributes of every covering surfel inside the depth
//                     window (two float4 atomics and one float atomic per pixel)
//   k_surfel_resolve  one thread per pixel: the weighted means written as the FP32 G-buffer
// The decisions evaluate the oracle's FP32 expressions with each product, sum, quotient and
// square root rounded in the same order, so which pixels a surfel covers, the nearest depth and
// the window reproduce bit for bit; only the attribute sums depend on the order of the atomics.
#include <string.h>

#include <cmath>

#include "epbr_internal.cuh"

namespace epbr {

constexpr int kSurfelChunk = 1024;  // box pixels per warp task

struct SurfelSetup {
  float4 c;   // view-space centre, n^ . c
  float4 n;   // view-space unit normal, 1 / a^2
  float4 t;   // view-space unit tangent, 1 / b^2
  float4 b;   // bitangent n^ x t^, c . t^
  float4 nw;  // world-space unit normal, c . b^
  int4 box;   // x0, y0, width, height
};

struct SurfelCam {
  float axes[9];  // the view axes in world space, axis k at 3 k
  float eye[3];
  float kx, ky, hw, hh, near, f;  // f = 1 + depth tolerance, rounded to FP32
  int W, H;
};

__device__ __forceinline__ float dot_rn(float a0, float a1, float a2, float b0, float b1, float b2) {
  return __fadd_rn(__fadd_rn(__fmul_rn(a0, b0), __fmul_rn(a1, b1)), __fmul_rn(a2, b2));
}

__global__ void __launch_bounds__(256) k_surfel_rays(SurfelCam cam, float* __restrict__ ux, float* __restrict__ uy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float c = __fadd_rn((float)i, 0.5f);
  if (i < cam.W) ux[i] = __fdiv_rn(__fsub_rn(__fdiv_rn(c, cam.hw), 1.0f), cam.kx);
  if (i < cam.H) uy[i] = __fdiv_rn(__fsub_rn(1.0f, __fdiv_rn(c, cam.hh)), cam.ky);
}

__global__ void __launch_bounds__(256) k_surfel_setup(const float4* __restrict__ rec, int N, SurfelCam cam,
                                                      SurfelSetup* __restrict__ setup,
                                                      long long* __restrict__ counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 r0 = __ldg(rec + 4 * (size_t)i), r1 = __ldg(rec + 4 * (size_t)i + 1), r2 = __ldg(rec + 4 * (size_t)i + 2);
  const float inf = __int_as_float(0x7f800000);
  SurfelSetup s;
  memset(&s, 0, sizeof(s));
  long long cnt = 0;
  const float d0 = __fsub_rn(r0.x, cam.eye[0]), d1 = __fsub_rn(r0.y, cam.eye[1]), d2 = __fsub_rn(r0.z, cam.eye[2]);
  float c[3], nv[3], tv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float* ax = cam.axes + 3 * k;
    c[k] = dot_rn(ax[0], ax[1], ax[2], d0, d1, d2);
    nv[k] = dot_rn(ax[0], ax[1], ax[2], r1.x, r1.y, r1.z);
    tv[k] = dot_rn(ax[0], ax[1], ax[2], r2.x, r2.y, r2.z);
  }
  const float a = r0.w, b = r1.w;
  bool ok = a > 0.0f && b > 0.0f && a < inf && b < inf;
  const float nn = dot_rn(nv[0], nv[1], nv[2], nv[0], nv[1], nv[2]);
  ok = ok && nn > 0.0f && nn < inf;
  const float inv = __fdiv_rn(1.0f, __fsqrt_rn(nn));
  const float n0 = __fmul_rn(nv[0], inv), n1 = __fmul_rn(nv[1], inv), n2 = __fmul_rn(nv[2], inv);
  const float dt = dot_rn(tv[0], tv[1], tv[2], n0, n1, n2);
  const float p0 = __fsub_rn(tv[0], __fmul_rn(n0, dt)), p1 = __fsub_rn(tv[1], __fmul_rn(n1, dt)),
              p2 = __fsub_rn(tv[2], __fmul_rn(n2, dt));
  const float tt = dot_rn(p0, p1, p2, p0, p1, p2);
  ok = ok && tt > 0.0f && tt < inf;
  const float invt = __fdiv_rn(1.0f, __fsqrt_rn(tt));
  const float t0 = __fmul_rn(p0, invt), t1 = __fmul_rn(p1, invt), t2 = __fmul_rn(p2, invt);
  const float b0 = __fsub_rn(__fmul_rn(n1, t2), __fmul_rn(n2, t1));
  const float b1 = __fsub_rn(__fmul_rn(n2, t0), __fmul_rn(n0, t2));
  const float b2 = __fsub_rn(__fmul_rn(n0, t1), __fmul_rn(n1, t0));
  ok = ok && __fsub_rn(-c[2], __fadd_rn(a, b)) >= cam.near;
  if (ok) {
    // Pixel box of the projected ellipse (the whole disk lies at eye depth >= near).  With
    // G = [a t^, b b^, c] the disk's boundary is G (cos, sin, 1); M maps view space to
    // homogeneous pixel coordinates taken relative to the projected centre (Xc, Yc), so
    // H = M G maps the unit circle onto the image conic, whose tangent lines l satisfy
    // l^T H D H^T l = 0 with D = diag(1, 1, -1).  The lines X' = x are l = (1, 0, -x): the
    // silhouette's extent along x is the two roots of C00 - 2 x C02 + x^2 C22 = 0 (C = H D H^T),
    // likewise along y.  The box holds every pixel whose centre lies within 1/8 pixel (plus 1e-4
    // of the extent) of that range: FP32 errors of these bounds are below 1e-3 pixel, and pixels
    // that the rounded ellipse test accepts lie within ~1e-6 of the ellipse's size of it.
    const float ec = -c[2];
    const float Xc = cam.hw * (1.0f + cam.kx * c[0] / ec), Yc = cam.hh * (1.0f - cam.ky * c[1] / ec);
    const float g0[3] = {a * t0, b * b0, c[0]}, g1[3] = {a * t1, b * b1, c[1]}, g2[3] = {a * t2, b * b2, c[2]};
    float h0[3], h1[3], h2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      h0[k] = cam.hw * cam.kx * g0[k] + (Xc - cam.hw) * g2[k];
      h1[k] = -cam.hh * cam.ky * g1[k] + (Yc - cam.hh) * g2[k];
      h2[k] = -g2[k];
    }
    auto dd = [](const float* u, const float* v) { return u[0] * v[0] + u[1] * v[1] - u[2] * v[2]; };
    const float C22 = dd(h2, h2);  // a^2 t_z^2 + b^2 b_z^2 - e_c^2 < 0 for a disk in front of the eye
    float lo[2], hi[2];
    const float* hr[2] = {h0, h1};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float C00 = dd(hr[q], hr[q]), C02 = dd(hr[q], h2);
      const float sq = sqrtf(fmaxf(C02 * C02 - C00 * C22, 0.0f));
      const float r0 = (C02 + sq) / C22, r1 = (C02 - sq) / C22;
      const float m = 0.125f + 1e-4f * fabsf(r1 - r0);
      lo[q] = fminf(r0, r1) - m;
      hi[q] = fmaxf(r0, r1) + m;
    }
    float fx0 = fmaxf(ceilf(Xc + lo[0] - 0.5f), 0.0f), fy0 = fmaxf(ceilf(Yc + lo[1] - 0.5f), 0.0f);
    float fx1 = fminf(floorf(Xc + hi[0] - 0.5f), (float)(cam.W - 1));
    float fy1 = fminf(floorf(Yc + hi[1] - 0.5f), (float)(cam.H - 1));
    if (!(C22 < 0.0f)) {  // a disk grazing the eye plane (rounding only): the whole view
      fx0 = fy0 = 0.0f;
      fx1 = (float)(cam.W - 1);
      fy1 = (float)(cam.H - 1);
    }
    if (fx1 >= fx0 && fy1 >= fy0) {  // false for a NaN bound as well
      const int x0 = (int)fx0, y0 = (int)fy0, w = (int)fx1 - x0 + 1, h = (int)fy1 - y0 + 1;
      const long long area = (long long)w * h;
      cnt = area > kSurfelChunk ? (area + kSurfelChunk - 1) / kSurfelChunk : 0;
      const float ia2 = __fdiv_rn(1.0f, __fmul_rn(a, a)), ib2 = __fdiv_rn(1.0f, __fmul_rn(b, b));
      s.c = make_float4(c[0], c[1], c[2], dot_rn(n0, n1, n2, c[0], c[1], c[2]));
      s.n = make_float4(n0, n1, n2, ia2);
      s.t = make_float4(t0, t1, t2, ib2);
      s.b = make_float4(b0, b1, b2, dot_rn(c[0], c[1], c[2], t0, t1, t2));
      const float rw = rsqrtf(fmaf(r1.x, r1.x, fmaf(r1.y, r1.y, r1.z * r1.z)));
      s.nw = make_float4(r1.x * rw, r1.y * rw, r1.z * rw, dot_rn(c[0], c[1], c[2], b0, b1, b2));
      s.box = make_int4(x0, y0, w, h);
    }
  }
  setup[i] = s;
  counts[i] = cnt;
}

// Eye depth at which the pixel ray d = (ux, uy, -1) meets the surfel inside its ellipse, else 0:
// with U = (n^.c)(d.t^) - (n^.d)(c.t^), V likewise with b^, covered when (n^.c)(n^.d) > 0 and
// U^2 / a^2 + V^2 / b^2 <= (n^.d)^2; the depth (n^.c) / (n^.d) is formed only then.
__device__ __forceinline__ float surfel_hit(const SurfelSetup& s, float ux, float uy) {
  const float nd = __fsub_rn(__fadd_rn(__fmul_rn(s.n.x, ux), __fmul_rn(s.n.y, uy)), s.n.z);
  const float dt = __fsub_rn(__fadd_rn(__fmul_rn(s.t.x, ux), __fmul_rn(s.t.y, uy)), s.t.z);
  const float db = __fsub_rn(__fadd_rn(__fmul_rn(s.b.x, ux), __fmul_rn(s.b.y, uy)), s.b.z);
  if (!(__fmul_rn(s.c.w, nd) > 0.0f)) return 0.0f;
  const float U = __fsub_rn(__fmul_rn(s.c.w, dt), __fmul_rn(nd, s.b.w));
  const float V = __fsub_rn(__fmul_rn(s.c.w, db), __fmul_rn(nd, s.nw.w));
  const float e = __fadd_rn(__fmul_rn(__fmul_rn(U, U), s.n.w), __fmul_rn(__fmul_rn(V, V), s.t.w));
  if (!(e <= __fmul_rn(nd, nd))) return 0.0f;
  const float sd = __fdiv_rn(s.c.w, nd);
  return (sd > 0.0f && sd < __int_as_float(0x7f800000)) ? sd : 0.0f;
}

// Pixels first .. last - 1 of surfel i's box (row order), lane `lane` of a warp taking every 32nd.
// Sums per pixel: acc_a (albedo, metal) and acc_b (normal, rough) float4 planes, acc_w weight.
// mat = (albedo, rough) and metal of the surfel (pass 1).
template <int PASS>
__device__ __forceinline__ void surfel_pixels(const SurfelSetup& s, float4 mat, float metal, int first, int last,
                                              int lane, const float* __restrict__ ux, const float* __restrict__ uy,
                                              float f, int W, unsigned* __restrict__ depth,
                                              float4* __restrict__ acc_a, float4* __restrict__ acc_b,
                                              float* __restrict__ acc_w) {
  const int w = s.box.z;
  // pixel first + lane of the box, then steps of 32 = dy rows and dx columns
  int ly = (first + lane) / w, lx = first + lane - ly * w;
  const int dy = 32 / w, dx = 32 - dy * w;
  for (int j = first + lane; j < last; j += 32) {
    const int x = s.box.x + lx, y = s.box.y + ly;
    lx += dx;
    ly += dy;
    if (lx >= w) lx -= w, ++ly;
    const float sd = surfel_hit(s, __ldg(ux + x), __ldg(uy + y));
    if (sd == 0.0f) continue;
    const size_t p = (size_t)y * W + x;
    if (PASS == 0) {
      atomicMin(depth + p, __float_as_uint(sd));  // positive floats order as their bits
      continue;
    }
    if (!(sd <= __fmul_rn(__uint_as_float(depth[p]), f))) continue;
    atomicAdd(acc_a + p, make_float4(mat.x, mat.y, mat.z, metal));
    atomicAdd(acc_b + p, make_float4(s.nw.x, s.nw.y, s.nw.z, mat.w));
    atomicAdd(acc_w + p, 1.0f);
  }
}

template <int PASS>
__global__ void __launch_bounds__(256) k_surfel_cover(const SurfelSetup* __restrict__ setup,
                                                      const long long* __restrict__ offsets, int N,
                                                      const long long* __restrict__ total_p,
                                                      const float* __restrict__ ux, const float* __restrict__ uy,
                                                      const float4* __restrict__ rec, float f, int W,
                                                      unsigned* __restrict__ depth, float4* __restrict__ acc_a,
                                                      float4* __restrict__ acc_b, float* __restrict__ acc_w) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  // boxes of at most kSurfelChunk pixels: one warp each, the next surfel's set-up loaded while the
  // current one's pixels are tested
  // (pass 1: and its material from the records)
  SurfelSetup next;
  float4 next_mat = make_float4(0, 0, 0, 0);
  float next_metal = 0.0f;
  if (warp < N) {
    next = setup[warp];
    if (PASS == 1) next_mat = __ldg(rec + 4 * (size_t)warp + 3), next_metal = __ldg(rec + 4 * (size_t)warp + 2).w;
  }
  for (long long i = warp; i < N; i += warps) {
    const SurfelSetup s = next;
    const float4 mat = next_mat;
    const float metal = next_metal;
    if (i + warps < N) {
      next = setup[i + warps];
      if (PASS == 1)
        next_mat = __ldg(rec + 4 * (size_t)(i + warps) + 3), next_metal = __ldg(rec + 4 * (size_t)(i + warps) + 2).w;
    }
    const int area = s.box.z * s.box.w;
    if (area == 0 || area > kSurfelChunk) continue;
    surfel_pixels<PASS>(s, mat, metal, 0, area, lane, ux, uy, f, W, depth, acc_a, acc_b, acc_w);
  }
  const long long total = *total_p;  // tasks of the larger boxes
  for (long long task = warp; task < total; task += warps) {
    int lo = 0, hi = N - 1;  // the last surfel with offsets[i] <= task (uniform across the warp)
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(offsets + mid) <= task) lo = mid;
      else hi = mid - 1;
    }
    const SurfelSetup s = setup[lo];
    const int first = (int)(task - __ldg(offsets + lo)) * kSurfelChunk;
    const float4 mat = PASS == 1 ? __ldg(rec + 4 * (size_t)lo + 3) : make_float4(0, 0, 0, 0);
    const float metal = PASS == 1 ? __ldg(rec + 4 * (size_t)lo + 2).w : 0.0f;
    surfel_pixels<PASS>(s, mat, metal, first, min(first + kSurfelChunk, s.box.z * s.box.w), lane, ux, uy, f, W, depth,
                        acc_a, acc_b, acc_w);
  }
}

__global__ void __launch_bounds__(256) k_surfel_resolve(const unsigned* __restrict__ depth,
                                                        const float4* __restrict__ acc_a,
                                                        const float4* __restrict__ acc_b,
                                                        const float* __restrict__ acc_w, int W, int H, GbufDev g,
                                                        float* __restrict__ weight, long long weight_pitch) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (x >= W || y >= H) return;
  const size_t p = (size_t)y * W + x;
  float4* rt0 = (float4*)(const_cast<char*>(g.rt[0]) + (size_t)y * g.pitch[0]) + x;
  float4* rt1 = (float4*)(const_cast<char*>(g.rt[1]) + (size_t)y * g.pitch[1]) + x;
  float* dep = (float*)(const_cast<char*>(g.rt[3]) + (size_t)y * g.pitch[3]) + x;
  const float w = acc_w[p];
  if (weight) ((float*)((char*)weight + (size_t)y * weight_pitch))[x] = w;
  if (w == 0.0f) {
    *rt0 = make_float4(0, 0, 0, 0);
    *rt1 = make_float4(0, 0, 0, 0);
    *dep = __int_as_float(0x7f800000);
    return;
  }
  const float iw = 1.0f / w;
  const float4 A = acc_a[p], B = acc_b[p];
  const float nn = fmaf(B.x, B.x, fmaf(B.y, B.y, B.z * B.z));
  const float rn = nn > 0.0f ? rsqrtf(nn) : 0.0f;
  *rt0 = make_float4(A.x * iw, A.y * iw, A.z * iw, A.w * iw);
  *rt1 = make_float4(B.x * rn, B.y * rn, B.z * rn, B.w * iw);
  *dep = __uint_as_float(depth[p]);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SurfelLayout {
  size_t depth, acc, ux, uy, setup, offsets, sums, bytes;
};

static SurfelLayout surfel_layout(long long N, int W, int H) {
  SurfelLayout l;
  const size_t px = (size_t)W * H;
  size_t off = 0;
  l.depth = off;
  off = align256(off + 4 * px);
  l.acc = off;
  off = align256(off + 9 * 4 * px);
  l.ux = off;
  off = align256(off + 4 * (size_t)W);
  l.uy = off;
  off = align256(off + 4 * (size_t)H);
  l.setup = off;
  off = align256(off + sizeof(SurfelSetup) * (size_t)N);
  l.offsets = off;
  off = align256(off + sizeof(long long) * (size_t)(N + 1));
  l.sums = off;
  off = align256(off + sizeof(long long) * (size_t)(scan_num_blocks(N) + 1));
  l.bytes = off;
  return l;
}

}  // namespace epbr

using namespace epbr;

extern "C" epbr_status epbr_surfel_workspace_size(int32_t num_surfels, int32_t width, int32_t height, size_t* bytes) {
  if (!bytes || num_surfels < 0 || num_surfels > (1 << 28) || width < 1 || height < 1 || width > (1 << 15) ||
      height > (1 << 15))
    return fail(EPBR_ERR_INVALID_ARG, "surfels: bytes NULL, num_surfels outside [0, 2^28] or size outside [1, 32768]");
  *bytes = surfel_layout(num_surfels, width, height).bytes;
  return ok();
}

extern "C" epbr_status epbr_surfel_gbuffer(const epbr_surfels* surfels, const epbr_camera* camera, float near_depth,
                                           float depth_tolerance, const epbr_gbuffer* out, float* weight,
                                           int64_t weight_pitch, void* workspace, size_t workspace_bytes,
                                           void* stream) {
  if (!surfels || !out) return fail(EPBR_ERR_INVALID_ARG, "surfels: surfels or gbuffer is NULL");
  epbr_status st = validate_camera(camera, out);
  if (st) return st;
  if (out->format != EPBR_GBUFFER_FP32) return fail(EPBR_ERR_INVALID_ARG, "surfels: the output G-buffer must be FP32");
  if ((st = validate_gbuffer(out, true))) return st;
  const int N = surfels->num_surfels;
  if (N < 0 || N > (1 << 28) || (N > 0 && !surfels->records) || (uintptr_t)surfels->records % 16)
    return fail(EPBR_ERR_INVALID_ARG, "surfels: records NULL, not 16-byte aligned or count outside [0, 2^28]");
  if (!(near_depth > 0.0f) || !std::isfinite(near_depth))
    return fail(EPBR_ERR_INVALID_ARG, "surfels: near must be > 0");
  if (!(depth_tolerance >= 0.0f) || !std::isfinite(depth_tolerance))
    return fail(EPBR_ERR_INVALID_ARG, "surfels: depth tolerance must be finite and >= 0");
  if (weight && (weight_pitch < 4LL * out->width || weight_pitch % 4 || (uintptr_t)weight % 4))
    return fail(EPBR_ERR_INVALID_ARG, "surfels: weight misaligned or pitch too small");
  const int W = out->width, H = out->height;
  const SurfelLayout l = surfel_layout(N, W, H);
  if (!workspace || (uintptr_t)workspace % 256 || workspace_bytes < l.bytes)
    return fail(EPBR_ERR_INVALID_ARG, "surfels: workspace NULL, not 256-byte aligned or below %zu bytes", l.bytes);
  char* ws = (char*)workspace;
  unsigned* depth = (unsigned*)(ws + l.depth);
  float4* acc_a = (float4*)(ws + l.acc);
  float4* acc_b = acc_a + (size_t)W * H;
  float* acc_w = (float*)(acc_b + (size_t)W * H);
  float* ux = (float*)(ws + l.ux);
  float* uy = (float*)(ws + l.uy);
  SurfelSetup* setup = (SurfelSetup*)(ws + l.setup);
  long long* offsets = (long long*)(ws + l.offsets);
  long long* sums = (long long*)(ws + l.sums);
  SurfelCam sc;
  const CamDev cd = make_cam(*camera);
  for (int k = 0; k < 3; ++k) {
    for (int i = 0; i < 3; ++i) sc.axes[3 * k + i] = cd.r[3 * i + k];  // column k of the rotation
    sc.eye[k] = cd.eye[k];
  }
  const double t = std::tan(0.5 * (double)camera->fov_y);
  sc.ky = (float)(1.0 / t);
  sc.kx = (float)((double)H / ((double)W * t));
  sc.hw = (float)(0.5 * W);
  sc.hh = (float)(0.5 * H);
  sc.near = near_depth;
  sc.f = 1.0f + depth_tolerance;
  sc.W = W;
  sc.H = H;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t plane = (size_t)W * H;
  if (cudaMemsetAsync(depth, 0xff, 4 * plane, s) != cudaSuccess || cudaMemsetAsync(acc_a, 0, 36 * plane, s) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "surfels: memset failed");
  const GbufDev gd = make_gbuf(*out);
  if (N > 0) {
    k_surfel_rays<<<(std::max(W, H) + 255) / 256, 256, 0, s>>>(sc, ux, uy);
    k_surfel_setup<<<(N + 255) / 256, 256, 0, s>>>((const float4*)surfels->records, N, sc, setup, offsets);
    launch_exclusive_scan(offsets, N, sums, s);
    const long long* total = sums + scan_num_blocks(N);
    const float4* rec = (const float4*)surfels->records;
    k_surfel_cover<0><<<num_sms() * 8, 256, 0, s>>>(setup, offsets, N, total, ux, uy, rec, sc.f, W, depth, acc_a,
                                                    acc_b, acc_w);
    k_surfel_cover<1><<<num_sms() * 8, 256, 0, s>>>(setup, offsets, N, total, ux, uy, rec, sc.f, W, depth, acc_a,
                                                    acc_b, acc_w);
  }
  dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
  k_surfel_resolve<<<grd, blk, 0, s>>>(depth, acc_a, acc_b, acc_w, W, H, gd, weight, weight_pitch);
  if ((st = check_launch("surfels"))) return st;
  return ok();
}
