// The G-buffer pass of mesh rendering (Sec. 4.1): triangles rasterised into the FP32 G-buffer.
//   k_raster_setup     one thread per triangle: view transform and projection in FP32 with every
//                      operation rounded, vertices snapped to 1/256 px, orientation, pixel
//                      bounding box; the triangle's work item count is its box area (0: culled)
//   k_scan_*           exclusive int64 prefix sum of the item counts (block scan, scan of the
//                      block totals, add)
//   k_raster_cover     one work item per (triangle, box pixel): threads take runs of 8 items (a
//                      binary search for the run's first triangle and for each later one, so runs
//                      of culled triangles cost nothing, and a walk along the box rows), test the pixel
//                      centre with 64-bit integer edge
//                      functions and a top-left rule, and keep the nearest (depth bits, index)
//                      with a 64-bit atomicMin per pixel
//   k_raster_resolve   one thread per pixel: the winning triangle's perspective-correct weights
//                      and interpolated attributes, written as the FP32 G-buffer
//   k_raster_depth     depth-only resolve: the shadow map of a light (Sec. 5.1 renders the scene
//                      "as a depth map" from each point light as from a normal camera)
// The coverage and depth decisions evaluate exactly the expressions of the oracle (integer edge
// functions; FP32 products, sums and quotients each rounded), so the covering triangle of every
// pixel is reproducible bit for bit.
#include <string.h>

#include <algorithm>
#include <cmath>

#include "epbr_internal.cuh"

namespace epbr {

constexpr int kScanThreads = 256, kScanItems = 4, kScanBlock = kScanThreads * kScanItems;
constexpr int kRunItems = 8;

// 64 bytes, two 32-byte sectors for the coverage's read of a triangle
struct TriSetup {
  int4 qab;    // snapped screen positions of a and b (1/256 px)
  int4 qc_xy;  // c, then the box origin x0, y0
  float4 iz;   // 1/z of a, b, c, then the area as a float
  int4 meta;   // box width | height << 16 (each at most 32768), then the vertex indices of a, b, c
};

__device__ __forceinline__ int box_width(const TriSetup& s) { return s.meta.x & 0xffff; }

struct RasterCam {
  float r[9];  // view_to_world rotation, row-major
  float eye[3];
  float kx, ky, hw, hh, near;
  int W, H;
};

// The cameras of a group of views rendered by one set of launches (the lights' shadow maps);
// a single view uses c[0].
constexpr int kMaxViews = 8;
struct RasterCams {
  RasterCam c[kMaxViews];
};

struct RVert {
  float az, iz;
  int qx, qy;
  bool ok;
};

__device__ __forceinline__ RVert raster_vertex(const float* __restrict__ v, const RasterCam& c) {
  float dx = __fsub_rn(v[0], c.eye[0]), dy = __fsub_rn(v[1], c.eye[1]), dz = __fsub_rn(v[2], c.eye[2]);
  // view axis k = column k of the view_to_world rotation: r[k], r[3 + k], r[6 + k]
  float ax = __fadd_rn(__fadd_rn(__fmul_rn(c.r[0], dx), __fmul_rn(c.r[3], dy)), __fmul_rn(c.r[6], dz));
  float ay = __fadd_rn(__fadd_rn(__fmul_rn(c.r[1], dx), __fmul_rn(c.r[4], dy)), __fmul_rn(c.r[7], dz));
  float az = __fadd_rn(__fadd_rn(__fmul_rn(c.r[2], dx), __fmul_rn(c.r[5], dy)), __fmul_rn(c.r[8], dz));
  RVert o;
  float e = -az;
  o.az = az;
  o.iz = __fdiv_rn(1.0f, e);
  float u = __fmul_rn(ax, o.iz), w = __fmul_rn(ay, o.iz);
  float X = __fmul_rn(c.hw, __fadd_rn(1.0f, __fmul_rn(u, c.kx)));
  float Y = __fmul_rn(c.hh, __fsub_rn(1.0f, __fmul_rn(w, c.ky)));
  o.ok = e >= c.near && fabsf(X) < 4194304.0f && fabsf(Y) < 4194304.0f;
  o.qx = o.ok ? __float2int_rn(X * 256.0f) : 0;
  o.qy = o.ok ? __float2int_rn(Y * 256.0f) : 0;
  return o;
}

__device__ __forceinline__ long long edge_fn(long long ax, long long ay, long long bx, long long by, long long px,
                                             long long py) {
  return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

// top-left rule: 0 for an edge whose zero-weight centres belong to the triangle, else 1
__device__ __forceinline__ int edge_excl(int ax, int ay, int bx, int by) {
  int dx = bx - ax, dy = by - ay;
  return (dy < 0 || (dy == 0 && dx > 0)) ? 0 : 1;
}

// blockIdx.y = the view: its set-ups and counts follow the previous views' (entry view * T + t).
__global__ void __launch_bounds__(256) k_raster_setup(const float* __restrict__ verts, int V, const int* __restrict__ tris,
                                                      int T, const __grid_constant__ RasterCams cams,
                                                      TriSetup* __restrict__ setup, long long* __restrict__ counts) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const RasterCam& cam = cams.c[blockIdx.y];
  setup += (size_t)blockIdx.y * T;
  counts += (size_t)blockIdx.y * T;
  int i[3] = {__ldg(tris + 3 * (size_t)t), __ldg(tris + 3 * (size_t)t + 1), __ldg(tris + 3 * (size_t)t + 2)};
  long long cnt = 0;
  TriSetup s;
  memset(&s, 0, sizeof(s));
  if (i[0] >= 0 && i[1] >= 0 && i[2] >= 0 && i[0] < V && i[1] < V && i[2] < V) {
    RVert a = raster_vertex(verts + 12 * (size_t)i[0], cam), b = raster_vertex(verts + 12 * (size_t)i[1], cam),
          c = raster_vertex(verts + 12 * (size_t)i[2], cam);
    long long area = a.ok && b.ok && c.ok ? edge_fn(a.qx, a.qy, b.qx, b.qy, c.qx, c.qy) : 0;
    if (area != 0) {
      int ia = i[0], ib = i[1], ic = i[2];
      if (area < 0) {  // orient so that the area is positive
        RVert tmp = b;
        b = c;
        c = tmp;
        ib = i[2];
        ic = i[1];
        area = -area;
      }
      long long xmin = min(a.qx, min(b.qx, c.qx)), xmax = max(a.qx, max(b.qx, c.qx));
      long long ymin = min(a.qy, min(b.qy, c.qy)), ymax = max(a.qy, max(b.qy, c.qy));
      // pixels whose centre 256 x + 128 lies in [min, max], clipped to the image
      long long x0 = max((xmin - 128 + 255) >> 8, 0LL), x1 = min((xmax - 128) >> 8, (long long)cam.W - 1);
      long long y0 = max((ymin - 128 + 255) >> 8, 0LL), y1 = min((ymax - 128) >> 8, (long long)cam.H - 1);
      if (x1 >= x0 && y1 >= y0) {
        cnt = (x1 - x0 + 1) * (y1 - y0 + 1);
        s.qab = make_int4(a.qx, a.qy, b.qx, b.qy);
        s.qc_xy = make_int4(c.qx, c.qy, (int)x0, (int)y0);
        s.meta = make_int4((int)((x1 - x0 + 1) | ((y1 - y0 + 1) << 16)), ia, ib, ic);
        s.iz = make_float4(a.iz, b.iz, c.iz, __ll2float_rn(area));
      }
    }
  }
  // only triangles with work items are ever read back (the coverage finds a triangle through its
  // non-empty item range, the resolves through a covered pixel's winner), so a culled one writes
  // its count alone: no set-up traffic for the triangles a view does not see
  if (cnt > 0) setup[t] = s;
  counts[t] = cnt;
}

// ---- exclusive int64 scan ------------------------------------------------------------------
__device__ __forceinline__ long long warp_incl_scan(long long v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long n = __shfl_up_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) >= o) v += n;
  }
  return v;
}

// Scans kScanBlock values per block in place (exclusive) and writes the block total.
__global__ void __launch_bounds__(kScanThreads) k_scan_block(long long* __restrict__ data, long long n,
                                                             long long* __restrict__ block_sums) {
  __shared__ long long s_warp[kScanThreads / 32];
  const long long base = (long long)blockIdx.x * kScanBlock + (long long)threadIdx.x * kScanItems;
  long long v[kScanItems], run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? data[base + k] : 0;
    run += v[k];
  }
  long long incl = warp_incl_scan(run);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
    w = warp_incl_scan(w);
    if (lane < kScanThreads / 32) s_warp[lane] = w;
  }
  __syncthreads();
  long long prefix = incl - run + (warp > 0 ? s_warp[warp - 1] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) data[base + k] = prefix;
    prefix += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = prefix;
}

// One block: exclusive scan of the block totals in place; total at sums[nb].
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(long long* __restrict__ sums, int nb) {
  __shared__ long long s_warp[kScanThreads / 32];
  __shared__ long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
    int i = b0 + threadIdx.x;
    long long v = i < nb ? sums[i] : 0;
    long long incl = warp_incl_scan(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      long long w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
      w = warp_incl_scan(w);
      if (lane < kScanThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    long long excl = s_carry + incl - v + (warp > 0 ? s_warp[warp - 1] : 0);
    if (i < nb) sums[i] = excl;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) s_carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = s_carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(long long* __restrict__ data, long long n,
                                                           const long long* __restrict__ sums) {
  const long long base = (long long)blockIdx.x * kScanBlock;
  const long long add = sums[blockIdx.x];
  for (int k = threadIdx.x; k < kScanBlock; k += kScanThreads)
    if (base + k < n) data[base + k] += add;
}

long long scan_num_blocks(long long n) { return (n + kScanBlock - 1) / kScanBlock; }

void launch_exclusive_scan(long long* data, long long n, long long* sums, cudaStream_t s) {
  const long long nb = scan_num_blocks(n);
  k_scan_block<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, sums);
  k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, (int)nb);
  k_scan_add<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, sums);
}

// ---- coverage --------------------------------------------------------------------------------
constexpr int kCoverThreads = 256;

// Threads take runs of 8 consecutive items: a binary search for the first item's triangle, then a
// walk along the box rows and on to the next triangles (each found by a binary search as well:
// a view that culls most triangles leaves long stretches of empty ones between two with items).
// T set-ups of views of Tv triangles each (set-up t: view t / Tv, triangle t % Tv); view v's keys
// start at keys + v * view_px.
__global__ void __launch_bounds__(kCoverThreads) k_raster_cover(const TriSetup* __restrict__ setup,
                                                                const long long* __restrict__ offsets, int T,
                                                                const long long* __restrict__ total_p, int W, int Tv,
                                                                long long view_px,
                                                                unsigned long long* __restrict__ keys) {
  const long long total = *total_p;
  const long long runs = (total + kRunItems - 1) / kRunItems;
  for (long long run = blockIdx.x * (long long)blockDim.x + threadIdx.x; run < runs;
       run += (long long)gridDim.x * blockDim.x) {
    long long item = run * kRunItems;
    int lo = 0, hi = T - 1;  // the last t with offsets[t] <= item
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (__ldg(offsets + mid) <= item) lo = mid;
      else hi = mid - 1;
    }
    int t = lo;
    long long t_begin = __ldg(offsets + t);
    long long t_end = t + 1 < T ? __ldg(offsets + t + 1) : total;
    TriSetup s = setup[t];
    const long long stop = min(item + kRunItems, total);
    int lx = 0, ly = 0;
    bool fresh = true;
    long long wc = 0, wa = 0, wb = 0;     // edge functions at the current pixel centre
    long long dc = 0, da = 0, db = 0;     // their change per pixel along a row
    for (; item < stop; ++item) {
      if (item >= t_end) {  // the next triangle with items
        ++t;
        t_begin = t_end;
        t_end = t + 1 < T ? __ldg(offsets + t + 1) : total;
        if (item >= t_end) {  // t has no items either: a binary search skips the stretch of empty ones
          int a = t + 1, b = T - 1;  // the last t' with offsets[t'] <= item
          while (a < b) {
            int mid = (a + b + 1) >> 1;
            if (__ldg(offsets + mid) <= item) a = mid;
            else b = mid - 1;
          }
          t = a;
          t_begin = __ldg(offsets + t);
          t_end = t + 1 < T ? __ldg(offsets + t + 1) : total;
        }
        s = setup[t];
        fresh = true;
      }
      if (fresh) {  // position of this item in the triangle's box
        const long long local = item - t_begin;
        ly = (int)(local / box_width(s));
        lx = (int)(local - (long long)ly * box_width(s));
        // E(p) = (b.x - a.x)(p.y - a.y) - (b.y - a.y)(p.x - a.x): a step of one pixel in x adds
        // -256 (b.y - a.y)
        dc = -256LL * (s.qab.w - s.qab.y);
        da = -256LL * (s.qc_xy.y - s.qab.w);
        db = -256LL * (s.qab.y - s.qc_xy.y);
      }
      const int x = s.qc_xy.z + lx, y = s.qc_xy.w + ly;
      if (fresh || lx == 0) {  // a run's first item, a new triangle or a new box row: evaluate
        const long long px = 256LL * x + 128, py = 256LL * y + 128;
        wc = edge_fn(s.qab.x, s.qab.y, s.qab.z, s.qab.w, px, py);
        wa = edge_fn(s.qab.z, s.qab.w, s.qc_xy.x, s.qc_xy.y, px, py);
        wb = edge_fn(s.qc_xy.x, s.qc_xy.y, s.qab.x, s.qab.y, px, py);
        fresh = false;
      } else {
        wc += dc;
        wa += da;
        wb += db;
      }
      if (++lx == box_width(s)) lx = 0, ++ly;
      if (wc < 0 || wa < 0 || wb < 0) continue;
      if ((wc == 0 && edge_excl(s.qab.x, s.qab.y, s.qab.z, s.qab.w)) ||
          (wa == 0 && edge_excl(s.qab.z, s.qab.w, s.qc_xy.x, s.qc_xy.y)) ||
          (wb == 0 && edge_excl(s.qc_xy.x, s.qc_xy.y, s.qab.x, s.qab.y)))
        continue;
      float s0 = __fmul_rn(__ll2float_rn(wa), s.iz.x), s1 = __fmul_rn(__ll2float_rn(wb), s.iz.y);
      float s2 = __fmul_rn(__ll2float_rn(wc), s.iz.z);
      float z = __fdiv_rn(s.iz.w, __fadd_rn(__fadd_rn(s0, s1), s2));
      const int v = t / Tv, tri = t - v * Tv;
      unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | (unsigned)tri;
      atomicMin(keys + (size_t)v * view_px + (size_t)y * W + x, key);
    }
  }
}

// ---- resolve ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_raster_resolve(const float* __restrict__ verts,
                                                        const TriSetup* __restrict__ setup,
                                                        const unsigned long long* __restrict__ keys, int W, int H,
                                                        GbufDev g, int* __restrict__ ids, long long ids_pitch) {
  int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (x >= W || y >= H) return;
  unsigned long long key = keys[(size_t)y * W + x];
  float4* rt0 = (float4*)(const_cast<char*>(g.rt[0]) + (size_t)y * g.pitch[0]) + x;
  float4* rt1 = (float4*)(const_cast<char*>(g.rt[1]) + (size_t)y * g.pitch[1]) + x;
  float* dep = (float*)(const_cast<char*>(g.rt[3]) + (size_t)y * g.pitch[3]) + x;
  int* idp = ids ? (int*)((char*)ids + (size_t)y * ids_pitch) + x : nullptr;
  if (key == ~0ULL) {
    *rt0 = make_float4(0, 0, 0, 0);
    *rt1 = make_float4(0, 0, 0, 0);
    *dep = __int_as_float(0x7f800000);
    if (idp) *idp = -1;
    return;
  }
  const int t = (int)(key & 0xffffffffULL);
  const TriSetup s = setup[t];
  const long long px = 256LL * x + 128, py = 256LL * y + 128;
  // perspective-correct weights b_i / z_i normalised, from the exact edge functions
  float wa = __ll2float_rn(edge_fn(s.qab.z, s.qab.w, s.qc_xy.x, s.qc_xy.y, px, py)) * s.iz.x;
  float wb = __ll2float_rn(edge_fn(s.qc_xy.x, s.qc_xy.y, s.qab.x, s.qab.y, px, py)) * s.iz.y;
  float wc = __ll2float_rn(edge_fn(s.qab.x, s.qab.y, s.qab.z, s.qab.w, px, py)) * s.iz.z;
  const float inv = rcp_ftz(wa + wb + wc);
  wa *= inv;
  wb *= inv;
  wc *= inv;
  // vertex values 3 .. 10 (normal, albedo, metal, rough) read as three float4 of each 48-byte
  // record (16-byte aligned, checked on the host): normal.x is the w of the first, normal.yz and
  // albedo.rg fill the second, albedo.b, metal and rough lead the third
  const float4* A = (const float4*)(verts + 12 * (size_t)s.meta.y);
  const float4* B = (const float4*)(verts + 12 * (size_t)s.meta.z);
  const float4* C = (const float4*)(verts + 12 * (size_t)s.meta.w);
  float at[8];
  {
    const float4 a0 = __ldg(A), a1 = __ldg(A + 1), a2 = __ldg(A + 2);
    const float4 b0 = __ldg(B), b1 = __ldg(B + 1), b2 = __ldg(B + 2);
    const float4 c0 = __ldg(C), c1 = __ldg(C + 1), c2 = __ldg(C + 2);
    const float va[8] = {a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z};
    const float vb[8] = {b0.w, b1.x, b1.y, b1.z, b1.w, b2.x, b2.y, b2.z};
    const float vc[8] = {c0.w, c1.x, c1.y, c1.z, c1.w, c2.x, c2.y, c2.z};
#pragma unroll
    for (int q = 0; q < 8; ++q) at[q] = fmaf(wa, va[q], fmaf(wb, vb[q], wc * vc[q]));
  }
  float3 n = f3(at[0], at[1], at[2]);
  n = n * rsqrt_ftz(dot3(n, n));
  *rt0 = make_float4(at[3], at[4], at[5], at[6]);
  *rt1 = make_float4(n.x, n.y, n.z, at[7]);
  *dep = __uint_as_float((unsigned)(key >> 32));
  if (idp) *idp = t;
}

// Depth-only resolve (shadow maps, Sec. 5.1): the winning triangle's eye depth, +inf where no
// triangle covers the texel.
__global__ void __launch_bounds__(256) k_raster_depth(const unsigned long long* __restrict__ keys, int W, int H,
                                                      float* __restrict__ out, long long pitch) {
  int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (x >= W || y >= H) return;
  keys += (size_t)blockIdx.z * W * H;  // view blockIdx.z: dense W x H images
  out = (float*)((char*)out + (size_t)blockIdx.z * H * pitch);
  const unsigned long long key = keys[(size_t)y * W + x];
  ((float*)((char*)out + (size_t)y * pitch))[x] =
      key == ~0ULL ? __int_as_float(0x7f800000) : __uint_as_float((unsigned)(key >> 32));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct RasterLayout {
  size_t keys, setup, offsets, sums, bytes;
};

// The workspace of `views` views of W x H pixels and T triangles each.
static RasterLayout raster_layout(long long T, int W, int H, int views = 1) {
  RasterLayout l;
  size_t off = 0;
  const long long n = T * views;
  l.keys = off;
  off = align256(off + sizeof(unsigned long long) * (size_t)W * H * views);
  l.setup = off;
  off = align256(off + sizeof(TriSetup) * (size_t)n);
  l.offsets = off;
  off = align256(off + sizeof(long long) * (size_t)(n + 1));
  l.sums = off;
  long long nb = scan_num_blocks(n);
  off = align256(off + sizeof(long long) * (size_t)(nb + 1));
  l.bytes = off;
  return l;
}

}  // namespace epbr

using namespace epbr;

extern "C" epbr_status epbr_raster_workspace_size(int32_t num_triangles, int32_t width, int32_t height, size_t* bytes) {
  if (!bytes || num_triangles < 0 || width < 1 || height < 1 || width > (1 << 15) || height > (1 << 15))
    return fail(EPBR_ERR_INVALID_ARG, "raster: bytes NULL, num_triangles < 0 or size outside [1, 32768]");
  *bytes = raster_layout(num_triangles, width, height).bytes;
  return ok();
}

namespace epbr {

static epbr_status validate_mesh(const epbr_mesh* mesh, float near_depth) {
  if (mesh->num_vertices < 0 || mesh->num_triangles < 0 || mesh->num_vertices > (1 << 28) ||
      (mesh->num_triangles > 0 && (!mesh->vertices || !mesh->triangles)) || (uintptr_t)mesh->vertices % 16 ||
      (uintptr_t)mesh->triangles % 4)
    return fail(EPBR_ERR_INVALID_ARG, "raster: vertices / triangles NULL, misaligned or counts out of range");
  if (!(near_depth > 0.0f) || !std::isfinite(near_depth)) return fail(EPBR_ERR_INVALID_ARG, "raster: near must be > 0");
  return EPBR_OK;
}

static RasterCam make_raster_cam(const epbr_camera& camera, float near_depth) {
  RasterCam rc;
  CamDev cd = make_cam(camera);
  for (int i = 0; i < 9; ++i) rc.r[i] = cd.r[i];
  for (int i = 0; i < 3; ++i) rc.eye[i] = cd.eye[i];
  const int W = camera.width, H = camera.height;
  double t = std::tan(0.5 * (double)camera.fov_y);
  rc.ky = (float)(1.0 / t);
  rc.kx = (float)((double)H / ((double)W * t));
  rc.hw = (float)(0.5 * W);
  rc.hh = (float)(0.5 * H);
  rc.near = near_depth;
  rc.W = W;
  rc.H = H;
  return rc;
}

// Set-up, scan and coverage of the mesh seen by `views` cameras (same size): the nearest (depth,
// triangle) key of every pixel of every view in the workspace's key images.
static epbr_status raster_keys(const epbr_mesh* mesh, const RasterCams& rc, int views, const RasterLayout& l,
                               char* ws, cudaStream_t s) {
  const int T = mesh->num_triangles;
  const int W = rc.c[0].W, H = rc.c[0].H;
  unsigned long long* keys = (unsigned long long*)(ws + l.keys);
  TriSetup* setup = (TriSetup*)(ws + l.setup);
  long long* offsets = (long long*)(ws + l.offsets);
  long long* sums = (long long*)(ws + l.sums);
  if (cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * (size_t)W * H * views, s) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "raster: memset failed");
  if (T > 0) {
    const long long n = (long long)T * views;
    k_raster_setup<<<dim3((T + 255) / 256, views), 256, 0, s>>>(mesh->vertices, mesh->num_vertices, mesh->triangles,
                                                                T, rc, setup, offsets);
    const long long nb = scan_num_blocks(n);
    launch_exclusive_scan(offsets, n, sums, s);
    k_raster_cover<<<num_sms() * 8, kCoverThreads, 0, s>>>(setup, offsets, (int)n, sums + nb, W, T, (long long)W * H,
                                                          keys);
  }
  return EPBR_OK;
}

}  // namespace epbr

extern "C" epbr_status epbr_raster_gbuffer(const epbr_mesh* mesh, const epbr_camera* camera, float near_depth,
                                           const epbr_gbuffer* out, int32_t* ids, int64_t ids_pitch, void* workspace,
                                           size_t workspace_bytes, void* stream) {
  if (!mesh || !out) return fail(EPBR_ERR_INVALID_ARG, "raster: mesh or gbuffer is NULL");
  epbr_status st = validate_camera(camera, out);
  if (st) return st;
  if (out->format != EPBR_GBUFFER_FP32) return fail(EPBR_ERR_INVALID_ARG, "raster: the output G-buffer must be FP32");
  if ((st = validate_gbuffer(out, true))) return st;
  if ((st = validate_mesh(mesh, near_depth))) return st;
  if (ids && (ids_pitch < 4LL * out->width || ids_pitch % 4 || (uintptr_t)ids % 4))
    return fail(EPBR_ERR_INVALID_ARG, "raster: ids misaligned or pitch too small");
  const int W = out->width, H = out->height, T = mesh->num_triangles;
  RasterLayout l = raster_layout(T, W, H);
  if (!workspace || (uintptr_t)workspace % 256 || workspace_bytes < l.bytes)
    return fail(EPBR_ERR_INVALID_ARG, "raster: workspace NULL, not 256-byte aligned or below %zu bytes", l.bytes);
  char* ws = (char*)workspace;
  cudaStream_t s = (cudaStream_t)stream;
  RasterCams rc;
  rc.c[0] = make_raster_cam(*camera, near_depth);
  if ((st = raster_keys(mesh, rc, 1, l, ws, s))) return st;
  GbufDev gd = make_gbuf(*out);
  dim3 blk(32, 8), grd((W + 31) / 32, (H + 7) / 8);
  k_raster_resolve<<<grd, blk, 0, s>>>(mesh->vertices, (const TriSetup*)(ws + l.setup),
                                       (const unsigned long long*)(ws + l.keys), W, H, gd, ids, ids_pitch);
  if ((st = check_launch("raster"))) return st;
  return ok();
}

extern "C" epbr_status epbr_shadow_maps_workspace_size(int32_t num_triangles, int32_t size, size_t* bytes) {
  if (!bytes || num_triangles < 0 || size < 1 || size > (1 << 15))
    return fail(EPBR_ERR_INVALID_ARG, "shadow_maps: bytes NULL, num_triangles < 0 or size outside [1, 32768]");
  *bytes = raster_layout(num_triangles, size, size, kMaxViews).bytes;
  return ok();
}

extern "C" epbr_status epbr_shadow_maps(const epbr_mesh* mesh, const epbr_camera* cameras, int32_t num_maps,
                                        float near_depth, float* maps, void* workspace, size_t workspace_bytes,
                                        void* stream) {
  if (!mesh || !cameras || num_maps < 0 || (num_maps > 0 && !maps) || (uintptr_t)maps % 4)
    return fail(EPBR_ERR_INVALID_ARG, "shadow_maps: mesh, cameras or maps NULL / misaligned, or num_maps < 0");
  if (num_maps == 0) return ok();
  epbr_status st = validate_mesh(mesh, near_depth);
  if (st) return st;
  const int S = cameras[0].width;
  for (int i = 0; i < num_maps; ++i) {
    const epbr_camera& c = cameras[i];
    if (c.width != S || c.height != S || S < 1 || S > (1 << 15) || !(c.fov_y > 0.0f && c.fov_y < 3.1f))
      return fail(EPBR_ERR_INVALID_ARG, "shadow_maps: camera %d must be square, of the first camera's size (%d), "
                                        "with a field of view in (0, 3.1) rad", i, S);
    for (int k = 0; k < 16; ++k)
      if (!std::isfinite(c.view_to_world[k])) return fail(EPBR_ERR_INVALID_ARG, "shadow_maps: camera %d not finite", i);
  }
  const long long T = mesh->num_triangles;
  if (T * kMaxViews >= (1LL << 31))
    return fail(EPBR_ERR_UNSUPPORTED, "shadow_maps: %lld triangles x %d views exceed 2^31 set-ups", T, kMaxViews);
  const RasterLayout full = raster_layout(T, S, S, kMaxViews);
  if (!workspace || (uintptr_t)workspace % 256 || workspace_bytes < full.bytes)
    return fail(EPBR_ERR_INVALID_ARG, "shadow_maps: workspace NULL, not 256-byte aligned or below %zu bytes",
                full.bytes);
  char* ws = (char*)workspace;
  cudaStream_t s = (cudaStream_t)stream;
  for (int i0 = 0; i0 < num_maps; i0 += kMaxViews) {  // up to kMaxViews lights per set of launches
    const int views = std::min(kMaxViews, num_maps - i0);
    const RasterLayout l = raster_layout(T, S, S, views);
    RasterCams rc;
    for (int v = 0; v < views; ++v) rc.c[v] = make_raster_cam(cameras[i0 + v], near_depth);
    if ((st = raster_keys(mesh, rc, views, l, ws, s))) return st;
    dim3 blk(32, 8), grd((S + 31) / 32, (S + 7) / 8, views);
    k_raster_depth<<<grd, blk, 0, s>>>((const unsigned long long*)(ws + l.keys), S, S, maps + (size_t)i0 * S * S,
                                       4LL * S);
  }
  if ((st = check_launch("shadow_maps"))) return st;
  return ok();
}
