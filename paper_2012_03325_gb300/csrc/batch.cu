// Many views in one graph launch (the batching form of the pass).
//
// k_batch: 256-thread blocks pull tiles of TW x TH pixels from an atomic counter over a tile
// list that spans every view (views with the most light work first).  Per tile, without leaving
// the SM:
//   1. unblurred AO for the tile's (TW/2) x (TH/2) half-resolution texels plus an R-texel halo,
//      into shared memory (Sec. 5.2; the halo texels are recomputed by neighbouring tiles);
//   2. the depth-aware blur of the tile's texels, from shared memory;
//   3. compose of every pixel (shade_core.cuh) with its view's lights staged in shared memory
//      and its lighting set, AO read from shared memory, tone map fused, stores.
// The counter is reset by a memset node and the kernel launched by a kernel node of one CUDA
// graph, built explicitly and replayed per frame.
// Staged plan: k_mv_ssao_raw, k_mv_ssao_blur and k_mv_shade, each one launch over the tiles of
// every view, joined by programmatic edges in an explicitly built graph.
// Per-view plan: the per-view entry points of every view recorded into the graph by stream
// capture (the only plan built that way).
// epbr_batch_autotune times the fused tile shapes and light-chunk sizes, the staged and the
// per-view plan on the batch itself and keeps the fastest.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "shade_core.cuh"
#include "ssao_core.cuh"

namespace epbr {

constexpr int kBatchThreads = 256;
constexpr int kBatchMaxR = 4;         // blur radius the fused tile supports
constexpr int kBatchMaxK = 64;        // SSAO samples the fused tile supports

struct ViewDev {
  GbufDev g;
  CamDev cam;
  const float4* lights;
  int NL, ibl, tiles_x, ao_w;  // ao_w: AO texels per row (staged mode)
  void* hdr;
  long long hdr_pitch;
  uint8_t* ldr;
  long long ldr_pitch;
  float* ao_raw;  // staged mode: the view's unblurred and blurred AO images (batch-owned)
  float* ao;
};

struct BatchDev {
  unsigned flags;
  int hdr_format;
  float exposure;
  int op;
  int light_chunk;
  SsaoDev ssao;
};

template <int FMT, int TW, int TH>
__global__ void __launch_bounds__(kBatchThreads, 2)
    k_batch(const ViewDev* __restrict__ views, const IblDev* __restrict__ ibls, const int4* __restrict__ tiles,
            int ntiles, int* __restrict__ counter, BatchDev bp) {
  constexpr int AW = TW / 2, AH = TH / 2;
  constexpr int RW = AW + 2 * kBatchMaxR, RH = AH + 2 * kBatchMaxR;
  constexpr int PPT = TW * TH / kBatchThreads;  // pixels per thread, taken in pairs
  static_assert(TW * TH % (2 * kBatchThreads) == 0, "tile must be a multiple of two blocks of pixels");
  __shared__ float s_raw[RH * RW];
  __shared__ float s_e[RH * RW];
  __shared__ float s_ao[AH * AW];
  __shared__ float4 s_lights[2 * kLightChunk];
  __shared__ float4 s_dup[2 * kLightChunk];
  __shared__ float4 s_kernel[kBatchMaxK];
  __shared__ ViewDev s_view;
  __shared__ IblDev s_ibl;
  __shared__ int s_tile;
  __shared__ int s_mono;

  const int tid = threadIdx.x;
  const int R = bp.ssao.R;
  const int rw = AW + 2 * R, rh = AH + 2 * R;
  for (int k = tid; k < bp.ssao.K; k += kBatchThreads) s_kernel[k] = __ldg(bp.ssao.kernel + k);
  int cur_view = -1;
  const float inf = __int_as_float(0x7f800000);
  for (;;) {
    __syncthreads();  // the previous tile is done with shared memory
    if (tid == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) break;
    const int4 td = __ldg(tiles + t);
    if (td.x != cur_view) {  // block-uniform: stage the view, its lighting set and its lights
      const int* src = (const int*)(views + td.x);
      for (int q = tid; q < (int)(sizeof(ViewDev) / 4); q += kBatchThreads) ((int*)&s_view)[q] = __ldg(src + q);
      __syncthreads();
      const int* isrc = (const int*)(ibls + s_view.ibl);
      for (int q = tid; q < (int)(sizeof(IblDev) / 4); q += kBatchThreads) ((int*)&s_ibl)[q] = __ldg(isrc + q);
      int nl = s_view.NL;
      bool mono = true;
      if (nl <= bp.light_chunk) mono = stage_lights(s_lights, s_view.lights, 0, nl, tid, kBatchThreads, s_dup);
      mono = __syncthreads_and(mono);
      if (tid == 0) s_mono = mono;
      cur_view = td.x;
      __syncthreads();
    }
    const ViewDev& v = s_view;
    const int W = v.g.W, H = v.g.H;
    const int Wa = (W + 1) / 2, Ha = (H + 1) / 2;
    const int x0 = td.y * TW, y0 = td.z * TH;
    const int i0 = x0 / 2 - R, j0 = y0 / 2 - R;
    // 1. unblurred AO with halo
    for (int q = tid; q < rw * rh; q += kBatchThreads) {
      int ty = q / rw, tx = q - ty * rw;
      int i = i0 + tx, j = j0 + ty;
      float2 r = make_float2(0.0f, inf);
      if (i >= 0 && i < Wa && j >= 0 && j < Ha) r = ssao_texel<FMT>(v.g, v.cam, bp.ssao, s_kernel, i, j);
      s_raw[ty * RW + tx] = r.x;
      s_e[ty * RW + tx] = r.y;
    }
    __syncthreads();
    // 2. blur of the tile's own texels
    for (int q = tid; q < AW * AH; q += kBatchThreads) {
      int ty = q / AW, tx = q - ty * AW;
      int c = (ty + R) * RW + tx + R;
      s_ao[q] = (x0 / 2 + tx < Wa && y0 / 2 + ty < Ha) ? ssao_blur_texel(bp.ssao, s_raw + c, s_e + c, RW) : 1.0f;
    }
    __syncthreads();
    // 3. compose + tone map, two pixels per thread at a time
    const int nl = v.NL;
    const bool staged = nl <= bp.light_chunk;
    for (int k = 0; k < PPT; k += 2) {
      int xs[2], ys[2], pxs[2], pys[2];
      bool in[2], act[2];
      Px s[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int q = tid + (k + h) * kBatchThreads;
        pys[h] = q / TW;
        pxs[h] = q - pys[h] * TW;
        xs[h] = x0 + pxs[h];
        ys[h] = y0 + pys[h];
        in[h] = xs[h] < W && ys[h] < H;
        if (in[h]) s[h] = px_setup<FMT>(v.g, v.cam, xs[h], ys[h]);
        act[h] = in[h] && s[h].surface;
      }
      shade_lights(s, act, nl, bp.flags, v.lights, s_lights, s_dup, bp.light_chunk, staged, s_mono != 0, tid,
                   kBatchThreads);
      float3 c[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float ao = act[h] ? s_ao[(pys[h] >> 1) * AW + (pxs[h] >> 1)] : 1.0f;
        if (in[h]) c[h] = px_finish(s[h], s_ibl, bp.flags, ao);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!in[h]) continue;
        if (v.hdr) {
          if (bp.hdr_format == EPBR_HDR_RGBA32F)
            store_hdr<EPBR_HDR_RGBA32F>(v.hdr, v.hdr_pitch, xs[h], ys[h], c[h]);
          else
            store_hdr<EPBR_HDR_RGBA16F>(v.hdr, v.hdr_pitch, xs[h], ys[h], c[h]);
        }
        ((unsigned*)(v.ldr + (size_t)ys[h] * v.ldr_pitch))[xs[h]] = pack_rgba8(c[h], bp.exposure, bp.op);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Staged mode: the three stages of the per-view pipeline, each one launch over a tile list that
// spans every view (one tile per block: 32x8 AO texels, 32x16 pixels for the compose; tiles of
// the costliest views first).
// ------------------------------------------------------------------------------------------
constexpr int kMvBX = 32, kMvBY = 8;
constexpr int kMvTileH = 2 * kMvBY;  // compose tiles: 32 x 16 pixels, two per thread

// Copies view td.x (and, when `with_ibl`, its lighting set) into shared memory.
__device__ __forceinline__ void mv_stage_view(const ViewDev* views, const IblDev* ibls, int vi, ViewDev& s_view,
                                              IblDev* s_ibl, int tid, int nthreads) {
  const int* src = (const int*)(views + vi);
  for (int q = tid; q < (int)(sizeof(ViewDev) / 4); q += nthreads) ((int*)&s_view)[q] = __ldg(src + q);
  __syncthreads();
  if (s_ibl) {
    const int* isrc = (const int*)(ibls + s_view.ibl);
    for (int q = tid; q < (int)(sizeof(IblDev) / 4); q += nthreads) ((int*)s_ibl)[q] = __ldg(isrc + q);
  }
}

template <int FMT>
__global__ void __launch_bounds__(kMvBX* kMvBY, 4)
    k_mv_ssao_raw(const ViewDev* __restrict__ views, const int4* __restrict__ tiles, BatchDev bp) {
  __shared__ float4 s_kernel[kBatchMaxK];
  __shared__ ViewDev s_view;
  int tid = threadIdx.y * kMvBX + threadIdx.x;
  griddep_launch_dependents();  // the blur may put its blocks beside this grid's last wave
  int4 td = __ldg(tiles + blockIdx.x);
  for (int k = tid; k < bp.ssao.K; k += kMvBX * kMvBY) s_kernel[k] = __ldg(bp.ssao.kernel + k);
  mv_stage_view(views, nullptr, td.x, s_view, nullptr, tid, kMvBX * kMvBY);
  __syncthreads();
  int Wa = (s_view.g.W + 1) / 2, Ha = (s_view.g.H + 1) / 2;
  int i = td.y * kMvBX + threadIdx.x, j = td.z * kMvBY + threadIdx.y;
  if (i >= Wa || j >= Ha) return;
  s_view.ao_raw[(size_t)j * s_view.ao_w + i] = ssao_texel<FMT>(s_view.g, s_view.cam, bp.ssao, s_kernel, i, j).x;
}

template <int FMT>
__global__ void __launch_bounds__(kMvBX* kMvBY) k_mv_ssao_blur(const ViewDev* __restrict__ views,
                                                               const int4* __restrict__ tiles, BatchDev bp) {
  constexpr int TWd = kMvBX + 2 * kBatchMaxR, THd = kMvBY + 2 * kBatchMaxR;
  __shared__ float s_ao[THd * TWd];
  __shared__ float s_e[THd * TWd];
  __shared__ ViewDev s_view;
  // after the raw pass by a programmatic edge: nothing is read before it has finished, and the
  // compose may start once every block is past this point
  griddep_wait();
  griddep_launch_dependents();
  int tid = threadIdx.y * kMvBX + threadIdx.x;
  int4 td = __ldg(tiles + blockIdx.x);
  mv_stage_view(views, nullptr, td.x, s_view, nullptr, tid, kMvBX * kMvBY);
  __syncthreads();
  const int R = bp.ssao.R;
  int Wa = (s_view.g.W + 1) / 2, Ha = (s_view.g.H + 1) / 2;
  int tw = kMvBX + 2 * R, th = kMvBY + 2 * R;
  int i0 = td.y * kMvBX - R, j0 = td.z * kMvBY - R;
  const float inf = __int_as_float(0x7f800000);
  for (int q = tid; q < tw * th; q += kMvBX * kMvBY) {
    int ty = q / tw, tx = q - ty * tw;
    int qi = i0 + tx, qj = j0 + ty;
    float a = 0.0f, e = inf;
    if (qi >= 0 && qi < Wa && qj >= 0 && qj < Ha) {
      a = s_view.ao_raw[(size_t)qj * s_view.ao_w + qi];
      e = gb_depth(s_view.g, 2 * qi, 2 * qj);
    }
    s_ao[ty * TWd + tx] = a;
    s_e[ty * TWd + tx] = e;
  }
  __syncthreads();
  int i = td.y * kMvBX + threadIdx.x, j = td.z * kMvBY + threadIdx.y;
  if (i >= Wa || j >= Ha) return;
  int c = (threadIdx.y + R) * TWd + threadIdx.x + R;
  s_view.ao[(size_t)j * s_view.ao_w + i] = ssao_blur_texel(bp.ssao, s_ao + c, s_e + c, TWd);
}

template <int FMT>
__global__ void __launch_bounds__(kMvBX* kMvBY, 2)
    k_mv_shade(const ViewDev* __restrict__ views, const IblDev* __restrict__ ibls, const int4* __restrict__ tiles,
               BatchDev bp) {
  __shared__ float4 s_lights[2 * kLightChunk];
  __shared__ float4 s_dup[2 * kLightChunk];
  __shared__ ViewDev s_view;
  __shared__ IblDev s_ibl;
  constexpr int kThreads = kMvBX * kMvBY;
  int tid = threadIdx.y * kMvBX + threadIdx.x;
  int4 td = __ldg(tiles + blockIdx.x);
  mv_stage_view(views, ibls, td.x, s_view, &s_ibl, tid, kThreads);
  __syncthreads();
  const ViewDev& v = s_view;
  int x = td.y * kMvBX + threadIdx.x;
  int yy[2] = {td.z * kMvTileH + 2 * (int)threadIdx.y, td.z * kMvTileH + 2 * (int)threadIdx.y + 1};
  bool in[2] = {x < v.g.W && yy[0] < v.g.H, x < v.g.W && yy[1] < v.g.H};
  PxRaw raw[2];
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (in[h]) raw[h] = px_load<FMT>(v.g, x, yy[h]);
  int nl = v.NL;
  bool mono = false;
  if (nl <= kLightChunk) mono = __syncthreads_and(stage_lights(s_lights, v.lights, 0, nl, tid, kThreads, s_dup));
  Px s[2];
  bool act[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (in[h]) s[h] = px_decode<FMT>(raw[h], v.cam, x, yy[h]);
    act[h] = in[h] && s[h].surface;
  }
  shade_lights(s, act, nl, bp.flags, v.lights, s_lights, s_dup, kLightChunk, nl <= kLightChunk, mono, tid, kThreads);
  // after the blur by a programmatic edge: the blur may still be running up to here; the AO is read,
  // and the images written, after it has finished
  griddep_wait();
  float ao[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) ao[h] = act[h] ? __ldg(v.ao + (size_t)(yy[h] >> 1) * v.ao_w + (x >> 1)) : 1.0f;
  float3 c[2];
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (in[h]) c[h] = px_finish(s[h], s_ibl, bp.flags, ao[h]);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!in[h]) continue;
    if (v.hdr) {
      if (bp.hdr_format == EPBR_HDR_RGBA32F)
        store_hdr<EPBR_HDR_RGBA32F>(v.hdr, v.hdr_pitch, x, yy[h], c[h]);
      else
        store_hdr<EPBR_HDR_RGBA16F>(v.hdr, v.hdr_pitch, x, yy[h], c[h]);
    }
    ((unsigned*)(v.ldr + (size_t)yy[h] * v.ldr_pitch))[x] = pack_rgba8(c[h], bp.exposure, bp.op);
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
struct TileShape {
  int w, h;
};
static const TileShape kShapes[] = {{64, 32}, {128, 32}, {64, 64}};
static const int kChunks[] = {128, 256};
enum { kModeFused = 0, kModeStaged = 1, kModePerView = 2 };

typedef void (*BatchKernel)(const ViewDev*, const IblDev*, const int4*, int, int*, BatchDev);

template <int FMT>
static BatchKernel pick_kernel(int tw, int th) {
  if (tw == 64 && th == 32) return k_batch<FMT, 64, 32>;
  if (tw == 128 && th == 32) return k_batch<FMT, 128, 32>;
  if (tw == 64 && th == 64) return k_batch<FMT, 64, 64>;
  return nullptr;
}

}  // namespace epbr

using namespace epbr;

struct epbr_batch {
  int n_views = 0, n_ibls = 0, fmt = 0;
  std::vector<ViewDev> views;
  std::vector<long long> view_cost;
  BatchDev bp;
  ViewDev* d_views = nullptr;
  IblDev* d_ibls = nullptr;
  int4* d_tiles = nullptr;     // fused: TW x TH tiles; staged: 32x8 pixel tiles
  int4* d_ao_tiles = nullptr;  // staged: 32x8 AO-texel tiles
  int* d_counter = nullptr;
  float* d_ao = nullptr;       // staged: every view's unblurred + blurred AO
  size_t tiles_cap = 0, ao_tiles_cap = 0;
  int ntiles = 0, n_ao_tiles = 0;
  int mode = kModeFused, tile_w = 64, tile_h = 32, chunk = 256;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int grid = 0;
  void* args[3][6];
  // per-view plan: the views, lighting sets and parameters as passed to epbr_batch_create (the
  // per-view entry points are recorded into the graph by stream capture)
  std::vector<epbr_view> src_views;
  std::vector<epbr_ibl> src_ibls;
  epbr_batch_params params;
};

static void drop_graph(epbr_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Tiles of every view, views by descending work per tile, a view's tiles together.
static std::vector<int4> make_tiles(const epbr_batch* b, int tw, int th, bool ao_image) {
  std::vector<int> order(b->n_views);
  for (int i = 0; i < b->n_views; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->view_cost[a] > b->view_cost[c]; });
  std::vector<int4> tiles;
  for (int vi : order) {
    const ViewDev& v = b->views[vi];
    int W = ao_image ? (v.g.W + 1) / 2 : v.g.W, H = ao_image ? (v.g.H + 1) / 2 : v.g.H;
    int tx = (W + tw - 1) / tw, ty = (H + th - 1) / th;
    for (int y = 0; y < ty; ++y)
      for (int x = 0; x < tx; ++x) tiles.push_back(make_int4(vi, x, y, 0));
  }
  return tiles;
}

static epbr_status upload_tiles(const std::vector<int4>& t, int4** dst, size_t* cap) {
  if (t.size() > *cap) {
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    if (cudaMalloc(dst, t.size() * sizeof(int4)) != cudaSuccess)
      return fail(EPBR_ERR_NO_MEMORY, "batch: tile list allocation failed");
    *cap = t.size();
  }
  if (cudaMemcpy(*dst, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "batch: tile upload failed");
  return EPBR_OK;
}

static epbr_status build_tiles(epbr_batch* b) {
  epbr_status st;
  if (b->mode == kModeFused) {
    std::vector<int4> t = make_tiles(b, b->tile_w, b->tile_h, false);
    if ((st = upload_tiles(t, &b->d_tiles, &b->tiles_cap))) return st;
    b->ntiles = (int)t.size();
  } else {
    if (!b->d_ao) {  // every view's AO images, allocated once
      size_t total = 0;
      for (const ViewDev& v : b->views) total += (size_t)((v.g.W + 1) / 2) * ((v.g.H + 1) / 2);
      if (cudaMalloc(&b->d_ao, 2 * total * sizeof(float)) != cudaSuccess)
        return fail(EPBR_ERR_NO_MEMORY, "batch: AO images (%zu bytes) allocation failed", 2 * total * sizeof(float));
      size_t off = 0;
      for (ViewDev& v : b->views) {
        size_t n = (size_t)((v.g.W + 1) / 2) * ((v.g.H + 1) / 2);
        v.ao_w = (v.g.W + 1) / 2;
        v.ao_raw = b->d_ao + off;
        v.ao = b->d_ao + total + off;
        off += n;
      }
    }
    std::vector<int4> t = make_tiles(b, kMvBX, kMvTileH, false), ta = make_tiles(b, kMvBX, kMvBY, true);
    if ((st = upload_tiles(t, &b->d_tiles, &b->tiles_cap))) return st;
    if ((st = upload_tiles(ta, &b->d_ao_tiles, &b->ao_tiles_cap))) return st;
    b->ntiles = (int)t.size();
    b->n_ao_tiles = (int)ta.size();
  }
  if (cudaMemcpy(b->d_views, b->views.data(), b->views.size() * sizeof(ViewDev), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return fail(EPBR_ERR_CUDA, "batch: view upload failed");
  return EPBR_OK;
}

// Adds a kernel node after `dep` (if any).  With `early` the edge is programmatic: the node's blocks
// may start once every block of `dep` has started and called griddep_launch_dependents (or
// exited), and the kernel calls griddep_wait before it reads what `dep` writes.
static epbr_status add_kernel(epbr_batch* b, cudaGraphNode_t* node, const cudaGraphNode_t* dep, void* func,
                              dim3 grid, dim3 block, void** args, bool early = false) {
  cudaKernelNodeParams kp = {};
  kp.func = func;
  kp.gridDim = grid;
  kp.blockDim = block;
  kp.kernelParams = args;
  const bool prog = early && dep;
  if (cudaGraphAddKernelNode(node, b->graph, prog ? nullptr : dep, (dep && !prog) ? 1 : 0, &kp) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "batch: kernel node failed: %s", cudaGetErrorString(cudaGetLastError()));
  if (prog) {
    cudaGraphEdgeData ed = {};
    ed.from_port = cudaGraphKernelNodePortProgrammatic;
    ed.type = cudaGraphDependencyTypeProgrammatic;
    if (cudaGraphAddDependencies(b->graph, dep, node, &ed, 1) != cudaSuccess)
      return fail(EPBR_ERR_CUDA, "batch: programmatic edge failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  return EPBR_OK;
}

// Per-view plan: epbr_ssao_raw, epbr_ssao_blur and epbr_shade_tonemap (EPBR_SHADE_EARLY_START)
// of every view, recorded into the batch's graph by capturing a private stream, so the graph
// replays the per-view kernels (TMA-tiled SSAO, two-texel blur, two-pixel compose) with the
// programmatic edges of their early launches and without per-launch host work.  Replaces the
// graph created by build_graph.
static epbr_status capture_per_view(epbr_batch* b) {
  cudaGraphDestroy(b->graph);
  b->graph = nullptr;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "batch: capture stream: %s", cudaGetErrorString(cudaGetLastError()));
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return fail(EPBR_ERR_CUDA, "batch: begin capture: %s", cudaGetErrorString(cudaGetLastError()));
  }
  epbr_status st = EPBR_OK;
  const epbr_batch_params& p = b->params;
  for (int i = 0; i < b->n_views && !st; ++i) {
    const epbr_view& v = b->src_views[i];
    const ViewDev& d = b->views[i];
    const int64_t ap = (int64_t)d.ao_w * 4;
    st = epbr_ssao_raw(&v.gbuffer, &v.camera, &p.ssao, d.ao_raw, ap, cs);
    if (!st) st = epbr_ssao_blur(&v.gbuffer, &p.ssao, d.ao_raw, ap, d.ao, ap, cs);
    if (!st) {
      epbr_shade_params sp;
      sp.flags = p.flags | EPBR_SHADE_EARLY_START;
      sp.ao_scale = 2;
      sp.ao = d.ao;
      sp.ao_pitch = ap;
      st = epbr_shade_tonemap(&v.gbuffer, &v.camera, v.lights, v.num_lights, &b->src_ibls[v.ibl_index], &sp, v.hdr,
                              p.hdr_format, v.hdr_pitch, &p.tonemap, v.ldr, v.ldr_pitch, cs);
    }
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (st) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess || !g) return fail(EPBR_ERR_CUDA, "batch: end capture: %s", cudaGetErrorString(e));
  b->graph = g;
  return EPBR_OK;
}

// Fused: memset(counter) -> k_batch.  Staged: k_mv_ssao_raw -> k_mv_ssao_blur -> k_mv_shade.
// Per view: the per-view entry points of every view, captured.
static epbr_status build_graph(epbr_batch* b) {
  drop_graph(b);
  b->bp.light_chunk = b->chunk;
  if (cudaGraphCreate(&b->graph, 0) != cudaSuccess) return fail(EPBR_ERR_CUDA, "batch: cudaGraphCreate failed");
  epbr_status st;
  bool fp32 = b->fmt == EPBR_GBUFFER_FP32;
  if (b->mode == kModeFused) {
    BatchKernel k = fp32 ? pick_kernel<EPBR_GBUFFER_FP32>(b->tile_w, b->tile_h)
                         : pick_kernel<EPBR_GBUFFER_COMPACT>(b->tile_w, b->tile_h);
    if (!k) return fail(EPBR_ERR_UNSUPPORTED, "batch: tile %dx%d not compiled", b->tile_w, b->tile_h);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k, kBatchThreads, 0) != cudaSuccess ||
        per_sm < 1)
      return fail(EPBR_ERR_CUDA, "batch: occupancy query failed");
    b->grid = std::max(1, std::min(b->ntiles, per_sm * num_sms()));
    void** a = b->args[0];
    a[0] = &b->d_views;
    a[1] = &b->d_ibls;
    a[2] = &b->d_tiles;
    a[3] = &b->ntiles;
    a[4] = &b->d_counter;
    a[5] = &b->bp;
    cudaMemsetParams mp = {};
    mp.dst = b->d_counter;
    mp.elementSize = 4;
    mp.width = 1;
    mp.height = 1;
    cudaGraphNode_t n_memset, n_kernel;
    if (cudaGraphAddMemsetNode(&n_memset, b->graph, nullptr, 0, &mp) != cudaSuccess)
      return fail(EPBR_ERR_CUDA, "batch: memset node failed");
    if ((st = add_kernel(b, &n_kernel, &n_memset, (void*)k, dim3(b->grid), dim3(kBatchThreads), a))) return st;
  } else if (b->mode == kModeStaged) {
    void* raw = fp32 ? (void*)k_mv_ssao_raw<EPBR_GBUFFER_FP32> : (void*)k_mv_ssao_raw<EPBR_GBUFFER_COMPACT>;
    void* blur = fp32 ? (void*)k_mv_ssao_blur<EPBR_GBUFFER_FP32> : (void*)k_mv_ssao_blur<EPBR_GBUFFER_COMPACT>;
    void* shade = fp32 ? (void*)k_mv_shade<EPBR_GBUFFER_FP32> : (void*)k_mv_shade<EPBR_GBUFFER_COMPACT>;
    b->args[0][0] = &b->d_views;
    b->args[0][1] = &b->d_ao_tiles;
    b->args[0][2] = &b->bp;
    b->args[1][0] = &b->d_views;
    b->args[1][1] = &b->d_ao_tiles;
    b->args[1][2] = &b->bp;
    b->args[2][0] = &b->d_views;
    b->args[2][1] = &b->d_ibls;
    b->args[2][2] = &b->d_tiles;
    b->args[2][3] = &b->bp;
    cudaGraphNode_t n0, n1, n2;
    dim3 blk(kMvBX, kMvBY);
    if ((st = add_kernel(b, &n0, nullptr, raw, dim3(b->n_ao_tiles), blk, b->args[0]))) return st;
    // programmatic edges: the blur's blocks wait on the SMs the raw pass's last wave leaves free, and
    // the compose's light loops run while the blur does (each waits before it reads the AO)
    if ((st = add_kernel(b, &n1, &n0, blur, dim3(b->n_ao_tiles), blk, b->args[1], true))) return st;
    if ((st = add_kernel(b, &n2, &n1, shade, dim3(b->ntiles), blk, b->args[2], true))) return st;
    b->grid = b->ntiles;
  } else {
    if ((st = capture_per_view(b))) return st;
    b->grid = b->ntiles;
  }
  if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "batch: graph instantiation failed: %s", cudaGetErrorString(cudaGetLastError()));
  return EPBR_OK;
}

static bool plan_valid(int mode, int tw, int th, int chunk) {
  if (chunk < 1 || chunk > kLightChunk) return false;
  if (mode == kModeStaged || mode == kModePerView) return true;
  return mode == kModeFused && pick_kernel<EPBR_GBUFFER_FP32>(tw, th) != nullptr;
}

static epbr_status set_plan(epbr_batch* b, int mode, int tw, int th, int chunk) {
  if (!plan_valid(mode, tw, th, chunk))
    return fail(EPBR_ERR_INVALID_ARG, "batch: plan mode %d tile %dx%d chunk %d not available", mode, tw, th, chunk);
  b->mode = mode;
  b->tile_w = mode == kModeFused ? tw : kMvBX;
  b->tile_h = mode == kModeFused ? th : kMvTileH;
  b->chunk = mode == kModeFused ? chunk : kLightChunk;
  epbr_status st = build_tiles(b);
  if (st) return st;
  return build_graph(b);
}

static std::string batch_key(const epbr_batch* b) {
  long long px = 0;
  int max_nl = 0;
  for (const ViewDev& v : b->views) {
    px += (long long)v.g.W * v.g.H;
    max_nl = std::max(max_nl, v.NL);
  }
  char buf[128];
  snprintf(buf, sizeof(buf), "fmt%d_views%d_mpx%lld_maxnl%d_k%d", b->fmt, b->n_views, px >> 20, max_nl, b->bp.ssao.K);
  return buf;
}

extern "C" epbr_status epbr_batch_create(const epbr_view* views, int32_t n_views, const epbr_ibl* ibls,
                                         int32_t n_ibls, const epbr_batch_params* p, epbr_batch** out) {
  if (!views || n_views < 1 || !ibls || n_ibls < 1 || !p || !out)
    return fail(EPBR_ERR_INVALID_ARG, "batch: NULL argument or empty batch");
  if (p->ssao.scale != 2 || p->ssao.blur_radius < 0 || p->ssao.blur_radius > kBatchMaxR ||
      p->ssao.num_samples < 1 || p->ssao.num_samples > kBatchMaxK || !p->ssao.kernel || !p->ssao.noise ||
      !(p->ssao.radius > 0.0f) || !(p->ssao.sigma_s > 0.0f) || !(p->ssao.sigma_z > 0.0f) ||
      (uintptr_t)p->ssao.kernel % 16 || (uintptr_t)p->ssao.noise % 8)
    return fail(EPBR_ERR_INVALID_ARG, "batch: ssao needs scale 2, blur_radius <= %d, 1..%d samples", kBatchMaxR,
                kBatchMaxK);
  if (p->hdr_format != EPBR_HDR_RGBA32F && p->hdr_format != EPBR_HDR_RGBA16F)
    return fail(EPBR_ERR_INVALID_ARG, "batch: hdr_format invalid");
  if (p->flags & ~(unsigned)(EPBR_SHADE_DIRECT | EPBR_SHADE_IBL | EPBR_SHADE_MULTISCATTER | EPBR_SHADE_DIFFUSE_ONLY))
    return fail(EPBR_ERR_INVALID_ARG, "batch: unknown flags");
  if (!(p->tonemap.exposure >= 0.0f) || (p->tonemap.op != EPBR_TONEMAP_ACES && p->tonemap.op != EPBR_TONEMAP_REINHARD))
    return fail(EPBR_ERR_INVALID_ARG, "batch: tonemap params invalid");
  int fmt = views[0].gbuffer.format;
  epbr_batch* b = new epbr_batch();
  b->n_views = n_views;
  b->n_ibls = n_ibls;
  b->fmt = fmt;
  b->views.resize(n_views);
  b->view_cost.resize(n_views);
  for (int i = 0; i < n_views; ++i) {
    const epbr_view& v = views[i];
    epbr_status st = validate_gbuffer(&v.gbuffer, true);
    if (!st) st = validate_camera(&v.camera, &v.gbuffer);
    if (!st && v.gbuffer.format != fmt) st = fail(EPBR_ERR_INVALID_ARG, "batch: views mix G-buffer formats");
    if (!st && (v.ibl_index < 0 || v.ibl_index >= n_ibls)) st = fail(EPBR_ERR_INVALID_ARG, "batch: view %d ibl_index", i);
    if (!st && (v.num_lights < 0 || v.num_lights > 65536 || (v.num_lights > 0 && (!v.lights || (uintptr_t)v.lights % 16))))
      st = fail(EPBR_ERR_INVALID_ARG, "batch: view %d lights", i);
    if (!st && (!v.ldr || (uintptr_t)v.ldr % 4 || v.ldr_pitch < 4LL * v.gbuffer.width || v.ldr_pitch % 4))
      st = fail(EPBR_ERR_INVALID_ARG, "batch: view %d ldr buffer", i);
    int bpp = p->hdr_format == EPBR_HDR_RGBA32F ? 16 : 8;
    if (!st && v.hdr && ((uintptr_t)v.hdr % bpp || v.hdr_pitch < (int64_t)bpp * v.gbuffer.width || v.hdr_pitch % bpp))
      st = fail(EPBR_ERR_INVALID_ARG, "batch: view %d hdr buffer", i);
    if (st) {
      delete b;
      return st;
    }
    ViewDev& d = b->views[i];
    memset(&d, 0, sizeof(d));
    d.g = make_gbuf(v.gbuffer);
    d.cam = make_cam(v.camera);
    d.lights = (const float4*)v.lights;
    d.NL = (p->flags & EPBR_SHADE_DIRECT) ? v.num_lights : 0;
    d.ibl = v.ibl_index;
    d.hdr = v.hdr;
    d.hdr_pitch = v.hdr_pitch;
    d.ldr = v.ldr;
    d.ldr_pitch = v.ldr_pitch;
    b->view_cost[i] = d.NL + 12;  // work per tile ~ lights + the fixed per-pixel part
  }
  std::vector<IblDev> hib(n_ibls);
  for (int i = 0; i < n_ibls; ++i) {
    const epbr_ibl& s = ibls[i];
    IblDev& d = hib[i];
    memset(&d, 0, sizeof(d));
    if ((p->flags & EPBR_SHADE_IBL) &&
        (!s.irradiance || !s.lut || s.num_levels < 1 || s.num_levels > EPBR_MAX_LEVELS || s.lut_size < 1)) {
      delete b;
      return fail(EPBR_ERR_INVALID_ARG, "batch: ibl %d incomplete", i);
    }
    d.irr = MapDev{(const float4*)s.irradiance, std::max(1, s.irr_width), std::max(1, s.irr_height)};
    for (int m = 0; m < EPBR_MAX_LEVELS; ++m)
      d.lev[m] = m < s.num_levels ? MapDev{(const float4*)s.level[m], s.level_width[m], s.level_height[m]}
                                  : MapDev{nullptr, 1, 1};
    d.lut = (const float2*)s.lut;
    d.S = std::max(1, s.lut_size);
    d.M = std::max(1, s.num_levels);
  }
  b->src_views.assign(views, views + n_views);
  b->src_ibls.assign(ibls, ibls + n_ibls);
  b->params = *p;
  memset(&b->bp, 0, sizeof(b->bp));
  b->bp.flags = p->flags;
  b->bp.hdr_format = p->hdr_format;
  b->bp.exposure = p->tonemap.exposure;
  b->bp.op = p->tonemap.op;
  b->bp.ssao = make_ssao(p->ssao);  // scale 2, checked above
  bool ok_alloc = cudaMalloc(&b->d_views, sizeof(ViewDev) * n_views) == cudaSuccess &&
                  cudaMalloc(&b->d_ibls, sizeof(IblDev) * n_ibls) == cudaSuccess &&
                  cudaMalloc(&b->d_counter, sizeof(int)) == cudaSuccess;
  if (!ok_alloc || cudaMemcpy(b->d_ibls, hib.data(), sizeof(IblDev) * n_ibls, cudaMemcpyHostToDevice) != cudaSuccess) {
    epbr_batch_destroy(b);
    return fail(EPBR_ERR_NO_MEMORY, "batch: descriptor allocation failed");
  }
  int tw = p->tile_w ? p->tile_w : 64, th = p->tile_h ? p->tile_h : 32, ch = p->light_chunk ? p->light_chunk : 256;
  epbr_status st = set_plan(b, kModeFused, tw, th, ch);
  if (st) {
    epbr_batch_destroy(b);
    return st;
  }
  *out = b;
  return ok();
}

extern "C" epbr_status epbr_batch_launch(epbr_batch* b, void* stream) {
  if (!b || !b->exec) return fail(EPBR_ERR_INVALID_ARG, "batch: not created");
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(EPBR_ERR_CUDA, "batch: cudaGraphLaunch: %s", cudaGetErrorString(e));
  return ok();
}

extern "C" epbr_status epbr_batch_get_plan(const epbr_batch* b, int32_t* mode, int32_t* tw, int32_t* th,
                                           int32_t* chunk) {
  if (!b || !mode || !tw || !th || !chunk) return fail(EPBR_ERR_INVALID_ARG, "batch: NULL argument");
  *mode = b->mode;
  *tw = b->tile_w;
  *th = b->tile_h;
  *chunk = b->chunk;
  return ok();
}

extern "C" epbr_status epbr_batch_set_plan(epbr_batch* b, int32_t mode, int32_t tw, int32_t th, int32_t chunk) {
  if (!b) return fail(EPBR_ERR_INVALID_ARG, "batch: NULL");
  epbr_status st = set_plan(b, mode, tw, th, chunk);
  return st ? st : ok();
}

// Times every candidate plan on the batch (2 warm-up + 3 timed graph launches each, CUDA events
// on `stream`) and keeps the fastest.  With `cache_path`, a plan stored there for the same batch
// key is used without timing, and a new result is appended.
extern "C" epbr_status epbr_batch_autotune(epbr_batch* b, const char* cache_path, void* stream) {
  if (!b) return fail(EPBR_ERR_INVALID_ARG, "batch: NULL");
  std::string key = batch_key(b);
  if (cache_path) {
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char k[160];
      int md, tw, th, ch;
      float ms;
      while (fscanf(f, "%159s %d %d %d %d %f", k, &md, &tw, &th, &ch, &ms) == 6) {
        if (key == k && plan_valid(md, tw, th, ch)) {
          fclose(f);
          epbr_status st = set_plan(b, md, tw, th, ch);
          return st ? st : ok();
        }
      }
      fclose(f);
    }
  }
  struct Cand {
    int mode, tw, th, ch;
  };
  std::vector<Cand> cands;
  for (const TileShape& sh : kShapes)
    for (int ch : kChunks) cands.push_back({kModeFused, sh.w, sh.h, ch});
  cands.push_back({kModeStaged, kMvBX, kMvBY, kLightChunk});
  cands.push_back({kModePerView, kMvBX, kMvBY, kLightChunk});
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(EPBR_ERR_CUDA, "autotune: event creation failed");
  float best = 1e30f;
  Cand bc = cands[0];
  epbr_status st = EPBR_OK;
  for (const Cand& c : cands) {
    if ((st = set_plan(b, c.mode, c.tw, c.th, c.ch))) break;
    for (int r = 0; r < 2; ++r) cudaGraphLaunch(b->exec, s);
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) cudaGraphLaunch(b->exec, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = fail(EPBR_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bc = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  if ((st = set_plan(b, bc.mode, bc.tw, bc.th, bc.ch))) return st;
  if (cache_path) {
    FILE* f = fopen(cache_path, "a");
    if (f) {
      fprintf(f, "%s %d %d %d %d %.4f\n", key.c_str(), bc.mode, bc.tw, bc.th, bc.ch, best / 3.0f);
      fclose(f);
    }
  }
  return ok();
}

extern "C" epbr_status epbr_batch_destroy(epbr_batch* b) {
  if (!b) return ok();
  drop_graph(b);
  if (b->d_views) cudaFree(b->d_views);
  if (b->d_ibls) cudaFree(b->d_ibls);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_ao_tiles) cudaFree(b->d_ao_tiles);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->d_ao) cudaFree(b->d_ao);
  delete b;
  return ok();
}

extern "C" epbr_status epbr_render_batch(const epbr_view* views, int32_t n_views, const epbr_ibl* ibls,
                                         int32_t n_ibls, const epbr_batch_params* p, void* stream) {
  epbr_batch* b = nullptr;
  epbr_status st = epbr_batch_create(views, n_views, ibls, n_ibls, p, &b);
  if (st) return st;
  st = epbr_batch_launch(b, stream);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  epbr_batch_destroy(b);
  if (st) return st;
  if (e != cudaSuccess) return fail(EPBR_ERR_CUDA, "render_batch: %s", cudaGetErrorString(e));
  return ok();
}
