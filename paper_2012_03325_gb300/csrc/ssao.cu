// Screen-space ambient occlusion (paper Sec. 5.2: normal-oriented hemisphere of Bavoil &
// Sainz 2008, at half resolution, then a bilateral blur).
//   k_ssao_raw   one thread per AO texel; the K kernel offsets sit in shared memory and the
//                depth taps go through the read-only cache (per-texel math in ssao_core.cuh)
//   k_ssao_blur  one thread per AO texel; (2R+1)^2 depth-aware taps read from a shared-memory
//                tile of AO values and depths with an R-texel halo
#include "ssao_core.cuh"

namespace epbr {

#ifndef EPBR_SSAO_MIN_BLOCKS
#define EPBR_SSAO_MIN_BLOCKS 4  // resident 256-thread blocks per SM the register budget targets
#endif

template <int FMT>
__global__ void __launch_bounds__(256, EPBR_SSAO_MIN_BLOCKS) k_ssao_raw(GbufDev g, CamDev cam, SsaoDev p, float* __restrict__ ao,
                                                  long long ao_pitch, int Wa, int Ha) {
  __shared__ float4 s_kernel[kMaxSsaoSamples];
  int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int k = tid; k < p.K; k += blockDim.x * blockDim.y) s_kernel[k] = __ldg(p.kernel + k);
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= Wa || j >= Ha) return;
  ((float*)((char*)ao + (size_t)j * ao_pitch))[i] = ssao_texel<FMT>(g, cam, p, s_kernel, i, j).x;
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
  dim3 blk(32, 8), grd((Wa + 31) / 32, (Ha + 7) / 8);
  GbufDev gd = make_gbuf(*g);
  CamDev cd = make_cam(*cam);
  SsaoDev sd = make_ssao(*p);
  cudaStream_t s = (cudaStream_t)stream;
  if (g->format == EPBR_GBUFFER_FP32)
    k_ssao_raw<EPBR_GBUFFER_FP32><<<grd, blk, 0, s>>>(gd, cd, sd, ao, ao_pitch, Wa, Ha);
  else
    k_ssao_raw<EPBR_GBUFFER_COMPACT><<<grd, blk, 0, s>>>(gd, cd, sd, ao, ao_pitch, Wa, Ha);
  if ((st = check_launch("k_ssao_raw"))) return st;
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
  if (g->format == EPBR_GBUFFER_FP32)
    k_ssao_blur<EPBR_GBUFFER_FP32><<<grd, blk, 0, s>>>(gd, sd, in, in_pitch, out, out_pitch, Wa, Ha);
  else
    k_ssao_blur<EPBR_GBUFFER_COMPACT><<<grd, blk, 0, s>>>(gd, sd, in, in_pitch, out, out_pitch, Wa, Ha);
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
