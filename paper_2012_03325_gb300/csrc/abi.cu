// Error plumbing, argument validation and the host-only layout queries of the C ABI.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <string>

#include "tma.cuh"

namespace epbr {

static thread_local std::string t_last_error;

epbr_status fail(epbr_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return code;
}

epbr_status ok() {
  t_last_error.clear();
  return EPBR_OK;
}

epbr_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(EPBR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return EPBR_OK;
}

static std::atomic<unsigned long long> g_tma_first_wait_ns{kTmaWaitNs};

unsigned long long tma_first_wait_ns() { return g_tma_first_wait_ns.load(); }

unsigned long long set_tma_first_wait_ns(unsigned long long ns) { return g_tma_first_wait_ns.exchange(ns); }

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

epbr_status validate_gbuffer(const epbr_gbuffer* g, bool need_material) {
  if (!g) return fail(EPBR_ERR_INVALID_ARG, "gbuffer is NULL");
  if (g->width < 1 || g->height < 1 || g->width > (1 << 15) || g->height > (1 << 15))
    return fail(EPBR_ERR_INVALID_ARG, "gbuffer size %dx%d outside [1, 32768]", g->width, g->height);
  if (g->format != EPBR_GBUFFER_FP32 && g->format != EPBR_GBUFFER_COMPACT)
    return fail(EPBR_ERR_INVALID_ARG, "gbuffer format %d unknown", g->format);
  // bytes per texel of rt[0], rt[1], rt[2], rt[3]
  const int fp32[4] = {16, 16, 0, 4}, compact[4] = {4, 4, 2, 4};
  const int* bpp = g->format == EPBR_GBUFFER_FP32 ? fp32 : compact;
  for (int i = 0; i < 4; ++i) {
    if (bpp[i] == 0) continue;
    bool needed = (i == 3) || (i == 1) || need_material;
    if (!needed) continue;
    if (!g->rt[i]) return fail(EPBR_ERR_INVALID_ARG, "gbuffer rt[%d] is NULL", i);
    if (!aligned(g->rt[i], (size_t)bpp[i]))
      return fail(EPBR_ERR_INVALID_ARG, "gbuffer rt[%d] not aligned to %d bytes", i, bpp[i]);
    if (g->pitch[i] < (int64_t)bpp[i] * g->width || g->pitch[i] % bpp[i] != 0)
      return fail(EPBR_ERR_INVALID_ARG, "gbuffer pitch[%d] = %lld invalid for width %d", i,
                  (long long)g->pitch[i], g->width);
  }
  return EPBR_OK;
}

epbr_status validate_camera(const epbr_camera* c, const epbr_gbuffer* g) {
  if (!c) return fail(EPBR_ERR_INVALID_ARG, "camera is NULL");
  if (!(c->fov_y > 0.0f && c->fov_y < 3.14159f)) return fail(EPBR_ERR_INVALID_ARG, "fov_y out of (0, pi)");
  if (g && (c->width != g->width || c->height != g->height))
    return fail(EPBR_ERR_INVALID_ARG, "camera size %dx%d differs from gbuffer %dx%d", c->width,
                c->height, g->width, g->height);
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(c->view_to_world[i])) return fail(EPBR_ERR_INVALID_ARG, "camera matrix not finite");
  return EPBR_OK;
}

epbr_status validate_env(const epbr_env* e) {
  if (!e || !e->texels) return fail(EPBR_ERR_INVALID_ARG, "env or env->texels is NULL");
  if (e->width < 1 || e->height < 1 || e->width > (1 << 16) || e->height > (1 << 16))
    return fail(EPBR_ERR_INVALID_ARG, "env size %dx%d outside [1, 65536]", e->width, e->height);
  if ((long long)e->width * e->height > (1LL << 28))
    return fail(EPBR_ERR_INVALID_ARG, "env has %lld texels, more than 2^28", (long long)e->width * e->height);
  if (!aligned(e->texels, 16)) return fail(EPBR_ERR_INVALID_ARG, "env texels not 16-byte aligned");
  return EPBR_OK;
}

}  // namespace epbr

using namespace epbr;

extern "C" const char* epbr_last_error(void) { return t_last_error.c_str(); }
extern "C" const char* epbr_version(void) { return "epbr 0.1 (sm_103a)"; }

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" epbr_status epbr_ibl_layout(const epbr_ibl_params* p, int32_t W, int32_t H, void* buffer,
                                       size_t* bytes, epbr_ibl* out) {
  if (!p || !bytes) return fail(EPBR_ERR_INVALID_ARG, "params or bytes is NULL");
  if (p->num_levels < 1 || p->num_levels > EPBR_MAX_LEVELS)
    return fail(EPBR_ERR_INVALID_ARG, "num_levels %d outside [1, %d]", p->num_levels, EPBR_MAX_LEVELS);
  if (p->lut_size < 1 || p->lut_size > 4096 || p->irr_width < 1 || p->irr_height < 1 ||
      p->irr_width > 4096 || p->irr_height > 4096 || p->prefilter_samples < 1 || p->lut_samples < 1)
    return fail(EPBR_ERR_INVALID_ARG, "ibl params out of range");
  if (W < 1 || H < 1 || W > (1 << 16) || H > (1 << 16) || (long long)W * H > (1LL << 28))
    return fail(EPBR_ERR_INVALID_ARG, "env size %dx%d outside [1, 65536]^2 or above 2^28 texels", W, H);
  size_t off = 0;
  size_t irr_off = off;
  off = align256(off + (size_t)p->irr_width * p->irr_height * 16);
  size_t lut_off = off;
  off = align256(off + (size_t)p->lut_size * p->lut_size * 8);
  size_t lvl_off[EPBR_MAX_LEVELS];
  for (int m = 0; m < p->num_levels; ++m) {
    int w = W >> m, h = H >> m;
    w = w < 1 ? 1 : w;
    h = h < 1 ? 1 : h;
    lvl_off[m] = off;
    off = align256(off + (size_t)w * h * 16);
  }
  *bytes = off;
  if (!buffer) return ok();
  if (!out) return fail(EPBR_ERR_INVALID_ARG, "out is NULL");
  if ((uintptr_t)buffer % 256) return fail(EPBR_ERR_INVALID_ARG, "buffer not 256-byte aligned");
  memset(out, 0, sizeof(*out));
  char* b = (char*)buffer;
  out->irradiance = (float*)(b + irr_off);
  out->irr_width = p->irr_width;
  out->irr_height = p->irr_height;
  out->lut = (float*)(b + lut_off);
  out->lut_size = p->lut_size;
  out->num_levels = p->num_levels;
  for (int m = 0; m < p->num_levels; ++m) {
    int w = W >> m, h = H >> m;
    out->level[m] = (float*)(b + lvl_off[m]);
    out->level_width[m] = w < 1 ? 1 : w;
    out->level_height[m] = h < 1 ? 1 : h;
  }
  return ok();
}
