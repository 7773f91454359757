// Internal device and host helpers shared by the libepbr translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/epbr.h"

namespace epbr {

// ------------------------------------------------------------------------------------------
// host: error reporting (thread-local message, see abi.cu)
// ------------------------------------------------------------------------------------------
epbr_status fail(epbr_status code, const char* fmt, ...);
epbr_status ok();
// Checks cudaGetLastError after launches; returns EPBR_ERR_CUDA with `what` on failure.
epbr_status check_launch(const char* what);
int num_sms();

// Exclusive int64 prefix sum of data[0 .. n) in place (raster.cu); sums needs
// scan_num_blocks(n) + 1 entries and receives the total at sums[scan_num_blocks(n)].
long long scan_num_blocks(long long n);
void launch_exclusive_scan(long long* data, long long n, long long* sums, cudaStream_t s);

// Launches kernel k; with `early` under programmatic stream serialisation, so that its blocks may
// start once every block of the previous kernel on the stream has started and called
// griddep_launch_dependents (or exited), instead of after that kernel has finished.  A kernel
// launched this way must call griddep_wait before it reads anything the previous kernel writes and
// before it writes anything the previous kernel reads.  Returns the launch's CUDA error.
template <typename... Params, typename... Args>
cudaError_t launch_kernel(void (*k)(Params...), dim3 grd, dim3 blk, size_t smem, cudaStream_t s, bool early,
                          Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grd;
  cfg.blockDim = blk;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = early ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, static_cast<Args&&>(args)...);
}

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInvPi = 0.318309886183790671538f;
constexpr float kInv2Pi = 0.159154943091895335769f;
constexpr float kRoughMin = 0.045f;
constexpr float kNvMin = 1e-4f;

// ------------------------------------------------------------------------------------------
// device: programmatic dependent launch (PTX griddepcontrol, sm_90 and later)
// ------------------------------------------------------------------------------------------
// Waits until the grid this one depends on (the previous kernel on the stream, for a launch with
// `early` set) has completed and its memory operations are visible; returns at once for a grid
// launched without it.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Allows a dependent grid launched with `early` to start its blocks before this grid completes.
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------------------------------------
// device: small vector algebra on float3
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 mul3(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
}
// Hardware approximations with denormal flushing (one MUFU instruction each, no fix-up code):
// relative error ~2^-22, far inside the 1e-4 tolerance of the method.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_ftz(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_ftz(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_ftz(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float sqrt_ftz(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float3 normalize3(float3 a) { return a * rsqrt_ftz(dot3(a, a)); }
__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }

// Camera in device-friendly form: rotation rows/columns, eye, per-pixel ray scale.
struct CamDev {
  float r[9];   // view_to_world rotation, r[3*i + j] = row i, column j
  float eye[3];
  float sx, sy;  // px = (2 (x + 0.5) / W - 1) * sx, py = (1 - 2 (y + 0.5) / H) * sy
  // the same as px = (x + cx) ax, py = (y + cy) ay with cx = 1/2 - W/2, cy = 1/2 - H/2: x + cx is
  // exact in FP32 (a multiple of 1/2 below 2^15), so px has one rounding of the product however
  // far from the centre the image reaches (ax, ay rounded from FP64)
  float ax, cx, ay, cy;
  float ix_scale, iy_scale;  // view -> pixel: x = 0.5 W (1 + px / sx), y = 0.5 H (1 - py / sy)
  int W, H;
};

__host__ inline CamDev make_cam(const epbr_camera& c) {
  CamDev d;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) d.r[3 * i + j] = c.view_to_world[4 * j + i];
  d.eye[0] = c.view_to_world[12];
  d.eye[1] = c.view_to_world[13];
  d.eye[2] = c.view_to_world[14];
  double t = tan(0.5 * (double)c.fov_y);
  double sx = t * (double)c.width / (double)c.height;
  d.sy = (float)t;
  d.sx = (float)sx;
  d.ax = (float)(2.0 * sx / c.width);
  d.cx = (float)(0.5 - 0.5 * c.width);
  d.ay = (float)(-2.0 * t / c.height);
  d.cy = (float)(0.5 - 0.5 * c.height);
  d.ix_scale = (float)(0.5 * c.width / sx);
  d.iy_scale = (float)(0.5 * c.height / t);
  d.W = c.width;
  d.H = c.height;
  return d;
}

// View-space ray (px, py, -1) of the centre of pixel (x, y).
__device__ __forceinline__ float3 view_ray(const CamDev& c, int x, int y) {
  return f3(((float)x + c.cx) * c.ax, ((float)y + c.cy) * c.ay, -1.0f);
}
__device__ __forceinline__ float3 rot(const CamDev& c, float3 a) {
  return f3(fmaf(c.r[0], a.x, fmaf(c.r[1], a.y, c.r[2] * a.z)),
            fmaf(c.r[3], a.x, fmaf(c.r[4], a.y, c.r[5] * a.z)),
            fmaf(c.r[6], a.x, fmaf(c.r[7], a.y, c.r[8] * a.z)));
}
__device__ __forceinline__ float3 rot_t(const CamDev& c, float3 a) {
  return f3(fmaf(c.r[0], a.x, fmaf(c.r[3], a.y, c.r[6] * a.z)),
            fmaf(c.r[1], a.x, fmaf(c.r[4], a.y, c.r[7] * a.z)),
            fmaf(c.r[2], a.x, fmaf(c.r[5], a.y, c.r[8] * a.z)));
}
__device__ __forceinline__ bool is_surface(float e) { return e > 0.0f && e < __int_as_float(0x7f800000); }

// ------------------------------------------------------------------------------------------
// device: equirect environment maps
// ------------------------------------------------------------------------------------------
struct MapDev {
  const float4* texels;
  int W, H;
};

// atan2 by octant reduction and an odd polynomial fitted to atan on [0, 1] (coefficients from
// gen_atan_poly.py, |error| ~1e-7 rad in FP32).  Signed zeros follow IEEE 754: the sign bit of
// x picks the half plane, so atan2(+-0, -0) = +-pi and atan2(+-0, +0) = +-0.
__device__ __forceinline__ float atan2_poly(float y, float x) {
  constexpr float c[8] = {
#include "atan_poly.inc"
  };
  float ax = fabsf(x), ay = fabsf(y);
  float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  float t = mn * rcp_ftz(fmaxf(mx, 1e-30f));
  float s = t * t;
  float p = c[7];
#pragma unroll
  for (int k = 6; k >= 0; --k) p = fmaf(p, s, c[k]);
  float r = t * p;
  r = ay > ax ? 1.57079632679489662f - r : r;
  r = signbit(x) ? 3.14159265358979324f - r : r;
  return copysignf(r, y);
}

__device__ __forceinline__ void dir_to_uv(float3 d, float& u, float& v) {
  u = fmaf(atan2_poly(d.x, -d.z), kInv2Pi, 0.5f);
  v = atan2_poly(sqrt_ftz(fmaf(d.x, d.x, d.z * d.z)), d.y) * kInvPi;
}

// Bilinear read at (u, v): wrap in u, clamp in v.
__device__ __forceinline__ float3 equirect_bilinear(const MapDev m, float u, float v) {
  float x = fmaf(u, (float)m.W, -0.5f), y = fmaf(v, (float)m.H, -0.5f);
  float x0 = floorf(x), y0 = floorf(y);
  float fx = x - x0, fy = y - y0;
  int ix = (int)x0, iy = (int)y0;
  int i0 = ix < 0 ? ix + m.W : (ix >= m.W ? ix - m.W : ix);
  int i1 = i0 + 1 == m.W ? 0 : i0 + 1;
  int j0 = min(max(iy, 0), m.H - 1), j1 = min(max(iy + 1, 0), m.H - 1);
  int r0 = j0 * m.W, r1 = j1 * m.W;  // 32-bit: maps hold at most 2^28 texels
  float4 a = __ldg(m.texels + (r0 + i0)), b = __ldg(m.texels + (r0 + i1));
  float4 p = __ldg(m.texels + (r1 + i0)), q = __ldg(m.texels + (r1 + i1));
  float3 top = xyz(a) + fx * (xyz(b) - xyz(a));
  float3 bot = xyz(p) + fx * (xyz(q) - xyz(p));
  return top + fy * (bot - top);
}

__device__ __forceinline__ float3 equirect_lookup(const MapDev m, float3 d) {
  float u, v;
  dir_to_uv(d, u, v);
  return equirect_bilinear(m, u, v);
}

// Branchless orthonormal basis (Duff et al., JCGT 2017) around unit n.
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b) {
  float s = copysignf(1.0f, n.z);
  float a = -rcp_ftz(s + n.z);  // |s + n.z| in [1, 2]
  float c = n.x * n.y * a;
  t = f3(fmaf(s * n.x * n.x, a, 1.0f), s * c, -s * n.x);
  b = f3(c, fmaf(n.y * n.y, a, s), -n.y);
}

// Kahan-compensated accumulator.
struct Kahan {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// G-buffer in kernel-argument form.
struct GbufDev {
  const char* rt[4];
  long long pitch[4];
  int W, H;
};

__host__ inline GbufDev make_gbuf(const epbr_gbuffer& g) {
  GbufDev d;
  for (int i = 0; i < 4; ++i) {
    d.rt[i] = (const char*)g.rt[i];
    d.pitch[i] = g.pitch[i];
  }
  d.W = g.width;
  d.H = g.height;
  return d;
}

__device__ __forceinline__ float gb_depth(const GbufDev& g, int x, int y) {
  return __ldg((const float*)(g.rt[3] + (size_t)y * g.pitch[3]) + x);
}

// Octahedral unit-vector decode (Cigolle et al. 2014).
__device__ __forceinline__ float3 oct_decode(__half2 h) {
  float2 p = __half22float2(h);
  float x = p.x, y = p.y;
  float z = 1.0f - fabsf(x) - fabsf(y);
  if (z < 0.0f) {
    float nx = (1.0f - fabsf(y)) * (x >= 0.0f ? 1.0f : -1.0f);
    float ny = (1.0f - fabsf(x)) * (y >= 0.0f ? 1.0f : -1.0f);
    x = nx;
    y = ny;
  }
  return normalize3(f3(x, y, z));
}

template <int FMT>
__device__ __forceinline__ float3 gb_normal(const GbufDev& g, int x, int y) {
  if (FMT == EPBR_GBUFFER_FP32) {
    float4 n = __ldg((const float4*)(g.rt[1] + (size_t)y * g.pitch[1]) + x);
    return normalize3(xyz(n));
  } else {
    unsigned int bits = __ldg((const unsigned int*)(g.rt[1] + (size_t)y * g.pitch[1]) + x);
    return oct_decode(*reinterpret_cast<const __half2*>(&bits));
  }
}

// Validation helpers shared by the entry points.
epbr_status validate_gbuffer(const epbr_gbuffer* g, bool need_material);
epbr_status validate_camera(const epbr_camera* c, const epbr_gbuffer* g);
epbr_status validate_env(const epbr_env* e);

}  // namespace epbr
