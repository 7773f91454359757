/*
 * epbr.h — C ABI of libepbr, a GB300 (sm_103a) implementation of the per-pixel deferred
 * physically-based shading pass of EasyPBR (Rosu & Behnke, "EasyPBR: A Lightweight
 * Physically-Based Renderer", arXiv 2012.03325).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an epbr_status.  On failure a thread-local message is available
 *    from epbr_last_error().  No C++ exception crosses this boundary.
 *  - The caller owns every buffer.  Buffers named "device" are CUDA device pointers on the
 *    current device; "host" structs are read during the call only and may be freed after it
 *    returns.  The library never frees caller memory and keeps no pointer after a call returns
 *    (except the objects with an explicit create/destroy pair).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All device
 *    work is enqueued asynchronously on it.  Argument validation is synchronous and happens
 *    before anything is enqueued; on a validation error nothing is enqueued.
 *  - Images are row-major; `pitch` arguments are bytes between consecutive rows and must be a
 *    multiple of 16 bytes for 16-byte texel formats (float4) and of the texel size otherwise.
 *  - Pixel (x, y) has its centre at (x + 0.5, y + 0.5); y grows downwards; the camera looks
 *    along its local -z axis.
 *  - Environment maps are equirectangular.  Direction d maps to
 *        u = 0.5 + atan2(d.x, -d.z) / (2 pi),   v = atan2(sqrt(d.x^2 + d.z^2), d.y) / pi,
 *    texel (i, j) has its centre at ((i + 0.5)/W, (j + 0.5)/H); bilinear filtering wraps in u
 *    and clamps in v.  (The paper stores the environment as a cubemap, Sec. 3.1; equirect is
 *    the representation used here.)
 */
#ifndef EPBR_H
#define EPBR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------------------------------- */
/* Status                                                                                   */
/* ---------------------------------------------------------------------------------------- */
typedef int32_t epbr_status;
enum {
  EPBR_OK = 0,
  EPBR_ERR_INVALID_ARG = 1,   /* a pointer, size, pitch, format or flag is invalid */
  EPBR_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement */
  EPBR_ERR_CUDA = 3,          /* a CUDA runtime call failed; message has cudaGetErrorString */
  EPBR_ERR_NO_MEMORY = 4,     /* workspace too small or a library-owned allocation failed */
  EPBR_ERR_ADMISSION = 5,     /* serving: request can never fit the memory budget */
  EPBR_ERR_TIMEOUT = 6,       /* a bounded wait ran out */
  EPBR_ERR_DEVICE_STATUS = 7  /* a kernel reported an error through its device status word */
};

/* Thread-local message describing the last failure of a call made by this thread. */
const char* epbr_last_error(void);
/* Library version string. */
const char* epbr_version(void);

/* ---------------------------------------------------------------------------------------- */
/* Scene description                                                                        */
/* ---------------------------------------------------------------------------------------- */

/* Pinhole camera.  view_to_world is a column-major 4x4 rigid transform: columns 0..2 are the
 * camera's x (right), y (up) and z (backwards) axes in world space, column 3 is the eye.
 * A pixel's view-space ray is r = (px, py, -1) with
 *   px = (2 (x + 0.5) / width - 1) * tan(fov_y / 2) * width / height,
 *   py = (1 - 2 (y + 0.5) / height) * tan(fov_y / 2),
 * and the surface point at eye depth e is e * r (view space).  Host struct. */
typedef struct epbr_camera {
  float view_to_world[16];
  float fov_y;       /* radians, in (0, pi) */
  int32_t width;     /* full-resolution pixels, >= 1 */
  int32_t height;    /* >= 1 */
} epbr_camera;

/* Point light: position, intensity and colour (Sec. 6 names exactly these three).
 * Radiance arriving at P is intensity * color / |pos - P|^2; no range cutoff, no shadow.
 * Arrays of lights live in DEVICE memory, 32 bytes each. */
typedef struct epbr_light {
  float pos[3];
  float intensity;
  float color[3];
  float pad;
} epbr_light;

/* G-buffer (Table 1 of the paper gives four render targets; Sec. 4 stores depth instead of
 * position).  Two storage formats:
 *   EPBR_GBUFFER_FP32     rt[0] float4 (albedo.r, albedo.g, albedo.b, metalness)  16 B/px
 *                         rt[1] float4 (normal.x, normal.y, normal.z, roughness)  16 B/px
 *                         rt[2] unused (may be NULL)
 *                         rt[3] float  eye depth e > 0, +inf where no surface      4 B/px
 *   EPBR_GBUFFER_COMPACT  rt[0] uchar4 (sRGB8 albedo r, g, b, weight)              4 B/px
 *                         rt[1] half2  octahedral unit normal (Cigolle et al. 2014) 4 B/px
 *                         rt[2] uchar2 (UNORM8 metalness, UNORM8 roughness)         2 B/px
 *                         rt[3] float  eye depth e, as above                        4 B/px
 * Normals are in world space.  Albedo is linear in FP32 form and sRGB-encoded in COMPACT form.
 * Roughness is clamped to [0.045, 1] and metalness to [0, 1] when decoded.  All rt pointers
 * are DEVICE pointers; pitch[i] is bytes per row of rt[i].  The weight channel (used by the
 * paper for surfel accumulation) is carried but not read.  Host struct. */
enum { EPBR_GBUFFER_FP32 = 0, EPBR_GBUFFER_COMPACT = 1 };
typedef struct epbr_gbuffer {
  int32_t format;
  int32_t width;
  int32_t height;
  int32_t reserved;
  const void* rt[4];
  int64_t pitch[4];
} epbr_gbuffer;

/* HDR environment map (Sec. 3.1: every texel acts as a light source).  DEVICE float4 texels
 * (r, g, b, ignored), dense rows of `width` texels, at most 2^28 texels.  Host struct. */
typedef struct epbr_env {
  const float* texels;
  int32_t width;
  int32_t height;
} epbr_env;

/* ---------------------------------------------------------------------------------------- */
/* Image-based lighting precompute (Sec. 3.1; split sum of Karis 2013)                     */
/* ---------------------------------------------------------------------------------------- */
#define EPBR_MAX_LEVELS 16

typedef struct epbr_ibl_params {
  int32_t num_levels;         /* M in [1, EPBR_MAX_LEVELS]: specular mips, level m has
                                 roughness m / (M - 1) (level 0 = copy of the source) */
  int32_t prefilter_samples;  /* GGX importance samples per prefiltered texel, >= 1 */
  int32_t lut_size;           /* S: the BRDF LUT is S x S float2, >= 1 */
  int32_t lut_samples;        /* GGX samples per LUT texel, >= 1 */
  int32_t irr_width;          /* diffuse irradiance map size (equirect), >= 1 */
  int32_t irr_height;
} epbr_ibl_params;

/* Precomputed lighting set, all DEVICE pointers into one caller-owned buffer:
 *   irradiance  float4[irr_height][irr_width]  cosine-weighted mean radiance E(n)/pi
 *   lut         float2[S][S]   row j = roughness (j + 0.5)/S, column i = n.v = (i + 0.5)/S,
 *                              value (A, B) with F_ss E_ss = F0 A + B
 *   level[m]    float4[level_height[m]][level_width[m]], sizes max(1, W_e >> m) x
 *               max(1, H_e >> m)
 * Filled by epbr_ibl_layout; read by epbr_shade.  Host struct. */
typedef struct epbr_ibl {
  float* irradiance;
  int32_t irr_width;
  int32_t irr_height;
  float* lut;
  int32_t lut_size;
  int32_t num_levels;
  float* level[EPBR_MAX_LEVELS];
  int32_t level_width[EPBR_MAX_LEVELS];
  int32_t level_height[EPBR_MAX_LEVELS];
} epbr_ibl;

/* Computes the size of one lighting set for an env of env_width x env_height texels.  If
 * `buffer` is NULL only *bytes is written.  Otherwise `buffer` must be a DEVICE allocation of
 * at least *bytes bytes aligned to 256 B, and *out receives pointers into it (each sub-array
 * 256-B aligned).  Host-only: enqueues nothing. */
epbr_status epbr_ibl_layout(const epbr_ibl_params* params, int32_t env_width,
                            int32_t env_height, void* buffer, size_t* bytes, epbr_ibl* out);

/* Workspace bytes that epbr_precompute_ibl / epbr_irradiance need (the irradiance reduction
 * keeps per-block partial sums there). */
epbr_status epbr_precompute_ibl_workspace_size(const epbr_ibl_params* params,
                                               int32_t env_width, int32_t env_height,
                                               size_t* bytes);

/* Full lighting-set precompute for one environment (Sec. 3.1: "increasingly blurrier
 * versions" for the diffuse term, split-sum prefiltered mips plus a BRDF integration table for
 * the specular term).  Runs epbr_brdf_lut, epbr_irradiance and epbr_prefilter on `stream`.
 * `ibl` must come from epbr_ibl_layout with the same params and env size.  `workspace` is a
 * DEVICE buffer of at least epbr_precompute_ibl_workspace_size bytes, 256-B aligned. */
epbr_status epbr_precompute_ibl(const epbr_env* env, const epbr_ibl_params* params,
                                const epbr_ibl* ibl, void* workspace, size_t workspace_bytes,
                                void* stream);

/* BRDF integration table (split sum, second factor; Sec. 3.1 citing Karis 2013).  For texel
 * (i, j): mu = (i + 0.5)/S, r = (j + 0.5)/S, alpha = r^2, v = (sqrt(1 - mu^2), 0, mu),
 * n = (0, 0, 1), Hammersley points (k/N, radical_inverse_2(k)), GGX half vectors, l = reflect.
 * A = (1/N) sum_{n.l>0} (1 - Fc) Gvis,  B = (1/N) sum_{n.l>0} Fc Gvis,  Fc = (1 - v.h)^5,
 * Gvis = G(n.l, n.v) (v.h) / ((n.h)(n.v)),  G Smith-Schlick with k = alpha / 2.
 * `lut` is DEVICE float2[S][S]. */
epbr_status epbr_brdf_lut(int32_t lut_size, int32_t num_samples, float* lut, void* stream);

/* Diffuse irradiance map: for output texel direction n,
 *   out(n) = sum_t L_t max(n.d_t, 0) Omega_t / sum_t max(n.d_t, 0) Omega_t
 * over every source texel t (exact row solid angle Omega_t), i.e. E(n)/pi as a ratio
 * estimator, exact for a uniform environment (0 where no texel centre lies in the hemisphere
 * of n, which only maps of one or two columns allow).  `out` is DEVICE float4[irr_h][irr_w].
 * `workspace` as for epbr_precompute_ibl. */
epbr_status epbr_irradiance(const epbr_env* env, int32_t irr_width, int32_t irr_height,
                            float* out, void* workspace, size_t workspace_bytes, void* stream);

/* Irradiance as epbr_irradiance, for callers that cannot allocate device memory: an engine or
 * tool plugin whose host application owns the whole device-memory budget and forbids foreign
 * allocations, or a frame loop that must not call cudaMalloc because it can synchronise the
 * device and stall the frame.  No counterpart in the paper.
 *  - Scratch: the per-block partial sums live in one library-owned device array of 8 MiB
 *    (every GPU that loads the library holds it until the process exits).  A request needing
 *    more (irr_width * irr_height * min(608, ceil(env texels / 1024)) * 16 bytes) is refused
 *    with EPBR_ERR_INVALID_ARG and nothing is enqueued; the default 32x16 map over a
 *    2048x1024 environment needs 4.75 MiB.
 *  - Set-up: the first call on each device looks up the array's device address with that
 *    device current (cudaGetSymbolAddress); make that first call before any stream capture.
 *    The address belongs to the context current at the call (the primary context, or a
 *    caller's own driver context): it is cached per device together with that context's
 *    unique id and looked up again when a call finds another context current, e.g. after
 *    cudaDeviceReset or from a caller's own context.
 *  - Sharing: every call on a device uses the same array, which keeps the previous call's
 *    contents (each call writes every partial it reads, so nothing needs clearing).  Calls
 *    whose work overlaps on the GPU (other streams, other threads) race on the array: order
 *    them on one stream or with events.
 * `out` is DEVICE float4[irr_h][irr_w]; no workspace argument. */
epbr_status epbr_irradiance_noalloc(const epbr_env* env, int32_t irr_width, int32_t irr_height,
                                    float* out, void* stream);

/* Specular prefilter chain (split sum, first factor): level 0 is a copy of the source; level
 * m >= 1 with roughness r = m/(M-1), alpha = r^2 and n = v = texel direction is
 *   sum_k L(l_k) (n.l_k) / sum_k (n.l_k)  over the GGX half vectors of N Hammersley points,
 * keeping n.l_k > 0, with L read bilinearly from the source.  `ibl` levels are written. */
epbr_status epbr_prefilter(const epbr_env* env, int32_t num_samples, const epbr_ibl* ibl,
                           void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Screen-space ambient occlusion (Sec. 5.2: normal-oriented hemisphere of Bavoil & Sainz     */
/* 2008, computed at half resolution and bilaterally blurred)                               */
/* ---------------------------------------------------------------------------------------- */
typedef struct epbr_ssao_params {
  int32_t num_samples;   /* K >= 1 */
  int32_t scale;         /* 1: AO at full resolution, 2: half resolution (the paper's) */
  float radius;          /* hemisphere radius, world/view units, > 0 */
  float bias;            /* depth bias, >= 0 */
  int32_t blur_radius;   /* bilateral blur half-width in AO texels (3 = 7x7), 0..8 */
  float sigma_s;         /* blur spatial sigma, AO texels, > 0 */
  float sigma_z;         /* blur relative depth sigma, > 0 */
  int32_t reserved;
  const float* kernel;   /* DEVICE float4[K]: tangent-space sample offsets (x, y, z > 0, -) */
  const float* noise;    /* DEVICE float2[16]: 4x4 tiled rotation vectors (view-space x, y) */
} epbr_ssao_params;

/* AO image size for a view: ceil(width/scale) x ceil(height/scale) floats. */
epbr_status epbr_ssao_size(const epbr_gbuffer* gbuffer, const epbr_ssao_params* params,
                           int32_t* ao_width, int32_t* ao_height);
/* Workspace bytes for epbr_ssao (the unblurred AO image). */
epbr_status epbr_ssao_workspace_size(const epbr_gbuffer* gbuffer,
                                     const epbr_ssao_params* params, size_t* bytes);

/* Unblurred AO.  AO texel (i, j) uses full-resolution pixel (scale*i, scale*j): view-space
 * point P and normal n; noise vector (noise[(j%4)*4 + i%4], 0) made orthogonal to n gives the
 * tangent frame (fallback to a branchless orthonormal basis when it is parallel to n).  Sample
 * S_k = P + radius * TBN * kernel[k] is projected to pixel (floor X, floor Y); its depth e_b is
 * fetched; the sample occludes by [e_b <= e_S - bias] * smoothstep(0, 1, radius / |e_P - e_b|).
 * Off-screen, behind-camera and background samples do not occlude.  AO = 1 - sum / K.  AO of a
 * background pixel is 1.  `ao` is DEVICE float, rows of `ao_pitch` bytes.  EPBR_ERR_UNSUPPORTED
 * when the depth plane spans more than 2^32 texels (height x pitch[3] / 4).  Scheduling: its
 * blocks release programmatic dependents (a kernel launched next with programmatic stream
 * serialisation, such as epbr_ssao_blur) at their start; results do not depend on it. */
epbr_status epbr_ssao_raw(const epbr_gbuffer* gbuffer, const epbr_camera* camera,
                          const epbr_ssao_params* params, float* ao, int64_t ao_pitch,
                          void* stream);

/* Whether epbr_ssao_raw takes its tiled form for this G-buffer (*tiled = 1) or not (0).  The
 * tiled form (the same values bit for bit) copies each block's depth footprint plus a 32-pixel
 * halo into shared memory with one TMA tile load, and a warp whose samples all project inside
 * that tile reads its taps from it; it applies at scale 2 to views of at most 1536 rows when the
 * depth plane rt[3] starts on a 16-byte boundary and its pitch is a multiple of 16 bytes (below
 * 2^40) and the driver provides cuTensorMapEncodeTiled.  Synchronous, enqueues nothing. */
epbr_status epbr_ssao_tiled(const epbr_gbuffer* gbuffer, const epbr_ssao_params* params,
                            int32_t* tiled);

/* Number of tiled-form warps whose first wait for their depth tile ran out (50 ms by default)
 * since the last call, then reset to 0.  Such warps read every tap from the depth plane instead,
 * so their AO is unaffected; a nonzero count means a copy stalled.  Such a block waits once more
 * (50 ms) before it exits; if that wait runs out too, its copy may still land in shared memory
 * that a later block uses, and this call returns EPBR_ERR_DEVICE_STATUS (with *count set, the
 * flag cleared): treat the AO of the launches since the previous call as suspect.  Synchronous
 * copies on the current device; the launches it should cover must have completed (synchronise
 * their stream first). */
epbr_status epbr_ssao_tile_timeouts(uint32_t* count);

/* Test hook for the fallback paths of the library's TMA staging: sets the limit of the first wait
 * for a staged copy (nanoseconds, at most the default 50 ms) used by later launches — the SSAO
 * depth tiles of epbr_ssao_raw and the compose's light list (epbr_shade, epbr_shade_tonemap) —
 * and returns the previous limit in *previous_ns (nullable).  0 makes every tiled SSAO warp and
 * every compose block give up at once, read global memory instead (the same results) and count
 * itself in epbr_ssao_tile_timeouts / epbr_shade_light_timeouts; the second wait before a block
 * exits keeps its 50 ms bound.  Process-wide; not for production use.  EPBR_ERR_INVALID_ARG
 * above the default. */
epbr_status epbr_ssao_set_tile_wait(uint64_t first_wait_ns, uint64_t* previous_ns);

/* Depth-aware blur of an AO image: out_p = sum_q w_q ao_q / sum_q w_q over the
 * (2R+1)^2 window (clipped to the image) with w_q = exp(-(dx^2+dy^2)/(2 sigma_s^2)) *
 * exp(-|e_q - e_p| / (sigma_z e_p)), background taps weighted 0; background pixels get 1.
 * Scheduling: launched as a programmatic dependent of the previous kernel on the stream; every
 * block waits for that kernel to finish (griddepcontrol.wait) before its first memory access, and
 * only then releases its own dependents (a compose launched with EPBR_SHADE_EARLY_START).
 */
epbr_status epbr_ssao_blur(const epbr_gbuffer* gbuffer, const epbr_ssao_params* params,
                           const float* ao_in, int64_t in_pitch, float* ao_out,
                           int64_t out_pitch, void* stream);

/* epbr_ssao_raw into `workspace`, then epbr_ssao_blur into `ao` (blur_radius 0: copy). */
epbr_status epbr_ssao(const epbr_gbuffer* gbuffer, const epbr_camera* camera,
                      const epbr_ssao_params* params, float* ao, int64_t ao_pitch,
                      void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Deferred compose (Sec. 3 Eq. 1 with the UE4 Cook-Torrance model; Sec. 3.1 IBL with the     */
/* multiple-scattering extension of Fdez-Aguera 2019; Sec. 5.4 compositing)                 */
/* ---------------------------------------------------------------------------------------- */
enum {
  EPBR_SHADE_DIRECT = 1,        /* sum over point lights */
  EPBR_SHADE_IBL = 2,           /* split-sum ambient term (needs ibl) */
  EPBR_SHADE_MULTISCATTER = 4,  /* Fdez-Aguera energy compensation of the IBL term */
  EPBR_SHADE_DIFFUSE_ONLY = 8,  /* Lambert only: albedo/pi direct, albedo*irradiance ambient */
  EPBR_SHADE_ALL = 7,
  /* Scheduling only (the image is the same): the compose may start while the kernel just
   * before it on the stream is still running (programmatic dependent launch).  It decodes the
   * G-buffer and sums the point lights at once, and waits for that kernel to finish before it
   * reads the AO image and before it writes its outputs.  Set it only when that kernel writes
   * none of the G-buffer, the lights, the lighting set and the shadow maps, and reads none of
   * the outputs: the SSAO passes of this library (epbr_ssao_raw, epbr_ssao_blur, epbr_ssao)
   * qualify, and the blur lets a compose start only after the raw AO it reads has finished. */
  EPBR_SHADE_EARLY_START = 16
};
enum { EPBR_HDR_RGBA32F = 0, EPBR_HDR_RGBA16F = 1 };

typedef struct epbr_shade_params {
  uint32_t flags;        /* EPBR_SHADE_* */
  int32_t ao_scale;      /* pixel (x, y) reads ao[(y/ao_scale) * pitch + x/ao_scale] */
  const float* ao;       /* DEVICE AO image or NULL (AO = 1); multiplies the ambient term */
  int64_t ao_pitch;      /* bytes */
} epbr_shade_params;

/* Per pixel: decode the G-buffer, reconstruct P from depth, v = normalize(eye - P),
 *   L_direct = sum_i [ (1 - F) c_diff / pi + D G F / (4 (n.l)(n.v)) ] I_i c_i / d_i^2 (n.l)
 * for n.l > 0 (GGX D with alpha = r^2, Smith-Schlick G with k = (r + 1)^2 / 8, Schlick F from
 * F0 = mix(0.04, albedo, metal), c_diff = albedo (1 - metal), n.v clamped to >= 1e-4), plus the
 * split-sum ambient term times AO.  Background pixels (e = +inf) get the environment's level 0
 * along the view ray (0 without IBL).  Output: DEVICE RGBA32F or RGBA16F (round to nearest,
 * saturated to +-65504), alpha = 1.  `lights` is DEVICE epbr_light[num_lights], num_lights in
 * [0, 65536].  `ibl` may be NULL when flags has no EPBR_SHADE_IBL. */
epbr_status epbr_shade(const epbr_gbuffer* gbuffer, const epbr_camera* camera,
                       const epbr_light* lights, int32_t num_lights, const epbr_ibl* ibl,
                       const epbr_shade_params* params, void* hdr, int32_t hdr_format,
                       int64_t hdr_pitch, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Tone mapping (Sec. 5.4: ACES, optional Reinhard, then gamma correction)                  */
/* ---------------------------------------------------------------------------------------- */
enum { EPBR_TONEMAP_ACES = 0, EPBR_TONEMAP_REINHARD = 1 };
typedef struct epbr_tonemap_params {
  float exposure;  /* x = exposure * hdr */
  int32_t op;      /* EPBR_TONEMAP_ACES (Narkowicz 2015 fit) or EPBR_TONEMAP_REINHARD x/(1+x) */
} epbr_tonemap_params;

/* out = round_half_up(255 * sRGB_OETF(clamp(op(x), 0, 1))), alpha 255, where
 * x = clamp(exposure * hdr.rgb, 0, 1e6) (NaN counts as 0; both operators are saturated long
 * before 1e6, and the clamp keeps +inf from turning the ACES ratio into NaN).
 * `hdr` DEVICE RGBA32F/RGBA16F, `out` DEVICE uchar4. */
epbr_status epbr_tonemap(const void* hdr, int32_t hdr_format, int32_t width, int32_t height,
                         int64_t hdr_pitch, const epbr_tonemap_params* params, uint8_t* out,
                         int64_t out_pitch, void* stream);

/* epbr_shade with the tone map fused into its epilogue: the 8-bit image is always written,
 * the HDR image only when `hdr` is not NULL.  With RGBA32F the result equals epbr_shade
 * followed by epbr_tonemap; with RGBA16F the tone map reads the FP32 value before rounding. */
epbr_status epbr_shade_tonemap(const epbr_gbuffer* gbuffer, const epbr_camera* camera,
                               const epbr_light* lights, int32_t num_lights, const epbr_ibl* ibl,
                               const epbr_shade_params* params, void* hdr, int32_t hdr_format,
                               int64_t hdr_pitch, const epbr_tonemap_params* tonemap,
                               uint8_t* ldr, int64_t ldr_pitch, void* stream);

/* epbr_shade and epbr_shade_tonemap copy a list of at most 256 lights into each block's shared
 * memory with one TMA bulk copy.  Number of compose blocks whose wait for that copy ran out (50 ms
 * by default; epbr_ssao_set_tile_wait sets this first wait too) since the last call, then reset
 * to 0.  Such blocks read the list from global memory instead, so their result is unaffected.
 * Such a block waits once more (50 ms) before it exits; if that wait runs out too, its copy may
 * still land in shared memory that a later block uses, and this call returns
 * EPBR_ERR_DEVICE_STATUS (with *count set, the flag cleared).  Synchronous copies on the current
 * device; synchronise the launches' stream first. */
epbr_status epbr_shade_light_timeouts(uint32_t* count);

/* ---------------------------------------------------------------------------------------- */
/* The G-buffer pass of mesh rendering (Sec. 4.1): triangles rasterised into the G-buffer    */
/* ---------------------------------------------------------------------------------------- */
typedef struct epbr_mesh {
  const float* vertices;     /* DEVICE float[num_vertices * 12], 16-byte aligned: world position xyz,
                                normal xyz, albedo rgb, metal, rough, unused */
  int32_t num_vertices;      /* 0 .. 2^28 */
  const int32_t* triangles;  /* DEVICE int32[num_triangles * 3] vertex indices (any winding) */
  int32_t num_triangles;
} epbr_mesh;

/* Device workspace epbr_raster_gbuffer needs: 8 B per pixel (nearest (depth, triangle) key),
 * 64 B and 8 B per triangle (set-up, item offsets), each part 256-byte aligned. */
epbr_status epbr_raster_workspace_size(int32_t num_triangles, int32_t width, int32_t height, size_t* bytes);

/* Writes the FP32 G-buffer `out` (rt[0] albedo + metal, rt[1] normal + rough, rt[3] eye depth;
 * background: zeros and depth +inf) of the mesh seen by `camera`.  Pixel (x, y) is covered by
 * a triangle when its centre lies inside it: vertices are transformed to view space and
 * projected in FP32 with every product, sum and quotient rounded, snapped to 1/256 pixel (round
 * half to even), and tested with 64-bit integer edge functions under a top-left rule, so that a
 * centre on an edge shared by two triangles belongs to exactly one.  The nearest covering
 * triangle writes the pixel: smallest FP32 eye depth A / ((b_a iz_a + b_b iz_b) + b_c iz_c)
 * (b the edge functions, A their sum, iz = 1/z), then smallest index.  Attributes are
 * interpolated perspective-correctly (weights b_i iz_i normalised), the normal normalised.  No
 * clipping and no back-face culling: a triangle with a vertex at eye depth below `near_depth`
 * (> 0), or projecting beyond 2^22 pixels, is not drawn.  `ids` (DEVICE int32, NULL allowed)
 * receives the winning triangle index, -1 for background.  `workspace` DEVICE, 256-byte
 * aligned, at least epbr_raster_workspace_size bytes.  Stream-ordered; no allocation. */
epbr_status epbr_raster_gbuffer(const epbr_mesh* mesh, const epbr_camera* camera, float near_depth,
                                const epbr_gbuffer* out, int32_t* ids, int64_t ids_pitch, void* workspace,
                                size_t workspace_bytes, void* stream);

/* Device workspace epbr_shadow_maps needs for maps of size x size texels: the key images and
 * triangle set-ups of up to 8 lights at a time (8 x (8 B per texel + 72 B per triangle), about
 * 130 MB for 512^2 maps of a 200,000-triangle mesh), reused group after group. */
epbr_status epbr_shadow_maps_workspace_size(int32_t num_triangles, int32_t size, size_t* bytes);

/* Shadow maps by rendering the mesh "only as a depth map" from each light as from a normal
 * camera (Sec. 5.1): map i is the eye depth of the mesh seen by cameras[i] (square, every camera
 * of the same size S, field of view in (0, 3.1) rad), exactly the depth plane epbr_raster_gbuffer
 * writes for that camera (same coverage, depth and tie rules; +inf where nothing is drawn).
 * `maps` is DEVICE float[num_maps][S][S] (dense rows), the layout epbr_shadows.maps takes; the
 * cameras are host structs (the world -> light-view rows epbr_shadows.cameras holds for shading
 * are the inverse of each camera's view_to_world).  Up to 8 lights are rendered by one set of
 * launches (set-up, scan, coverage, depth), groups one after the other through `workspace`
 * (DEVICE, 256-byte aligned, epbr_shadow_maps_workspace_size bytes), stream-ordered; no
 * allocation.  EPBR_ERR_UNSUPPORTED above 2^28 triangles.  Re-render when the scene or a light
 * moves. */
epbr_status epbr_shadow_maps(const epbr_mesh* mesh, const epbr_camera* cameras, int32_t num_maps,
                             float near_depth, float* maps, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* The G-buffer pass of surfel rendering (Sec. 4.3): elliptical disks splatted and blended   */
/* ---------------------------------------------------------------------------------------- */
typedef struct epbr_surfels {
  const float* records;  /* DEVICE float[num_surfels * 16], 16-byte aligned: centre xyz, semi-axis a
                            (along the tangent), normal xyz, semi-axis b (along the bitangent),
                            tangent xyz, metal, albedo rgb, rough (world space) */
  int32_t num_surfels;   /* 0 .. 2^28 */
  int32_t reserved;
} epbr_surfels;

/* Device workspace epbr_surfel_gbuffer needs: 40 B per pixel (nearest depth, nine attribute
 * sums), 4 B per pixel column and row (pixel rays), 96 B and 8 B per surfel (set-up, task
 * offsets), each part 256-byte aligned. */
epbr_status epbr_surfel_workspace_size(int32_t num_surfels, int32_t width, int32_t height, size_t* bytes);

/* Writes the FP32 G-buffer `out` (rt[0] albedo + metal, rt[1] normal + rough, rt[3] eye depth;
 * background: zeros and depth +inf) of the surfels seen by `camera`.  A surfel is the ellipse of
 * semi-axes a, b in the plane through its centre with its normal, a along the tangent made
 * orthogonal to the normal, b along the bitangent normal x tangent; both faces are drawn.  A
 * surfel is dropped when its normal or orthogonalised tangent is zero, a semi-axis is not a
 * positive finite number, or (eye depth of its centre) - (a + b) < near_depth.  Pixel (x, y) is
 * covered when the ray through its centre meets the surfel's plane at eye depth s > 0 inside the
 * ellipse.  The pixel's depth is the smallest s; every covering surfel with
 * s <= depth * (1 + depth_tolerance) adds its albedo, unit normal, metal and rough with weight 1,
 * and the G-buffer holds their means (the normal renormalised).  These decisions are evaluated in
 * FP32 with every product, sum, quotient and square root rounded, in a fixed order, so they are
 * reproducible bit for bit; the sums are float atomics (their order varies).  `weight` (DEVICE
 * float, NULL allowed, rows of weight_pitch bytes) receives the number of blended surfels, 0 for
 * background.  `workspace` DEVICE, 256-byte aligned, at least epbr_surfel_workspace_size bytes.
 * Stream-ordered; no allocation. */
epbr_status epbr_surfel_gbuffer(const epbr_surfels* surfels, const epbr_camera* camera, float near_depth,
                                float depth_tolerance, const epbr_gbuffer* out, float* weight,
                                int64_t weight_pitch, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Eye-dome lighting for point clouds (Sec. 4.2; Boucheny 2009): shading from depth alone    */
/* ---------------------------------------------------------------------------------------- */
typedef struct epbr_edl_params {
  float strength;      /* A >= 0 */
  int32_t radius;      /* r: neighbour distance in pixels, 1..8 */
  int32_t directions;  /* N: neighbours at angles 2 pi k / N, 1..16 */
} epbr_edl_params;

/* Per pixel p with a surface: w = (1/N) sum_k max(0, log2 e_p - log2 e_{q_k}), q_k = p +
 * (round(r cos(2 pi k/N)), round(r sin(2 pi k/N))) (round half away from zero), a neighbour
 * outside the image or without a surface counting as infinitely far; output = G-buffer colour
 * (rt[0]: FP32 rgb, or sRGB8 in the compact layout) * exp(-A w) * AO; background pixels 0,
 * alpha 1.  The G-buffer needs rt[0] and the depth rt[3] only (a point cloud has no normals).
 * `ao` DEVICE or NULL (read at (x/ao_scale, y/ao_scale), ao_scale 1..8).  Outputs `hdr` (NULL
 * allowed) and `ldr` (NULL allowed, needs `tonemap`), at least one. */
epbr_status epbr_edl(const epbr_gbuffer* gbuffer, const epbr_edl_params* params, const float* ao, int64_t ao_pitch,
                     int32_t ao_scale, void* hdr, int32_t hdr_format, int64_t hdr_pitch,
                     const epbr_tonemap_params* tonemap, uint8_t* ldr, int64_t ldr_pitch, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Shadow maps with 3x3 percentage-closer filtering for the point lights (Sec. 5.1; Williams */
/* 1978, Reeves et al. 1987)                                                                 */
/* ---------------------------------------------------------------------------------------- */
typedef struct epbr_shadows {
  const float* maps;     /* DEVICE: one size x size map per light, map i at maps + i*size*size,
                            row-major eye depths along the light camera's view axis, +inf where
                            the map holds no surface; 4-byte aligned */
  const float* cameras;  /* DEVICE float[num_lights * 16], 16-byte aligned: per light the rows of
                            the world -> light-view matrix (12 floats; the light camera looks along
                            -z, x right, y up), then f = 1 / tan(fov / 2), then 3 unused */
  int32_t size;          /* S: map width and height, 1..8192 */
  float bias_const;      /* b0 >= 0 */
  float bias_slope;      /* b1 >= 0: a tap lights the fragment when z <= d + b0 + b1 z */
} epbr_shadows;

/* epbr_shade_tonemap with each light's direct term multiplied by its visibility: the fragment
 * P maps to light-view q, depth z = -q.z, texel coordinates s = (q.x f / z + 1) S/2,
 * t = (1 - q.y f / z) S/2, texel (floor s, floor t); visibility = lit taps of the 3x3 block
 * around that texel / 9, a tap outside the map and a fragment behind the light (z <= 0) being
 * lit.  The ambient term and background are unshadowed.  Outputs: `hdr` (NULL allowed) and
 * `ldr` (NULL allowed, needs `tonemap`), at least one.  The maps are the caller's (render them
 * once and reuse them while the scene and lights stay still, as Sec. 5.1 does). */
epbr_status epbr_shade_shadows(const epbr_gbuffer* gbuffer, const epbr_camera* camera, const epbr_light* lights,
                               int32_t num_lights, const epbr_ibl* ibl, const epbr_shade_params* params,
                               const epbr_shadows* shadows, void* hdr, int32_t hdr_format, int64_t hdr_pitch,
                               const epbr_tonemap_params* tonemap, uint8_t* ldr, int64_t ldr_pitch, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Bloom (Sec. 5.3: bright map, image pyramid of up to six levels blurred from the second one */
/* upwards, added onto the image)                                                            */
/* ---------------------------------------------------------------------------------------- */
typedef struct epbr_bloom_params {
  float threshold;  /* a pixel enters the bright map when its luminance exceeds this */
  float strength;   /* s: factor of the added levels, >= 0 */
  float sigma;      /* Gaussian sigma in texels of each level, > 0 */
  int32_t radius;   /* R: blur taps on each side, 0..8 */
  int32_t levels;   /* L: pyramid levels including the full-resolution bright map, 2..6 */
} epbr_bloom_params;

/* Device workspace epbr_bloom needs for a width x height image: levels 1 .. L-1 before and
 * after the blur, RGBA32F, each 256-byte aligned. */
epbr_status epbr_bloom_workspace_size(int32_t width, int32_t height, const epbr_bloom_params* params,
                                      size_t* bytes);

/* Y = X + s * sum_{k=1}^{L-1} U_k, per pixel, where
 *   bright map B = X where lum(X) > threshold, else 0; lum = (0.2126 R + 0.7152 G) + 0.0722 B
 *     evaluated in FP32 with every product and sum rounded (no contraction);
 *   level 0 = B; level k = 2x2 box average of level k-1, ceil(W_{k-1}/2) x ceil(H_{k-1}/2),
 *     clamped to the edge;
 *   levels 1 .. L-1 are blurred with a separable Gaussian of radius R, weights
 *     exp(-d^2 / (2 sigma^2)) normalised over |d| <= R, clamped to the edge;
 *   U_k = blurred level k sampled bilinearly (clamp to edge) at texel coordinate
 *     (x + 1/2) / 2^k - 1/2 for pixel x (likewise y).
 * `hdr` DEVICE RGBA32F/RGBA16F input (alpha ignored); `workspace` DEVICE, at least
 * epbr_bloom_workspace_size bytes, 16-byte aligned.  Outputs (at least one): `out_hdr` DEVICE
 * RGBA32F/RGBA16F (alpha 1; may equal `hdr` when the format and pitch are the same: every pixel
 * is read before it is written, by the same thread), and `ldr` DEVICE uchar4, the tone map of
 * Y with `tonemap` (required with `ldr`).  Stream-ordered; no allocation. */
epbr_status epbr_bloom(const void* hdr, int32_t hdr_format, int64_t hdr_pitch, int32_t width, int32_t height,
                       const epbr_bloom_params* params, void* workspace, size_t workspace_bytes,
                       void* out_hdr, int32_t out_format, int64_t out_pitch,
                       const epbr_tonemap_params* tonemap, uint8_t* ldr, int64_t ldr_pitch, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Batching: many views of uneven size in one persistent launch (a system form layered on the */
/* pass; the paper renders one view per frame, Sec. 4)                                       */
/* ---------------------------------------------------------------------------------------- */

/* One view of a batch.  All pointers DEVICE; the G-buffer format must be the same for every
 * view of a batch.  `ldr` (uchar4) is required, `hdr` optional (NULL). */
typedef struct epbr_view {
  epbr_gbuffer gbuffer;
  epbr_camera camera;
  const epbr_light* lights;
  int32_t num_lights;
  int32_t ibl_index;     /* index into the lighting sets passed with the batch */
  void* hdr;
  int64_t hdr_pitch;
  uint8_t* ldr;
  int64_t ldr_pitch;
} epbr_view;

typedef struct epbr_batch_params {
  uint32_t flags;                  /* EPBR_SHADE_* for every view */
  int32_t hdr_format;              /* EPBR_HDR_RGBA32F or EPBR_HDR_RGBA16F */
  epbr_ssao_params ssao;           /* shared; scale must be 2, blur_radius <= 4, <= 64 samples */
  epbr_tonemap_params tonemap;
  int32_t tile_w, tile_h;          /* fused-mode pixels per tile: 64x32, 128x32 or 64x64;
                                      0 = 64x32 */
  int32_t light_chunk;             /* fused-mode lights per shared-memory chunk, 1..256; 0 = 256 */
} epbr_batch_params;

/* Batch execution modes (a plan = mode + tile shape + light chunk):
 *   EPBR_BATCH_FUSED   one persistent kernel; per tile of tile_w x tile_h pixels: unblurred
 *                      SSAO with a halo, blur, compose, tone map, all in shared memory
 *   EPBR_BATCH_STAGED  three kernels (SSAO, blur, compose + tone map), each over the tiles of
 *                      every view, AO images in batch-owned memory; the graph joins them by
 *                      programmatic edges (the compose's light loop may run while the blur does,
 *                      its AO read waits for the blur)
 *   EPBR_BATCH_PER_VIEW epbr_ssao_raw, epbr_ssao_blur and epbr_shade_tonemap (with
 *                      EPBR_SHADE_EARLY_START) of every view, recorded into the graph by stream
 *                      capture: the per-view kernels without per-launch host work */
enum { EPBR_BATCH_FUSED = 0, EPBR_BATCH_STAGED = 1, EPBR_BATCH_PER_VIEW = 2 };

/* Library-owned batch: device copies of the view descriptors, the tile list and a CUDA graph
 * (memset of the tile counter -> the fused kernel).  The views' buffers are referenced, not
 * copied: relaunching renders whatever they hold at launch time. */
typedef struct epbr_batch epbr_batch;

/* Renders every view with the same arithmetic as epbr_ssao + epbr_shade_tonemap per view.
 * Allocates the batch's descriptors, tile lists and (staged mode) AO images — the one place
 * the library allocates device memory; synchronous.  Starts with the fused 64x32 plan. */
epbr_status epbr_batch_create(const epbr_view* views, int32_t n_views, const epbr_ibl* ibls,
                              int32_t n_ibls, const epbr_batch_params* params, epbr_batch** out);
/* Enqueues one replay of the batch's graph on `stream`. */
epbr_status epbr_batch_launch(epbr_batch* batch, void* stream);
/* Times every plan (each fused tile shape x light chunk, the staged and the per-view mode) on this batch and
 * keeps the fastest (synchronises `stream`).  With `cache_path`, a plan stored for the same
 * batch key is reused without timing, and new results are appended as text lines
 * "key mode tile_w tile_h chunk ms". */
epbr_status epbr_batch_autotune(epbr_batch* batch, const char* cache_path, void* stream);
epbr_status epbr_batch_get_plan(const epbr_batch* batch, int32_t* mode, int32_t* tile_w,
                                int32_t* tile_h, int32_t* light_chunk);
epbr_status epbr_batch_set_plan(epbr_batch* batch, int32_t mode, int32_t tile_w, int32_t tile_h,
                                int32_t light_chunk);
/* Waits for nothing: destroy only after the batch's launches have completed. */
epbr_status epbr_batch_destroy(epbr_batch* batch);
/* create + launch + wait for `stream` + destroy. */
epbr_status epbr_render_batch(const epbr_view* views, int32_t n_views, const epbr_ibl* ibls,
                              int32_t n_ibls, const epbr_batch_params* params, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Serving: a request loop with continuous batching (a system form layered on the pass; the   */
/* paper's stated use is generating synthetic training images, Sec. 8.1)                     */
/* ---------------------------------------------------------------------------------------- */
typedef struct epbr_serve_config {
  size_t memory_budget;         /* device bytes for admitted requests' buffers (one arena) */
  int32_t max_in_flight;        /* requests admitted at once */
  int32_t num_streams;          /* streams their work is spread over, 1..64 */
  const epbr_ibl* ibls;         /* resident lighting sets; must outlive the server */
  int32_t num_ibls;
  uint32_t flags;               /* EPBR_SHADE_* */
  epbr_ssao_params ssao;        /* scale must be 2; kernel/noise DEVICE pointers */
  epbr_tonemap_params tonemap;
} epbr_serve_config;

/* One render request.  All pointers are HOST memory that must stay valid until the request's
 * result has been collected (pinned memory lets the copies overlap other requests' work). */
typedef struct epbr_request {
  int32_t format;               /* EPBR_GBUFFER_FP32 or EPBR_GBUFFER_COMPACT, rows dense */
  int32_t width, height;
  int32_t ibl_index;            /* which resident lighting set */
  const void* rt[4];            /* G-buffer planes as in epbr_gbuffer */
  epbr_camera camera;
  const epbr_light* lights;
  int32_t num_lights;
  int32_t reserved;
  uint8_t* ldr_out;             /* width * height * 4 bytes, RGBA8 result */
  double deadline_ms;           /* > 0: cancelled (EPBR_ERR_TIMEOUT) if still queued after it */
} epbr_request;

typedef struct epbr_result {
  epbr_status status;           /* EPBR_OK, EPBR_ERR_TIMEOUT (cancelled in the queue), ... */
  int32_t deferred;             /* 1 if admission waited for memory */
  double queue_ms;              /* submit -> admission */
  double latency_ms;            /* submit -> result in host memory */
  char message[160];
} epbr_result;

typedef struct epbr_serve_stats {
  uint64_t submitted, admitted, completed, deferred, rejected, timed_out, failed;
  int32_t in_flight, queued;
  size_t bytes_in_use, peak_bytes;
} epbr_serve_stats;

typedef struct epbr_server epbr_server;

/* Allocates the arena and streams and starts the scheduler thread.  Requests are admitted in
 * arrival order whenever a slot is free and the arena can hold the request's G-buffer, lights,
 * AO images and 8-bit image; admitted requests run concurrently on the server's streams. */
epbr_status epbr_serve_create(const epbr_serve_config* config, epbr_server** out);
/* Device bytes a request occupies while admitted. */
epbr_status epbr_serve_request_bytes(const epbr_request* request, size_t* bytes);
/* Queues a request (thread-safe).  EPBR_ERR_ADMISSION when it alone exceeds the budget. */
epbr_status epbr_serve_submit(epbr_server* server, const epbr_request* request, uint64_t* ticket);
/* Non-blocking: *done = 1 and the result (ticket consumed) once the request has finished. */
epbr_status epbr_serve_poll(epbr_server* server, uint64_t ticket, int32_t* done, epbr_result* out);
/* Blocks up to timeout_ms; EPBR_ERR_TIMEOUT if the request is still running (ticket kept). */
epbr_status epbr_serve_wait(epbr_server* server, uint64_t ticket, int32_t timeout_ms, epbr_result* out);
epbr_status epbr_serve_get_stats(epbr_server* server, epbr_serve_stats* out);
/* Cancels queued requests, waits for admitted ones, frees everything. */
epbr_status epbr_serve_destroy(epbr_server* server);

#ifdef __cplusplus
}
#endif
#endif /* EPBR_H */
