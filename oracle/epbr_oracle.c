/*
 * epbr_oracle.c — plain, slow, double-precision CPU restatement of the deferred PBR shading
 * pass of EasyPBR (arXiv 2012.03325).  TEST INFRASTRUCTURE ONLY: it exists to check the CUDA
 * library and is called only by the test suite, the package's smoke check and the benchmark's
 * CPU-baseline leg.  It shares no code, header, table or constant generator with the CUDA
 * path and includes nothing from it.
 *
 * Each function follows the definition it cites, in the order the source states it, with no
 * blocking, fusion or reordering:
 *   - reflectance equation (paper Sec. 3, Eq. 1) with the Cook-Torrance model of UE4 (Sec. 3;
 *     Karis 2013: GGX distribution, Smith-Schlick geometry with k = (r+1)^2/8, Schlick Fresnel);
 *   - image-based lighting (Sec. 3.1): diffuse irradiance by exact quadrature, split-sum
 *     prefiltered environment and BRDF table (Karis 2013, Hammersley + GGX importance
 *     sampling, k = alpha/2), multiple-scattering compensation (Fdez-Aguera 2019);
 *   - G-buffer of Table 1 with position reconstructed from depth (Sec. 4);
 *   - normal-oriented hemisphere SSAO at half resolution with a bilateral blur (Sec. 5.2;
 *     Bavoil & Sainz 2008);
 *   - ACES filmic tone mapping (Narkowicz 2015 fit) or Reinhard, then the sRGB transfer
 *     function of IEC 61966-2-1 (Sec. 5.4);
 *   - shadow maps with 3x3 percentage-closer filtering for the point lights (Sec. 5.1;
 *     Williams 1978, Reeves et al. 1987);
 *   - eye-dome lighting for point clouds (Sec. 4.2; Boucheny 2009);
 *   - the G-buffer pass of mesh rendering (Sec. 4.1): triangle rasterisation with a depth test
 *     and perspective-correct attribute interpolation;
 *   - bloom (Sec. 5.3): bright map, an image pyramid of up to six levels, a Gaussian blur of
 *     every level from the second one up, the blurred levels added onto the image;
 *   - surfel splatting into the G-buffer (Sec. 4.3): elliptical disks on their (normal, tangent,
 *     bitangent) basis, the surfels within a small depth window of the nearest one blended.
 * Conventions the paper leaves open (equirect mapping, sample sets, SSAO constants, rounding)
 * are stated beside the code that uses them.
 *
 * Parity status: every function here is pinned by the CPU test suite (closed forms, invariants,
 * brute-force quadrature, special cases); see tests/test_oracle_pins.py.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------------ */
/* threads: split an index range into contiguous chunks                                       */
/* ------------------------------------------------------------------------------------------ */
typedef void (*or_body_fn)(void* ctx, long i0, long i1);
typedef struct {
  or_body_fn fn;
  void* ctx;
  long i0, i1;
} or_job;

static void* or_job_run(void* p) {
  or_job* j = (or_job*)p;
  j->fn(j->ctx, j->i0, j->i1);
  return NULL;
}

static int or_threads(int requested) {
  if (requested > 0) return requested;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

static void or_parallel_for(long n, int threads, or_body_fn fn, void* ctx) {
  int t = or_threads(threads);
  if (t > n) t = (int)(n > 0 ? n : 1);
  if (t <= 1) {
    fn(ctx, 0, n);
    return;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * t);
  or_job* jobs = (or_job*)malloc(sizeof(or_job) * t);
  for (int k = 0; k < t; ++k) {
    jobs[k].fn = fn;
    jobs[k].ctx = ctx;
    jobs[k].i0 = n * k / t;
    jobs[k].i1 = n * (k + 1) / t;
    pthread_create(&th[k], NULL, or_job_run, &jobs[k]);
  }
  for (int k = 0; k < t; ++k) pthread_join(th[k], NULL);
  free(th);
  free(jobs);
}

int or_num_threads(int requested) { return or_threads(requested); }

/* ------------------------------------------------------------------------------------------ */
/* small vector helpers                                                                        */
/* ------------------------------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void normalize3(double* a) {
  double s = sqrt(dot3(a, a));
  a[0] /= s;
  a[1] /= s;
  a[2] /= s;
}
static void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Branchless orthonormal basis around a unit vector n (Duff et al., JCGT 6(1), 2017). */
static void onb_duff(const double* n, double* t, double* b) {
  double s = copysign(1.0, n[2]);
  double a = -1.0 / (s + n[2]);
  double c = n[0] * n[1] * a;
  t[0] = 1.0 + s * n[0] * n[0] * a;
  t[1] = s * c;
  t[2] = -s * n[0];
  b[0] = c;
  b[1] = s + n[1] * n[1] * a;
  b[2] = -n[1];
}

/* ------------------------------------------------------------------------------------------ */
/* equirectangular environment maps (the paper uses a cubemap, Sec. 3.1)                      */
/*   u = 0.5 + atan2(d.x, -d.z) / (2 pi),  v = atan2(sqrt(d.x^2 + d.z^2), d.y) / pi           */
/* ------------------------------------------------------------------------------------------ */
static void dir_to_uv(const double* d, double* u, double* v) {
  *u = 0.5 + atan2(d[0], -d[2]) / (2.0 * OR_PI);
  *v = atan2(sqrt(d[0] * d[0] + d[2] * d[2]), d[1]) / OR_PI;
}
static void uv_to_dir(double u, double v, double* d) {
  double phi = 2.0 * OR_PI * (u - 0.5), th = OR_PI * v;
  d[0] = sin(th) * sin(phi);
  d[1] = cos(th);
  d[2] = -sin(th) * cos(phi);
}
/* Bilinear read of an RGBA (4 doubles per texel) equirect map: wrap in u, clamp in v. */
static void equirect_bilinear(const double* map, int W, int H, double u, double v, double* out) {
  double x = u * W - 0.5, y = v * H - 0.5;
  double x0 = floor(x), y0 = floor(y);
  double fx = x - x0, fy = y - y0;
  long ix0 = (long)x0, iy0 = (long)y0;
  long i0 = ((ix0 % W) + W) % W, i1 = (((ix0 + 1) % W) + W) % W;
  long j0 = iy0 < 0 ? 0 : (iy0 > H - 1 ? H - 1 : iy0);
  long j1 = iy0 + 1 < 0 ? 0 : (iy0 + 1 > H - 1 ? H - 1 : iy0 + 1);
  for (int c = 0; c < 3; ++c) {
    double a = map[(j0 * W + i0) * 4 + c], b = map[(j0 * W + i1) * 4 + c];
    double p = map[(j1 * W + i0) * 4 + c], q = map[(j1 * W + i1) * 4 + c];
    out[c] = (1.0 - fy) * ((1.0 - fx) * a + fx * b) + fy * ((1.0 - fx) * p + fx * q);
  }
}
static void equirect_lookup(const double* map, int W, int H, const double* d, double* out) {
  double u, v;
  dir_to_uv(d, &u, &v);
  equirect_bilinear(map, W, H, u, v, out);
}

/* ------------------------------------------------------------------------------------------ */
/* Hammersley set and GGX importance sampling (Karis 2013)                                     */
/* ------------------------------------------------------------------------------------------ */
/* Van der Corput radical inverse in base 2: the bits of i mirrored about the binary point. */
static double radical_inverse2(uint32_t i) {
  double r = 0.0, f = 0.5;
  while (i) {
    if (i & 1u) r += f;
    f *= 0.5;
    i >>= 1;
  }
  return r;
}
/* Tangent frame of the sampling around unit n, built from the environment's pole axis y as
 * Karis 2013's reference code builds it from its up vector: t = normalize(y x n), b = n x t.  It
 * turns with n about the pole axis (rotating n about y rotates t and b alike).  For n on the
 * axis itself (y x n = 0; no texel centre of an equirect map lies there) the Duff et al. basis
 * is used. */
static void onb_pole(const double* n, double* t, double* b) {
  double len2 = n[2] * n[2] + n[0] * n[0];
  if (!(len2 > 0.0)) {
    onb_duff(n, t, b);
    return;
  }
  double inv = 1.0 / sqrt(len2);
  t[0] = n[2] * inv; /* y x n = (n.z, 0, -n.x) */
  t[1] = 0.0;
  t[2] = -n[0] * inv;
  cross3(n, t, b);
}

/* Half vector for Hammersley point (xi1, xi2) = (k/N, radical_inverse(k)) around n:
 * phi = 2 pi xi1, cos(theta) = sqrt((1 - xi2) / (1 + (alpha^2 - 1) xi2)), i.e. the inverse CDF
 * of the GGX distribution of normals D(h)(n.h), in the frame of onb_pole. */
static void ggx_half_vector(double xi1, double xi2, double alpha, const double* n, double* h) {
  double a2 = alpha * alpha;
  double phi = 2.0 * OR_PI * xi1;
  double ct = sqrt((1.0 - xi2) / (1.0 + (a2 - 1.0) * xi2));
  double st = sqrt(1.0 - ct * ct);
  double hx = st * cos(phi), hy = st * sin(phi), hz = ct;
  double t[3], b[3];
  onb_pole(n, t, b);
  for (int c = 0; c < 3; ++c) h[c] = t[c] * hx + b[c] * hy + n[c] * hz;
}

/* ------------------------------------------------------------------------------------------ */
/* Cook-Torrance BRDF of UE4 (paper Sec. 3; Karis 2013)                                        */
/* ------------------------------------------------------------------------------------------ */
static double ggx_D(double nh, double alpha) {
  double a2 = alpha * alpha;
  double den = nh * nh * (a2 - 1.0) + 1.0;
  return a2 / (OR_PI * den * den);
}
static double smith_schlick_G1(double x, double k) { return x / (x * (1.0 - k) + k); }

#define OR_ROUGH_MIN 0.045
#define OR_NV_MIN 1e-4

/* f_r(l, v) in RGB for unit n, l, v and a metalness/roughness material:
 *   f = (1 - F) c_diff / pi + D G F / (4 (n.l)(n.v)),
 * D = GGX with alpha = r^2, G = G1(n.l) G1(n.v) with k = (r + 1)^2 / 8,
 * F = F0 + (1 - F0)(1 - v.h)^5, F0 = mix(0.04, albedo, metal), c_diff = albedo (1 - metal).
 * n.l and n.v must be positive. */
void or_brdf(const double* n, const double* l, const double* v, const double* albedo,
             double metal, double rough, double* out) {
  double h[3] = {l[0] + v[0], l[1] + v[1], l[2] + v[2]};
  normalize3(h);
  double nl = dot3(n, l), nv = dot3(n, v), nh = dot3(n, h), vh = dot3(v, h);
  double alpha = rough * rough;
  double k = (rough + 1.0) * (rough + 1.0) / 8.0;
  double D = ggx_D(nh, alpha);
  double G = smith_schlick_G1(nl, k) * smith_schlick_G1(nv, k);
  double fc = pow(1.0 - vh, 5.0);
  for (int c = 0; c < 3; ++c) {
    double F0 = 0.04 * (1.0 - metal) + albedo[c] * metal;
    double F = F0 + (1.0 - F0) * fc;
    double cdiff = albedo[c] * (1.0 - metal);
    out[c] = (1.0 - F) * cdiff / OR_PI + D * G * F / (4.0 * nl * nv);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* A1: BRDF integration table (split sum, second factor)                                       */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int S, N;
  double* out;
} lut_ctx;

static void lut_body(void* p, long i0, long i1) {
  lut_ctx* c = (lut_ctx*)p;
  const double n[3] = {0.0, 0.0, 1.0};
  for (long t = i0; t < i1; ++t) {
    int i = (int)(t % c->S), j = (int)(t / c->S);
    double mu = (i + 0.5) / c->S, r = (j + 0.5) / c->S;
    double alpha = r * r, k = alpha / 2.0;
    double v[3] = {sqrt(1.0 - mu * mu), 0.0, mu};
    double A = 0.0, B = 0.0;
    for (int s = 0; s < c->N; ++s) {
      double h[3], l[3];
      ggx_half_vector((double)s / c->N, radical_inverse2((uint32_t)s), alpha, n, h);
      double vh = dot3(v, h);
      for (int q = 0; q < 3; ++q) l[q] = 2.0 * vh * h[q] - v[q];
      double nl = l[2], nh = h[2], nv = mu;
      if (nl > 0.0) {
        double G = smith_schlick_G1(nl, k) * smith_schlick_G1(nv, k);
        double Gvis = G * vh / (nh * nv);
        double Fc = pow(1.0 - vh, 5.0);
        A += (1.0 - Fc) * Gvis;
        B += Fc * Gvis;
      }
    }
    c->out[t * 2 + 0] = A / c->N;
    c->out[t * 2 + 1] = B / c->N;
  }
}

/* out: S*S*2 doubles, row j = roughness, column i = n.v. */
int or_brdf_lut(int S, int N, double* out, int threads) {
  if (S < 1 || N < 1 || !out) return 1;
  lut_ctx c = {S, N, out};
  or_parallel_for((long)S * S, threads, lut_body, &c);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* A2: diffuse irradiance by exact quadrature over every source texel                          */
/*   out(n) = sum_t L_t max(n.d_t, 0) Omega_t / sum_t max(n.d_t, 0) Omega_t                   */
/*   Omega of row y = (2 pi / W)(cos(pi y / H) - cos(pi (y + 1) / H))                          */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  const double* env;
  int We, He, Wi, Hi;
  const int* texels;
  double* out;
} irr_ctx;

static void irr_body(void* p, long i0, long i1) {
  irr_ctx* c = (irr_ctx*)p;
  for (long t = i0; t < i1; ++t) {
    long idx = c->texels ? c->texels[t] : t;
    int i = (int)(idx % c->Wi), j = (int)(idx / c->Wi);
    double n[3];
    uv_to_dir((i + 0.5) / c->Wi, (j + 0.5) / c->Hi, n);
    double num[3] = {0, 0, 0}, den = 0.0;
    for (int y = 0; y < c->He; ++y) {
      double omega = (2.0 * OR_PI / c->We) * (cos(OR_PI * y / c->He) - cos(OR_PI * (y + 1) / c->He));
      for (int x = 0; x < c->We; ++x) {
        double d[3];
        uv_to_dir((x + 0.5) / c->We, (y + 0.5) / c->He, d);
        double w = dot3(n, d);
        if (w <= 0.0) continue;
        w *= omega;
        const double* L = c->env + ((long)y * c->We + x) * 4;
        num[0] += L[0] * w;
        num[1] += L[1] * w;
        num[2] += L[2] * w;
        den += w;
      }
    }
    /* A direction whose hemisphere holds no texel centre (maps of one or two columns) makes
     * the ratio 0/0; it is defined as 0 (no light arrives).  A reading: Sec. 3.1 is silent. */
    for (int q = 0; q < 3; ++q) c->out[t * 3 + q] = den > 0.0 ? num[q] / den : 0.0;
  }
}

/* env: He*We*4 doubles.  texels: indices j*Wi+i to evaluate (NULL = all, in order).
 * out: n*3 doubles. */
int or_irradiance(const double* env, int We, int He, int Wi, int Hi, const int* texels,
                  long n, double* out, int threads) {
  if (!env || !out || We < 1 || He < 1 || Wi < 1 || Hi < 1) return 1;
  irr_ctx c = {env, We, He, Wi, Hi, texels, out};
  long cnt = texels ? n : (long)Wi * Hi;
  or_parallel_for(cnt, threads, irr_body, &c);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* A3: GGX-prefiltered environment level m >= 1 (split sum, first factor), n = v = R           */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  const double* env;
  int We, He, M, N, level, Wl, Hl;
  const int* texels;
  double* out;
} pre_ctx;

static void pre_body(void* p, long i0, long i1) {
  pre_ctx* c = (pre_ctx*)p;
  double r = (c->M > 1) ? (double)c->level / (c->M - 1) : 0.0;
  double alpha = r * r;
  for (long t = i0; t < i1; ++t) {
    long idx = c->texels ? c->texels[t] : t;
    int i = (int)(idx % c->Wl), j = (int)(idx / c->Wl);
    double n[3];
    uv_to_dir((i + 0.5) / c->Wl, (j + 0.5) / c->Hl, n);
    const double* v = n;
    double sum[3] = {0, 0, 0}, wsum = 0.0;
    for (int s = 0; s < c->N; ++s) {
      double h[3], l[3], L[3];
      ggx_half_vector((double)s / c->N, radical_inverse2((uint32_t)s), alpha, n, h);
      double vh = dot3(v, h);
      for (int q = 0; q < 3; ++q) l[q] = 2.0 * vh * h[q] - v[q];
      double nl = dot3(n, l);
      if (nl > 0.0) {
        equirect_lookup(c->env, c->We, c->He, l, L);
        for (int q = 0; q < 3; ++q) sum[q] += L[q] * nl;
        wsum += nl;
      }
    }
    for (int q = 0; q < 3; ++q) c->out[t * 3 + q] = sum[q] / wsum;
  }
}

static int level_dim(int d, int m) {
  int r = d >> m;
  return r < 1 ? 1 : r;
}

/* Texels of level `level` (1 <= level < M) of the chain over env (He*We*4 doubles). */
int or_prefilter(const double* env, int We, int He, int M, int N, int level, const int* texels,
                 long n, double* out, int threads) {
  if (!env || !out || M < 2 || level < 1 || level >= M || N < 1) return 1;
  pre_ctx c = {env, We, He, M, N, level, level_dim(We, level), level_dim(He, level), texels, out};
  long cnt = texels ? n : (long)c.Wl * c.Hl;
  or_parallel_for(cnt, threads, pre_body, &c);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* A4: G-buffer decode                                                                          */
/* Decoded layout, 9 doubles per pixel: albedo rgb (linear), metal, normal xyz, rough, depth.   */
/* ------------------------------------------------------------------------------------------ */
/* IEEE binary16 bits -> value, from the format's definition. */
static double half_to_double(uint16_t h) {
  int s = (h >> 15) & 1, e = (h >> 10) & 31, f = h & 1023;
  double v;
  if (e == 0)
    v = ldexp((double)f, -24);
  else if (e == 31)
    v = f ? NAN : INFINITY;
  else
    v = ldexp(1024.0 + f, e - 25);
  return s ? -v : v;
}
/* sRGB electro-optical transfer (IEC 61966-2-1) for code c / 255. */
static double srgb_decode(double x) {
  return x <= 0.04045 ? x / 12.92 : pow((x + 0.055) / 1.055, 2.4);
}

/* Compact form of Table 1: rt0 RGBA8 sRGB albedo + weight, rt1 2 x FP16 octahedral normal
 * (Cigolle et al. 2014), rt2 2 x UNORM8 (metal, rough), rt3 FP32 depth. */
int or_decode_compact(const uint8_t* rt0, const uint16_t* rt1, const uint8_t* rt2,
                      const float* depth, long npx, double* gb) {
  for (long p = 0; p < npx; ++p) {
    double* o = gb + p * 9;
    for (int c = 0; c < 3; ++c) o[c] = srgb_decode(rt0[p * 4 + c] / 255.0);
    o[3] = rt2[p * 2 + 0] / 255.0;
    double x = half_to_double(rt1[p * 2 + 0]), y = half_to_double(rt1[p * 2 + 1]);
    double z = 1.0 - fabs(x) - fabs(y);
    if (z < 0.0) {
      double nx = (1.0 - fabs(y)) * (x >= 0.0 ? 1.0 : -1.0);
      double ny = (1.0 - fabs(x)) * (y >= 0.0 ? 1.0 : -1.0);
      x = nx;
      y = ny;
    }
    o[4] = x;
    o[5] = y;
    o[6] = z;
    o[7] = rt2[p * 2 + 1] / 255.0;
    o[8] = depth[p];
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* camera: pixel rays and position from depth (Sec. 4: position is not stored)                  */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  double v2w[16]; /* column-major */
  double fov_y;
  int W, H;
} or_camera;

static void view_ray(const or_camera* cam, double x, double y, double* r) {
  double t = tan(0.5 * cam->fov_y), aspect = (double)cam->W / cam->H;
  r[0] = (2.0 * x / cam->W - 1.0) * t * aspect;
  r[1] = (1.0 - 2.0 * y / cam->H) * t;
  r[2] = -1.0;
}
static void rot_apply(const or_camera* cam, const double* a, double* b) {
  for (int i = 0; i < 3; ++i) b[i] = cam->v2w[i] * a[0] + cam->v2w[4 + i] * a[1] + cam->v2w[8 + i] * a[2];
}
static void rot_apply_t(const or_camera* cam, const double* a, double* b) {
  for (int i = 0; i < 3; ++i)
    b[i] = cam->v2w[4 * i + 0] * a[0] + cam->v2w[4 * i + 1] * a[1] + cam->v2w[4 * i + 2] * a[2];
}
static int is_surface(double e) { return e > 0.0 && e < INFINITY; }

/* ------------------------------------------------------------------------------------------ */
/* A5 / A6: SSAO (Sec. 5.2)                                                                     */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int K, scale, blur_radius;
  double radius, bias, sigma_s, sigma_z;
  const double* kernel; /* K*3 */
  const double* noise;  /* 16*2 */
} or_ssao_params;

static double smoothstep01(double x) {
  x = clampd(x, 0.0, 1.0);
  return x * x * (3.0 - 2.0 * x);
}

/* Occlusion of one sample against depth pixel (ix, iy), or -1 when nothing is there. */
static double occ_at(const double* gb, const or_camera* cam, const or_ssao_params* sp, long ix,
                     long iy, double eP, double eS) {
  if (ix < 0 || iy < 0 || ix >= cam->W || iy >= cam->H) return 0.0;
  double eb = gb[(iy * cam->W + ix) * 9 + 8];
  if (!is_surface(eb)) return 0.0;
  if (!(eb <= eS - sp->bias)) return 0.0;
  return smoothstep01(sp->radius / fabs(eP - eb));
}

#define OR_TIE_PX 2e-3
#define OR_TIE_DEPTH 1e-5

/* Raw AO of AO texel (i, j); lo/hi bound the value over every outcome of a pixel-boundary or
 * depth-comparison decision that lies within rounding distance of its threshold. */
static void ssao_raw_texel(const double* gb, const or_camera* cam, const or_ssao_params* sp,
                           int i, int j, double* ao, double* lo, double* hi) {
  long X0 = (long)sp->scale * i, Y0 = (long)sp->scale * j;
  const double* g = gb + (Y0 * cam->W + X0) * 9;
  double eP = g[8];
  if (!is_surface(eP)) {
    *ao = *lo = *hi = 1.0;
    return;
  }
  double r[3], P[3], nw[3] = {g[4], g[5], g[6]}, n[3];
  view_ray(cam, X0 + 0.5, Y0 + 0.5, r);
  for (int q = 0; q < 3; ++q) P[q] = eP * r[q];
  normalize3(nw);
  rot_apply_t(cam, nw, n);
  /* Tangent frame: the tiled noise vector made orthogonal to n (Gram-Schmidt). */
  const double* nz = sp->noise + ((j % 4) * 4 + (i % 4)) * 2;
  double rv[3] = {nz[0], nz[1], 0.0}, t[3], b[3];
  double rn = dot3(rv, n);
  for (int q = 0; q < 3; ++q) t[q] = rv[q] - n[q] * rn;
  double tl = sqrt(dot3(t, t));
  int frame_tie = fabs(tl - 1e-4) < 1e-6;
  if (tl < 1e-4) {
    onb_duff(n, t, b);
  } else {
    for (int q = 0; q < 3; ++q) t[q] /= tl;
    cross3(n, t, b);
  }
  double tA = tan(0.5 * cam->fov_y), aspect = (double)cam->W / cam->H;
  double sum = 0.0, sum_lo = 0.0, sum_hi = 0.0;
  for (int k = 0; k < sp->K; ++k) {
    const double* ks = sp->kernel + k * 3;
    double S[3];
    for (int q = 0; q < 3; ++q) S[q] = P[q] + sp->radius * (t[q] * ks[0] + b[q] * ks[1] + n[q] * ks[2]);
    double eS = -S[2];
    double occ = 0.0, olo, ohi;
    if (eS <= 0.0) {
      olo = ohi = 0.0;
      if (eS > -OR_TIE_DEPTH) olo = 0.0, ohi = 1.0;
    } else {
      double x = ((S[0] / eS) / (tA * aspect) + 1.0) * 0.5 * cam->W;
      double y = (1.0 - (S[1] / eS) / tA) * 0.5 * cam->H;
      long ix = (long)floor(x), iy = (long)floor(y);
      occ = occ_at(gb, cam, sp, ix, iy, eP, eS);
      olo = ohi = occ;
      /* candidate pixels: the nominal one, plus the neighbour across a boundary in reach */
      long cx[2] = {ix, ix}, cy[2] = {iy, iy};
      double fx = x - floor(x), fy = y - floor(y);
      if (fx < OR_TIE_PX) cx[1] = ix - 1;
      if (fx > 1.0 - OR_TIE_PX) cx[1] = ix + 1;
      if (fy < OR_TIE_PX) cy[1] = iy - 1;
      if (fy > 1.0 - OR_TIE_PX) cy[1] = iy + 1;
      for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) {
          long px = cx[a], py = cy[c];
          double o = occ_at(gb, cam, sp, px, py, eP, eS);
          if (o < olo) olo = o;
          if (o > ohi) ohi = o;
          if (px >= 0 && py >= 0 && px < cam->W && py < cam->H) {
            double eb = gb[(py * cam->W + px) * 9 + 8];
            if (is_surface(eb) && fabs(eb - (eS - sp->bias)) <= OR_TIE_DEPTH * (eS > 1.0 ? eS : 1.0)) {
              double full = smoothstep01(sp->radius / fabs(eP - eb));
              if (0.0 < olo) olo = 0.0;
              if (full > ohi) ohi = full;
            }
          }
        }
    }
    sum += occ;
    sum_lo += olo;
    sum_hi += ohi;
  }
  *ao = 1.0 - sum / sp->K;
  *lo = 1.0 - sum_hi / sp->K;
  *hi = 1.0 - sum_lo / sp->K;
  if (frame_tie) {
    *lo = 0.0;
    *hi = 1.0;
  }
}

typedef struct {
  const double* gb;
  const or_camera* cam;
  const or_ssao_params* sp;
  int mode, Wa, Ha;
  const int* texels;
  double *ao, *lo, *hi;
} ssao_ctx;

/* Bilateral blur weight of AO texel q seen from texel p (Sec. 5.2): a Gaussian of the texel
 * offset (sigma_s in AO texels) times a range term that falls with the relative depth step,
 * exp(-|e_q - e_p| / (sigma_z e_p)). */
static double blur_weight(const or_ssao_params* sp, int dx, int dy, double ep, double eq) {
  return exp(-(dx * dx + dy * dy) / (2.0 * sp->sigma_s * sp->sigma_s)) * exp(-fabs(eq - ep) / (sp->sigma_z * ep));
}

/* Blurred AO of texel (i, j).  raw == NULL: the raw AO of each tap (and its tie bounds) comes
 * from ssao_raw_texel; otherwise from the given Ha*Wa raw AO image (no ties).  Background taps
 * (no surface at the tap's pixel) carry no weight; a background texel is 1. */
static void ssao_blur_texel(const double* gb, const or_camera* cam, const or_ssao_params* sp, int Wa, int Ha,
                            const double* raw, int i, int j, double* ao, double* lo, double* hi) {
  double ep = gb[(((long)sp->scale * j) * cam->W + (long)sp->scale * i) * 9 + 8];
  if (!is_surface(ep)) {
    *ao = *lo = *hi = 1.0;
    return;
  }
  double num = 0.0, nlo = 0.0, nhi = 0.0, den = 0.0;
  for (int dy = -sp->blur_radius; dy <= sp->blur_radius; ++dy)
    for (int dx = -sp->blur_radius; dx <= sp->blur_radius; ++dx) {
      int qi = i + dx, qj = j + dy;
      if (qi < 0 || qj < 0 || qi >= Wa || qj >= Ha) continue;
      double eq = gb[(((long)sp->scale * qj) * cam->W + (long)sp->scale * qi) * 9 + 8];
      if (!is_surface(eq)) continue;
      double w = blur_weight(sp, dx, dy, ep, eq);
      double a, l, h;
      if (raw) {
        a = l = h = raw[(long)qj * Wa + qi];
      } else {
        ssao_raw_texel(gb, cam, sp, qi, qj, &a, &l, &h);
      }
      num += w * a;
      nlo += w * l;
      nhi += w * h;
      den += w;
    }
  *ao = num / den;
  *lo = nlo / den;
  *hi = nhi / den;
}

static void ssao_body(void* p, long i0, long i1) {
  ssao_ctx* c = (ssao_ctx*)p;
  const or_ssao_params* sp = c->sp;
  for (long t = i0; t < i1; ++t) {
    long idx = c->texels ? c->texels[t] : t;
    int i = (int)(idx % c->Wa), j = (int)(idx / c->Wa);
    if (c->mode == 0 || sp->blur_radius == 0) {
      ssao_raw_texel(c->gb, c->cam, sp, i, j, &c->ao[t], &c->lo[t], &c->hi[t]);
      continue;
    }
    ssao_blur_texel(c->gb, c->cam, sp, c->Wa, c->Ha, NULL, i, j, &c->ao[t], &c->lo[t], &c->hi[t]);
  }
}

/* mode 0: raw AO, mode 1: blurred AO.  texels: indices j*Wa+i of the AO image (NULL = all).
 * ao/lo/hi: n doubles each. */
int or_ssao(const double* gb, const or_camera* cam, const or_ssao_params* sp, int mode,
            const int* texels, long n, double* ao, double* lo, double* hi, int threads) {
  if (!gb || !cam || !sp || sp->K < 1 || (sp->scale != 1 && sp->scale != 2)) return 1;
  int Wa = (cam->W + sp->scale - 1) / sp->scale, Ha = (cam->H + sp->scale - 1) / sp->scale;
  ssao_ctx c = {gb, cam, sp, mode, Wa, Ha, texels, ao, lo, hi};
  long cnt = texels ? n : (long)Wa * Ha;
  or_parallel_for(cnt, threads, ssao_body, &c);
  return 0;
}

/* The bilateral blur alone, applied to a given raw AO image (Ha*Wa doubles, the AO layout of
 * or_ssao) with the depths of the G-buffer: the same blur as or_ssao mode 1.  out: Ha*Wa. */
int or_ssao_blur_image(const double* gb, const or_camera* cam, const or_ssao_params* sp, const double* raw,
                       double* out) {
  if (!gb || !cam || !sp || !raw || !out || (sp->scale != 1 && sp->scale != 2) || sp->blur_radius < 0) return 1;
  int Wa = (cam->W + sp->scale - 1) / sp->scale, Ha = (cam->H + sp->scale - 1) / sp->scale;
  for (int j = 0; j < Ha; ++j)
    for (int i = 0; i < Wa; ++i) {
      double lo, hi;
      ssao_blur_texel(gb, cam, sp, Wa, Ha, raw, i, j, &out[(long)j * Wa + i], &lo, &hi);
    }
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* A7-A10: compose (direct lights + split-sum IBL + background)                                 */
/* ------------------------------------------------------------------------------------------ */
#define OR_MAX_LEVELS 16
typedef struct {
  const double* irr; /* Hi*Wi*4 */
  int Wi, Hi;
  int M;
  const double* level[OR_MAX_LEVELS]; /* each Hl*Wl*4 */
  int Wl[OR_MAX_LEVELS], Hl[OR_MAX_LEVELS];
  const double* lut; /* S*S*2 */
  int S;
} or_ibl;

enum { OR_DIRECT = 1, OR_IBL = 2, OR_MULTI = 4, OR_DIFFUSE_ONLY = 8 };

static void lut_bilinear(const or_ibl* ib, double mu, double r, double* A, double* B) {
  int S = ib->S;
  double x = mu * S - 0.5, y = r * S - 0.5;
  double x0 = floor(x), y0 = floor(y), fx = x - x0, fy = y - y0;
  long i0 = (long)clampd(x0, 0, S - 1), i1 = (long)clampd(x0 + 1, 0, S - 1);
  long j0 = (long)clampd(y0, 0, S - 1), j1 = (long)clampd(y0 + 1, 0, S - 1);
  for (int c = 0; c < 2; ++c) {
    double a = ib->lut[(j0 * S + i0) * 2 + c], b = ib->lut[(j0 * S + i1) * 2 + c];
    double p = ib->lut[(j1 * S + i0) * 2 + c], q = ib->lut[(j1 * S + i1) * 2 + c];
    double v = (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * p + fx * q);
    if (c == 0) *A = v; else *B = v;
  }
}

typedef struct {
  const double* gb;
  const or_camera* cam;
  const double* lights; /* N*7: pos xyz, intensity, color rgb */
  int NL;
  const or_ibl* ibl;
  const double* ao;
  int Wa, Ha, ao_scale;
  int flags;
  const long* pixels;
  double* out;
  const struct or_shadows_s* sh; /* NULL: unshadowed */
  double *out_lo, *out_hi;       /* with sh: bounds over tied shadow decisions (NULL allowed) */
} shade_ctx;

/* ------------------------------------------------------------------------------------------ */
/* Shadow maps with 3x3 percentage-closer filtering (Sec. 5.1; Williams 1978, Reeves 1987)     */
/* ------------------------------------------------------------------------------------------ */
/* Readings: each light renders one perspective depth map "as if it were a normal camera": cams
 * holds per light the world->light-view matrix (3 rows of 4; the light camera looks along -z)
 * and f = 1/tan(fov/2), square maps of S x S eye depths (+inf = nothing).  A fragment at light
 * depth z = -q.z > 0 projects to texel coordinates s = (q.x f / z + 1) S/2, t = (1 - q.y f / z) S/2
 * (row 0 at the top, as the main camera) and texel (floor s, floor t).  A tap lights it when
 * z <= d + b0 + b1 z; taps outside the map and fragments behind the light (z <= 0) are lit.
 * Visibility = lit taps of the 3x3 block around the texel / 9; it multiplies the light's whole
 * direct term.  Ties: a tap whose d is within OR_TIE_DEPTH * max(z, 1) of the threshold may go
 * either way, and so may the block when s or t lies within OR_TIE_PX of a texel edge; vis_lo /
 * vis_hi bound the visibility over those choices. */
typedef struct or_shadows_s {
  const double* maps; /* NL*S*S */
  const double* cams; /* NL*16: rows 0..2 of the world->view matrix (12), f, 3 unused */
  int S;
  double b0, b1;
} or_shadows;

static int shadow_block_lit(const or_shadows* sh, const double* map, int bi, int bj, double z, int mode) {
  /* mode 0: exact decisions; -1: ties count as shadowed; +1: ties count as lit */
  double thr = z - sh->b0 - sh->b1 * z, tie = OR_TIE_DEPTH * (z > 1.0 ? z : 1.0);
  int lit = 0;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      long i = bi + dx, j = bj + dy;
      if (i < 0 || j < 0 || i >= sh->S || j >= sh->S) {
        ++lit;
        continue;
      }
      double d = map[j * sh->S + i];
      if (mode == 0) lit += d >= thr;
      else if (mode < 0) lit += d >= thr + tie;
      else lit += d >= thr - tie;
    }
  return lit;
}

static void shadow_vis(const or_shadows* sh, int light, const double* P, double* vis, double* vlo, double* vhi) {
  const double* V = sh->cams + 16 * (long)light;
  double q[3];
  for (int r = 0; r < 3; ++r) q[r] = V[4 * r] * P[0] + V[4 * r + 1] * P[1] + V[4 * r + 2] * P[2] + V[4 * r + 3];
  double z = -q[2];
  if (!(z > 0.0)) {
    *vis = *vlo = *vhi = 1.0;
    return;
  }
  double f = V[12], S = sh->S;
  double sx = (q[0] * f / z + 1.0) * 0.5 * S, sy = (1.0 - q[1] * f / z) * 0.5 * S;
  if (!(fabs(sx) < 1e9 && fabs(sy) < 1e9)) { /* far outside the frustum */
    *vis = *vlo = *vhi = 1.0;
    return;
  }
  double fx = floor(sx), fy = floor(sy);
  const double* map = sh->maps + (long)light * sh->S * sh->S;
  *vis = shadow_block_lit(sh, map, (int)fx, (int)fy, z, 0) / 9.0;
  int cx[2] = {(int)fx, (int)fx}, cy[2] = {(int)fy, (int)fy};
  if (sx - fx < OR_TIE_PX) cx[1] = (int)fx - 1;
  if (sx - fx > 1.0 - OR_TIE_PX) cx[1] = (int)fx + 1;
  if (sy - fy < OR_TIE_PX) cy[1] = (int)fy - 1;
  if (sy - fy > 1.0 - OR_TIE_PX) cy[1] = (int)fy + 1;
  int lo = 9, hi = 0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      int l = shadow_block_lit(sh, map, cx[a], cy[b], z, -1), h = shadow_block_lit(sh, map, cx[a], cy[b], z, 1);
      lo = l < lo ? l : lo;
      hi = h > hi ? h : hi;
    }
  *vlo = lo / 9.0;
  *vhi = hi / 9.0;
}

static void shade_pixel(const shade_ctx* c, long pix, double* out, double* lo, double* hi) {
  const or_camera* cam = c->cam;
  int x = (int)(pix % cam->W), y = (int)(pix / cam->W);
  const double* g = c->gb + pix * 9;
  double r[3], dw[3], eye[3] = {cam->v2w[12], cam->v2w[13], cam->v2w[14]};
  view_ray(cam, x + 0.5, y + 0.5, r);
  rot_apply(cam, r, dw);
  double e = g[8];
  out[0] = out[1] = out[2] = 0.0;
  lo[0] = lo[1] = lo[2] = hi[0] = hi[1] = hi[2] = 0.0;
  if (!is_surface(e)) {
    /* A9: background shows the environment along the view ray. */
    if ((c->flags & OR_IBL) && c->ibl) equirect_lookup(c->ibl->level[0], c->ibl->Wl[0], c->ibl->Hl[0], dw, out);
    for (int q = 0; q < 3; ++q) lo[q] = hi[q] = out[q];
    return;
  }
  double P[3], v[3], n[3] = {g[4], g[5], g[6]};
  for (int q = 0; q < 3; ++q) P[q] = eye[q] + e * dw[q];
  for (int q = 0; q < 3; ++q) v[q] = eye[q] - P[q];
  normalize3(v);
  normalize3(n);
  double albedo[3] = {g[0], g[1], g[2]};
  double metal = clampd(g[3], 0.0, 1.0), rough = clampd(g[7], OR_ROUGH_MIN, 1.0);
  double nv_raw = dot3(n, v), nv = nv_raw > OR_NV_MIN ? nv_raw : OR_NV_MIN;
  int diffuse_only = (c->flags & OR_DIFFUSE_ONLY) != 0;
  double F0[3], cdiff[3];
  for (int q = 0; q < 3; ++q) {
    F0[q] = 0.04 * (1.0 - metal) + albedo[q] * metal;
    cdiff[q] = albedo[q] * (1.0 - metal);
  }
  /* A7: direct lighting, Eq. 1 restricted to point lights. */
  if (c->flags & OR_DIRECT) {
    double alpha = rough * rough, k = (rough + 1.0) * (rough + 1.0) / 8.0;
    for (int i = 0; i < c->NL; ++i) {
      const double* Lt = c->lights + i * 7;
      double lv[3] = {Lt[0] - P[0], Lt[1] - P[1], Lt[2] - P[2]};
      double d2 = dot3(lv, lv);
      double l[3] = {lv[0], lv[1], lv[2]};
      normalize3(l);
      double nl = dot3(n, l);
      if (!(nl > 0.0)) continue;
      double rad[3] = {Lt[3] * Lt[4] / d2, Lt[3] * Lt[5] / d2, Lt[3] * Lt[6] / d2};
      double vis = 1.0, vlo = 1.0, vhi = 1.0;
      if (c->sh) shadow_vis(c->sh, i, P, &vis, &vlo, &vhi);
      if (diffuse_only) {
        for (int q = 0; q < 3; ++q) {
          double t = albedo[q] / OR_PI * rad[q] * nl;
          out[q] += vis * t;
          lo[q] += vlo * t;
          hi[q] += vhi * t;
        }
        continue;
      }
      double h[3] = {l[0] + v[0], l[1] + v[1], l[2] + v[2]};
      normalize3(h);
      double nh = dot3(n, h), vh = dot3(v, h);
      double D = ggx_D(nh, alpha);
      double G = smith_schlick_G1(nl, k) * smith_schlick_G1(nv, k);
      double fc = pow(1.0 - vh, 5.0);
      for (int q = 0; q < 3; ++q) {
        double F = F0[q] + (1.0 - F0[q]) * fc;
        double spec = D * G * F / (4.0 * nl * nv);
        double diff = (1.0 - F) * cdiff[q] / OR_PI;
        double t = (diff + spec) * rad[q] * nl;
        out[q] += vis * t;
        lo[q] += vlo * t;
        hi[q] += vhi * t;
      }
    }
  }
  /* A8: split-sum ambient term, optionally with multiple scattering. */
  if ((c->flags & OR_IBL) && c->ibl) {
    const or_ibl* ib = c->ibl;
    double aoval = 1.0;
    if (c->ao) {
      long ai = x / c->ao_scale, aj = y / c->ao_scale;
      aoval = c->ao[aj * c->Wa + ai];
    }
    double irr[3];
    equirect_lookup(ib->irr, ib->Wi, ib->Hi, n, irr);
    if (diffuse_only) {
      for (int q = 0; q < 3; ++q) {
        out[q] += albedo[q] * irr[q] * aoval;
        lo[q] += albedo[q] * irr[q] * aoval;
        hi[q] += albedo[q] * irr[q] * aoval;
      }
      return;
    }
    double R[3];
    for (int q = 0; q < 3; ++q) R[q] = 2.0 * nv_raw * n[q] - v[q];
    double pref[3];
    double lod = rough * (ib->M - 1);
    int l0 = (int)floor(lod);
    if (l0 > ib->M - 1) l0 = ib->M - 1;
    int l1 = l0 + 1 < ib->M ? l0 + 1 : ib->M - 1;
    double tl = lod - l0, p0[3], p1[3];
    equirect_lookup(ib->level[l0], ib->Wl[l0], ib->Hl[l0], R, p0);
    equirect_lookup(ib->level[l1], ib->Wl[l1], ib->Hl[l1], R, p1);
    for (int q = 0; q < 3; ++q) pref[q] = (1.0 - tl) * p0[q] + tl * p1[q];
    double A, B;
    lut_bilinear(ib, clampd(nv, 0.0, 1.0), rough, &A, &B);
    double fcv = pow(1.0 - nv, 5.0);
    for (int q = 0; q < 3; ++q) {
      double Fr = (1.0 - rough > F0[q] ? 1.0 - rough : F0[q]) - F0[q];
      double kS = F0[q] + Fr * fcv;
      double La;
      if (c->flags & OR_MULTI) {
        /* Fdez-Aguera 2019: single-scatter energy plus a geometric series of bounces. */
        double FssEss = kS * A + B;
        double Ess = A + B, Ems = 1.0 - Ess;
        double Favg = F0[q] + (1.0 - F0[q]) / 21.0;
        double Fms = FssEss * Favg / (1.0 - Ems * Favg);
        double kD = cdiff[q] * (1.0 - FssEss - Fms * Ems);
        La = FssEss * pref[q] + (Fms * Ems + kD) * irr[q];
      } else {
        La = (1.0 - kS) * cdiff[q] * irr[q] + (kS * A + B) * pref[q];
      }
      out[q] += La * aoval;
      lo[q] += La * aoval;
      hi[q] += La * aoval;
    }
  }
}

static void shade_body(void* p, long i0, long i1) {
  shade_ctx* c = (shade_ctx*)p;
  for (long t = i0; t < i1; ++t) {
    long pix = c->pixels ? c->pixels[t] : t;
    double lo[3], hi[3];
    shade_pixel(c, pix, c->out + t * 3, lo, hi);
    if (c->out_lo)
      for (int q = 0; q < 3; ++q) c->out_lo[t * 3 + q] = lo[q];
    if (c->out_hi)
      for (int q = 0; q < 3; ++q) c->out_hi[t * 3 + q] = hi[q];
  }
}

/* gb: W*H*9 decoded G-buffer; lights: NL*7; ao: Ha*Wa doubles or NULL; pixels: flat indices
 * y*W+x (NULL = all).  out: n*3 doubles of linear HDR radiance. */
int or_shade(const double* gb, const or_camera* cam, const double* lights, int NL,
             const or_ibl* ibl, const double* ao, int ao_scale, int flags, const long* pixels,
             long n, double* out, int threads) {
  if (!gb || !cam || !out || (NL > 0 && !lights)) return 1;
  if ((flags & OR_IBL) && !ibl) return 1;
  int s = ao_scale > 0 ? ao_scale : 1;
  shade_ctx c = {gb, cam, lights, NL, ibl, ao, (cam->W + s - 1) / s, (cam->H + s - 1) / s, s,
                 flags, pixels, out, NULL, NULL, NULL};
  long cnt = pixels ? n : (long)cam->W * cam->H;
  or_parallel_for(cnt, threads, shade_body, &c);
  return 0;
}

/* or_shade with shadow maps (Sec. 5.1): each light's direct term times its PCF visibility;
 * out_lo / out_hi (NULL allowed) receive the radiance with every tied shadow decision taken
 * the darker / the brighter way. */
int or_shade_shadows(const double* gb, const or_camera* cam, const double* lights, int NL,
                     const or_ibl* ibl, const double* ao, int ao_scale, int flags, const or_shadows* sh,
                     const long* pixels, long n, double* out, double* out_lo, double* out_hi, int threads) {
  if (!gb || !cam || !out || !sh || (NL > 0 && !lights) || sh->S < 1 || !sh->maps || !sh->cams) return 1;
  if ((flags & OR_IBL) && !ibl) return 1;
  int s = ao_scale > 0 ? ao_scale : 1;
  shade_ctx c = {gb, cam, lights, NL, ibl, ao, (cam->W + s - 1) / s, (cam->H + s - 1) / s, s,
                 flags, pixels, out, sh, out_lo, out_hi};
  long cnt = pixels ? n : (long)cam->W * cam->H;
  or_parallel_for(cnt, threads, shade_body, &c);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* A11: tone mapping and sRGB encoding (Sec. 5.4)                                               */
/* ------------------------------------------------------------------------------------------ */
static double aces_fit(double x) { return x * (2.51 * x + 0.03) / (x * (2.43 * x + 0.59) + 0.14); }
static double srgb_encode(double y) { return y <= 0.0031308 ? 12.92 * y : 1.055 * pow(y, 1.0 / 2.4) - 0.055; }

/* hdr: n*3 linear values; out: n*4 bytes (alpha 255); scaled: n*3 values 255*sRGB before
 * rounding (NULL allowed). */
int or_tonemap(const double* hdr, long n, double exposure, int op, uint8_t* out, double* scaled) {
  for (long p = 0; p < n; ++p) {
    for (int c = 0; c < 3; ++c) {
      /* Input clamp to [0, 1e6] (NaN -> 0): both operators saturate long before 1e6, and
       * the ACES ratio of +inf would be NaN.  A reading; Sec. 5.4 names only the operators. */
      double x = exposure * hdr[p * 3 + c];
      x = x > 0.0 ? x : 0.0;
      x = x < 1e6 ? x : 1e6;
      double y = (op == 1) ? x / (1.0 + x) : aces_fit(x);
      y = clampd(y, 0.0, 1.0);
      double s = 255.0 * srgb_encode(y);
      if (scaled) scaled[p * 3 + c] = s;
      out[p * 4 + c] = (uint8_t)floor(s + 0.5);
    }
    out[p * 4 + 3] = 255;
  }
  return 0;
}

/* Helpers exposed for tests: the equirect mapping and the sample set. */
void or_dir_to_uv(const double* d, double* uv) { dir_to_uv(d, &uv[0], &uv[1]); }
void or_uv_to_dir(double u, double v, double* d) { uv_to_dir(u, v, d); }
double or_radical_inverse2(uint32_t i) { return radical_inverse2(i); }
void or_ggx_half_vector(double xi1, double xi2, double alpha, const double* n, double* h) {
  ggx_half_vector(xi1, xi2, alpha, n, h);
}
void or_equirect_lookup(const double* map, int W, int H, const double* d, double* out) {
  equirect_lookup(map, W, H, d, out);
}

/* ------------------------------------------------------------------------------------------ */
/* Bloom (Sec. 5.3)                                                                            */
/* ------------------------------------------------------------------------------------------ */
/* Readings of the paper's description (it names the steps, not their constants):
 *   bright map   B(x) = X(x) where the luminance of X(x) exceeds the threshold, else 0; the
 *                luminance is the Rec. 709 weighting 0.2126 R + 0.7152 G + 0.0722 B.  The
 *                comparison decides a discrete outcome, so it is made in FP32 in one fixed
 *                order, ((0.2126 R + 0.7152 G) + 0.0722 B) with every product and sum rounded
 *                to FP32 (the CUDA path evaluates the same expression), on FP32 inputs;
 *   pyramid      level 0 = B at full resolution; level k = 2x2 box average of level k-1, size
 *                ceil(W_{k-1} / 2) x ceil(H_{k-1} / 2), the odd last row / column averaging its
 *                edge texel with itself (clamp to edge); L levels in total, 2 <= L <= 6;
 *   blur         levels 1 .. L-1 ("from the second one upwards"): separable Gaussian of radius
 *                R texels, weights exp(-d^2 / (2 sigma^2)) normalised to sum 1 over |d| <= R,
 *                clamp to edge, rows then columns;
 *   compositing  Y(x) = X(x) + s * sum_{k=1}^{L-1} U_k(x), U_k = level k after the blur sampled
 *                bilinearly (clamp to edge) at the centre of pixel x, which lies at texel
 *                coordinate (x + 1/2) / 2^k - 1/2 of level k.  Level 0 (the bright map itself)
 *                is not added: it is the pyramid's source, and adding it would brighten the
 *                bright pixels in place instead of spreading them. */
typedef struct {
  double threshold, strength, sigma;
  int radius, levels;
} or_bloom_params;

static int bright_f32(double r, double g, double b, double threshold) {
  float lr = 0.2126f * (float)r;
  float lg = 0.7152f * (float)g;
  float lb = 0.0722f * (float)b;
  float lum = (lr + lg) + lb;
  return lum > (float)threshold;
}

/* x: W*H*3 (FP32-representable values); y: W*H*3 output; levels_out (NULL allowed): levels
 * 1 .. L-1 before (pyr) and after (blurred) the blur, each level row-major RGB, concatenated in
 * level order, sum_k W_k H_k 3 doubles each.  Returns 0, or -1 on bad arguments. */
int or_bloom(const double* x, int W, int H, const or_bloom_params* bp, double* y, double* pyr, double* blurred) {
  if (W < 1 || H < 1 || bp->levels < 2 || bp->levels > 6 || bp->radius < 0 || bp->radius > 8 ||
      !(bp->sigma > 0.0))
    return -1;
  int L = bp->levels, R = bp->radius;
  double* lev[6] = {0};
  int Wl[6], Hl[6];
  Wl[0] = W;
  Hl[0] = H;
  lev[0] = (double*)malloc(sizeof(double) * 3 * (size_t)W * H);
  for (long p = 0; p < (long)W * H; ++p) {
    int on = bright_f32(x[3 * p], x[3 * p + 1], x[3 * p + 2], bp->threshold);
    for (int c = 0; c < 3; ++c) lev[0][3 * p + c] = on ? x[3 * p + c] : 0.0;
  }
  for (int k = 1; k < L; ++k) {
    Wl[k] = (Wl[k - 1] + 1) / 2;
    Hl[k] = (Hl[k - 1] + 1) / 2;
    lev[k] = (double*)malloc(sizeof(double) * 3 * (size_t)Wl[k] * Hl[k]);
    const double* src = lev[k - 1];
    int Ws = Wl[k - 1], Hs = Hl[k - 1];
    for (int j = 0; j < Hl[k]; ++j)
      for (int i = 0; i < Wl[k]; ++i)
        for (int c = 0; c < 3; ++c) {
          double sum = 0.0;
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
              int si = 2 * i + a < Ws ? 2 * i + a : Ws - 1;
              int sj = 2 * j + b < Hs ? 2 * j + b : Hs - 1;
              sum += src[3 * ((long)sj * Ws + si) + c];
            }
          lev[k][3 * ((long)j * Wl[k] + i) + c] = 0.25 * sum;
        }
  }
  /* Gaussian weights, normalised */
  double w[17], wsum = 0.0;
  for (int d = -R; d <= R; ++d) {
    w[d + R] = exp(-(double)(d * d) / (2.0 * bp->sigma * bp->sigma));
    wsum += w[d + R];
  }
  for (int d = 0; d <= 2 * R; ++d) w[d] /= wsum;
  long off = 0;
  for (int k = 1; k < L; ++k) {
    int Wk = Wl[k], Hk = Hl[k];
    if (pyr) memcpy(pyr + off, lev[k], sizeof(double) * 3 * (size_t)Wk * Hk);
    double* t = (double*)malloc(sizeof(double) * 3 * (size_t)Wk * Hk);
    for (int j = 0; j < Hk; ++j) /* rows */
      for (int i = 0; i < Wk; ++i)
        for (int c = 0; c < 3; ++c) {
          double sum = 0.0;
          for (int d = -R; d <= R; ++d) {
            int q = i + d < 0 ? 0 : (i + d >= Wk ? Wk - 1 : i + d);
            sum += w[d + R] * lev[k][3 * ((long)j * Wk + q) + c];
          }
          t[3 * ((long)j * Wk + i) + c] = sum;
        }
    for (int j = 0; j < Hk; ++j) /* columns */
      for (int i = 0; i < Wk; ++i)
        for (int c = 0; c < 3; ++c) {
          double sum = 0.0;
          for (int d = -R; d <= R; ++d) {
            int q = j + d < 0 ? 0 : (j + d >= Hk ? Hk - 1 : j + d);
            sum += w[d + R] * t[3 * ((long)q * Wk + i) + c];
          }
          lev[k][3 * ((long)j * Wk + i) + c] = sum;
        }
    free(t);
    if (blurred) memcpy(blurred + off, lev[k], sizeof(double) * 3 * (size_t)Wk * Hk);
    off += 3L * Wk * Hk;
  }
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      double add[3] = {0.0, 0.0, 0.0};
      for (int k = 1; k < L; ++k) {
        int Wk = Wl[k], Hk = Hl[k];
        double scale = (double)(1 << k);
        double u = (px + 0.5) / scale - 0.5, v = (py + 0.5) / scale - 0.5;
        double x0 = floor(u), y0 = floor(v), fx = u - x0, fy = v - y0;
        int i0 = (int)clampd(x0, 0, Wk - 1), i1 = (int)clampd(x0 + 1, 0, Wk - 1);
        int j0 = (int)clampd(y0, 0, Hk - 1), j1 = (int)clampd(y0 + 1, 0, Hk - 1);
        for (int c = 0; c < 3; ++c) {
          double a = lev[k][3 * ((long)j0 * Wk + i0) + c], b = lev[k][3 * ((long)j0 * Wk + i1) + c];
          double p = lev[k][3 * ((long)j1 * Wk + i0) + c], q = lev[k][3 * ((long)j1 * Wk + i1) + c];
          add[c] += (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * p + fx * q);
        }
      }
      for (int c = 0; c < 3; ++c) {
        long o = 3 * ((long)py * W + px) + c;
        y[o] = x[o] + bp->strength * add[c];
      }
    }
  for (int k = 0; k < L; ++k) free(lev[k]);
  return 0;
}

/* Helper exposed for tests: visibility of world point P for one light -> (vis, vis_lo, vis_hi). */
void or_shadow_vis(const or_shadows* sh, int light, const double* P, double* out) {
  shadow_vis(sh, light, P, &out[0], &out[1], &out[2]);
}

/* ------------------------------------------------------------------------------------------ */
/* Eye-dome lighting for point clouds (Sec. 4.2; Boucheny 2009)                                */
/* ------------------------------------------------------------------------------------------ */
/* Readings: the paper darkens a pixel the more its depth exceeds its screen neighbours'.
 *   obscurance  w(p) = (1/N) sum_k max(0, log2 e_p - log2 e_{q_k}), q_k = p + (round(r cos t_k),
 *               round(r sin t_k)), t_k = 2 pi k / N (round half away from zero, in FP64);
 *               a neighbour outside the image or without a surface counts as infinitely far
 *               (contributes 0)
 *   shade       s(p) = exp(-A w(p)) (A: strength); output = G-buffer colour * s * AO (AO
 *               optional, nearest at (x / ao_scale, y / ao_scale)); background pixels 0. */
typedef struct {
  double strength;
  int radius, directions;
} or_edl_params;

static double edl_log_depth(const double* gb, int W, int H, int x, int y) {
  if (x < 0 || y < 0 || x >= W || y >= H) return INFINITY;
  double e = gb[((long)y * W + x) * 9 + 8];
  return is_surface(e) ? log2(e) : INFINITY;
}

/* gb: W*H*9 decoded G-buffer (albedo 0..2, depth 8); out: W*H*3. */
int or_edl(const double* gb, int W, int H, const or_edl_params* ep, const double* ao, int ao_scale, double* out) {
  if (W < 1 || H < 1 || ep->radius < 1 || ep->directions < 1 || ep->directions > 64) return -1;
  int N = ep->directions, dx[64], dy[64];
  for (int k = 0; k < N; ++k) {
    double t = 2.0 * OR_PI * k / N;
    dx[k] = (int)round(ep->radius * cos(t));
    dy[k] = (int)round(ep->radius * sin(t));
  }
  int s = ao_scale > 0 ? ao_scale : 1, Wa = (W + s - 1) / s;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      long p = (long)y * W + x;
      double lp = edl_log_depth(gb, W, H, x, y);
      if (isinf(lp)) {
        out[3 * p] = out[3 * p + 1] = out[3 * p + 2] = 0.0;
        continue;
      }
      double w = 0.0;
      for (int k = 0; k < N; ++k) {
        double lq = edl_log_depth(gb, W, H, x + dx[k], y + dy[k]);
        double d = lp - lq;
        w += d > 0.0 ? d : 0.0;
      }
      w /= N;
      double sh = exp(-ep->strength * w);
      if (ao) sh *= ao[(long)(y / s) * Wa + x / s];
      for (int c = 0; c < 3; ++c) out[3 * p + c] = gb[p * 9 + c] * sh;
    }
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Mesh rendering into the G-buffer (Sec. 4.1)                                                 */
/* ------------------------------------------------------------------------------------------ */
/* Readings (the paper rasterises with OpenGL): pixel (x, y) is covered by a triangle when its
 * centre lies inside it; the nearest covering triangle (smallest eye depth, then smallest index)
 * writes the pixel; attributes are interpolated perspective-correctly (affine in 1/z).  Which
 * triangle covers a pixel is decided exactly: vertices go to view space and the screen in FP32
 * with every product, sum and quotient rounded (the CUDA path evaluates the same expressions),
 * are snapped to 1/256 pixel (round half to even), and coverage uses 64-bit integer edge
 * functions with a top-left rule on shared edges; the depth of the test is the FP32 value
 * A / ((b0 iz0 + b1 iz1) + b2 iz2) (b_i the integer edge functions, A their sum, iz_i = 1/z_i).
 * No clipping: a triangle with a vertex at eye depth below `near`, or projecting beyond 2^22
 * pixels, is not drawn; no back-face culling.  Vertices: 12 values each, position xyz, normal
 * xyz, albedo rgb, metal, rough, unused.  Attributes are interpolated in FP64 with the weights
 * b_i iz_i / sum_j b_j iz_j; the normal is normalised. */
typedef struct {
  float ax, ay, az;   /* view-space position */
  long long qx, qy;   /* snapped screen position, 1/256 px */
  float iz;           /* 1 / eye depth */
  int ok;
} or_rvert;

static or_rvert raster_vertex(const double* v, const or_camera* cam, float kx, float ky, float hw, float hh, float near) {
  /* view = R^T (p - eye), R's columns are the view axes in world space */
  float px = (float)v[0], py = (float)v[1], pz = (float)v[2];
  float ex = (float)cam->v2w[12], ey = (float)cam->v2w[13], ez = (float)cam->v2w[14];
  float dx = px - ex, dy = py - ey, dz = pz - ez;
  float r[9];
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < 3; ++i) r[3 * c + i] = (float)cam->v2w[4 * c + i]; /* column c, row i */
  or_rvert o;
  float t0, t1;
  t0 = r[0] * dx; t1 = r[1] * dy; o.ax = (t0 + t1); t0 = r[2] * dz; o.ax = o.ax + t0;
  t0 = r[3] * dx; t1 = r[4] * dy; o.ay = (t0 + t1); t0 = r[5] * dz; o.ay = o.ay + t0;
  t0 = r[6] * dx; t1 = r[7] * dy; o.az = (t0 + t1); t0 = r[8] * dz; o.az = o.az + t0;
  float e = -o.az;
  o.ok = e >= near;
  o.iz = 1.0f / e;
  float u = o.ax * o.iz, w = o.ay * o.iz;
  float X = hw * (1.0f + u * kx), Y = hh * (1.0f - w * ky);
  o.ok = o.ok && fabsf(X) < 4194304.0f && fabsf(Y) < 4194304.0f;
  o.qx = o.ok ? (long long)lrintf(X * 256.0f) : 0;
  o.qy = o.ok ? (long long)lrintf(Y * 256.0f) : 0;
  return o;
}

static long long edge_fn(long long ax, long long ay, long long bx, long long by, long long px, long long py) {
  return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

/* top-left rule for edge a -> b of a triangle with positive area in this orientation */
static int edge_bias(long long ax, long long ay, long long bx, long long by) {
  long long dx = bx - ax, dy = by - ay;
  return (dy < 0 || (dy == 0 && dx > 0)) ? 0 : -1;
}

/* verts: V*12, tris: T*3.  gb: W*H*9 (albedo 0..2, metal 3, normal 4..6, rough 7, depth 8;
 * background: zeros and depth +inf); ids: W*H triangle index or -1 (NULL allowed). */
int or_raster(const double* verts, int V, const int* tris, long T, const or_camera* cam, double near, double* gb,
              int* ids) {
  int W = cam->W, H = cam->H;
  double t = tan(0.5 * cam->fov_y);
  float ky = (float)(1.0 / t), kx = (float)((double)H / ((double)W * t));
  float hw = (float)(0.5 * W), hh = (float)(0.5 * H), nearf = (float)near;
  unsigned long long* best = (unsigned long long*)malloc(sizeof(unsigned long long) * (size_t)W * H);
  for (long p = 0; p < (long)W * H; ++p) best[p] = ~0ULL;
  for (long tr = 0; tr < T; ++tr) {
    int i0 = tris[3 * tr], i1 = tris[3 * tr + 1], i2 = tris[3 * tr + 2];
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= V || i1 >= V || i2 >= V) continue;
    or_rvert a = raster_vertex(verts + 12 * (long)i0, cam, kx, ky, hw, hh, nearf);
    or_rvert b = raster_vertex(verts + 12 * (long)i1, cam, kx, ky, hw, hh, nearf);
    or_rvert c = raster_vertex(verts + 12 * (long)i2, cam, kx, ky, hw, hh, nearf);
    if (!a.ok || !b.ok || !c.ok) continue;
    long long area = edge_fn(a.qx, a.qy, b.qx, b.qy, c.qx, c.qy);
    if (area == 0) continue;
    if (area < 0) { /* orient so that the area is positive */
      or_rvert tmp = b;
      b = c;
      c = tmp;
      area = -area;
    }
    long long xmin = a.qx < b.qx ? (a.qx < c.qx ? a.qx : c.qx) : (b.qx < c.qx ? b.qx : c.qx);
    long long xmax = a.qx > b.qx ? (a.qx > c.qx ? a.qx : c.qx) : (b.qx > c.qx ? b.qx : c.qx);
    long long ymin = a.qy < b.qy ? (a.qy < c.qy ? a.qy : c.qy) : (b.qy < c.qy ? b.qy : c.qy);
    long long ymax = a.qy > b.qy ? (a.qy > c.qy ? a.qy : c.qy) : (b.qy > c.qy ? b.qy : c.qy);
    /* pixels whose centre (256 x + 128) lies in [min, max] */
    long long x0 = (xmin - 128 + 255) >> 8, x1 = (xmax - 128) >> 8, y0 = (ymin - 128 + 255) >> 8, y1 = (ymax - 128) >> 8;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > W - 1) x1 = W - 1;
    if (y1 > H - 1) y1 = H - 1;
    int bab = edge_bias(a.qx, a.qy, b.qx, b.qy), bbc = edge_bias(b.qx, b.qy, c.qx, c.qy),
        bca = edge_bias(c.qx, c.qy, a.qx, a.qy);
    float areaf = (float)area;
    for (long long y = y0; y <= y1; ++y)
      for (long long x = x0; x <= x1; ++x) {
        long long px = 256 * x + 128, py = 256 * y + 128;
        long long wc = edge_fn(a.qx, a.qy, b.qx, b.qy, px, py); /* weight of c */
        long long wa = edge_fn(b.qx, b.qy, c.qx, c.qy, px, py); /* weight of a */
        long long wb = edge_fn(c.qx, c.qy, a.qx, a.qy, px, py); /* weight of b */
        /* inside: every weight positive, or zero on a top-left edge */
        if (wc < 0 || wa < 0 || wb < 0) continue;
        if ((wc == 0 && bab) || (wa == 0 && bbc) || (wb == 0 && bca)) continue;
        float fa = (float)wa, fb = (float)wb, fc = (float)wc;
        float s0 = fa * a.iz, s1 = fb * b.iz, s2 = fc * c.iz;
        float sum = (s0 + s1) + s2;
        float z = areaf / sum;
        unsigned zb;
        memcpy(&zb, &z, 4);
        unsigned long long key = ((unsigned long long)zb << 32) | (unsigned long long)tr;
        long p = (long)y * W + x;
        if (key < best[p]) best[p] = key;
      }
  }
  for (long p = 0; p < (long)W * H; ++p) {
    double* o = gb + 9 * p;
    if (best[p] == ~0ULL) {
      for (int q = 0; q < 8; ++q) o[q] = 0.0;
      o[8] = INFINITY;
      if (ids) ids[p] = -1;
      continue;
    }
    long tr = (long)(best[p] & 0xffffffffULL);
    unsigned zb = (unsigned)(best[p] >> 32);
    float z;
    memcpy(&z, &zb, 4);
    int vi[3] = {tris[3 * tr], tris[3 * tr + 1], tris[3 * tr + 2]};
    or_rvert r3[3];
    for (int k = 0; k < 3; ++k) r3[k] = raster_vertex(verts + 12 * (long)vi[k], cam, kx, ky, hw, hh, nearf);
    long long px = 256 * (p % W) + 128, py = 256 * (p / W) + 128;
    /* barycentric weights in FP64 from the exact edge functions (orientation-independent) */
    double bw[3];
    bw[0] = (double)edge_fn(r3[1].qx, r3[1].qy, r3[2].qx, r3[2].qy, px, py);
    bw[1] = (double)edge_fn(r3[2].qx, r3[2].qy, r3[0].qx, r3[0].qy, px, py);
    bw[2] = (double)edge_fn(r3[0].qx, r3[0].qy, r3[1].qx, r3[1].qy, px, py);
    double wsum = 0.0, w[3];
    for (int k = 0; k < 3; ++k) {
      w[k] = bw[k] / (-(double)r3[k].az);
      wsum += w[k];
    }
    for (int k = 0; k < 3; ++k) w[k] /= wsum;
    double attr[11] = {0};
    for (int k = 0; k < 3; ++k)
      for (int q = 0; q < 11; ++q) attr[q] += w[k] * verts[12 * (long)vi[k] + q];
    double n[3] = {attr[3], attr[4], attr[5]};
    normalize3(n);
    o[0] = attr[6];
    o[1] = attr[7];
    o[2] = attr[8];
    o[3] = attr[9];
    o[4] = n[0];
    o[5] = n[1];
    o[6] = n[2];
    o[7] = attr[10];
    o[8] = z;
    if (ids) ids[p] = (int)tr;
  }
  free(best);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* surfel splatting into the G-buffer (Sec. 4.3)                                              */
/* ------------------------------------------------------------------------------------------ */
/* A surfel is an oriented elliptical disk.  Record of 16 values: centre p.xyz, semi-axis a (along
 * the tangent), normal n.xyz, semi-axis b (along the bitangent), tangent t.xyz, metal,
 * albedo.rgb, rough.  The paper draws each surfel as a rectangle on its (normal, tangent,
 * bitangent) basis, discards the fragments outside the ellipse, and lets surfels that overlap
 * within a small depth distance accumulate their attributes and a weight, the composing pass
 * dividing by the weight.  Readings:
 *   - the surfel's frame in view space: centre c = R^T (p - eye), unit normal n^ = R^T n / |R^T n|,
 *     unit tangent t^ = the part of R^T t orthogonal to n^, normalised, bitangent b^ = n^ x t^.  A
 *     surfel is dropped when its normal or orthogonalised tangent is zero, a semi-axis is not a
 *     positive finite number, or its nearest possible point is nearer than `near` (eye depth of c
 *     minus (a + b) below near);
 *   - the ray through a pixel centre, d = (u_x, u_y, -1) at eye depth 1 with
 *     u_x = ((x + 1/2) / hw - 1) / k_x and u_y = (1 - (y + 1/2) / hh) / k_y, meets the surfel's
 *     plane at eye depth s = (n^ . c) / (n^ . d); the pixel is covered when 0 < s < inf and the
 *     hit point's coordinates u = s (d . t^) - c . t^ and v = s (d . b^) - c . b^ satisfy
 *     u^2 / a^2 + v^2 / b^2 <= 1 (both faces count).  The test is evaluated multiplied through by
 *     (n^ . d)^2, without the quotient: U = (n^ . c)(d . t^) - (n^ . d)(c . t^), V likewise with
 *     b^, covered when (n^ . c)(n^ . d) > 0 and U^2 / a^2 + V^2 / b^2 <= (n^ . d)^2; s itself is
 *     formed only for a covered pixel;
 *   - the pixel's depth is the smallest s over the covering surfels; every covering surfel with
 *     s <= (that depth) * (1 + tol) adds its albedo, world-space unit normal, metal and rough with
 *     weight 1; the G-buffer holds the weighted means (the summed normal renormalised, a zero sum
 *     left zero) and the smallest depth; a pixel no surfel covers is background (zeros, depth
 *     +inf), and its weight is 0.
 * The decisions (which surfels survive, which pixels they cover, the smallest depth, the depth
 * window) are evaluated in FP32, each product, sum, quotient and square root rounded, in the
 * order written here; the sums and means are FP64.  The pixel box searched per surfel is the
 * bounding box of its rectangle's projected corners (FP64) widened by two pixels. */
typedef struct {
  float c[3], n[3], t[3], b[3];
  float nc, ct, cb, ia2, ib2;
  double nw[3];
  double box[4]; /* x0, y0, x1, y1 */
  int ok;
} or_surfel;

static float dot3f(const float* a, const float* b) {
  float t0 = a[0] * b[0];
  float t1 = a[1] * b[1];
  float s = t0 + t1;
  float t2 = a[2] * b[2];
  return s + t2;
}

static or_surfel surfel_setup(const double* rec, const float* axes /* 3 view axes in world space */,
                              const float* eye, float near, float kx, float ky, float hw, float hh) {
  or_surfel o;
  memset(&o, 0, sizeof(o));
  float p[3] = {(float)rec[0], (float)rec[1], (float)rec[2]};
  float nw[3] = {(float)rec[4], (float)rec[5], (float)rec[6]};
  float tw[3] = {(float)rec[8], (float)rec[9], (float)rec[10]};
  float a = (float)rec[3], b = (float)rec[7];
  float d[3] = {p[0] - eye[0], p[1] - eye[1], p[2] - eye[2]};
  float nv[3], tv[3];
  for (int k = 0; k < 3; ++k) {
    o.c[k] = dot3f(axes + 3 * k, d);
    nv[k] = dot3f(axes + 3 * k, nw);
    tv[k] = dot3f(axes + 3 * k, tw);
  }
  if (!(a > 0.0f) || !(b > 0.0f) || !(a < INFINITY) || !(b < INFINITY)) return o;
  float nn = dot3f(nv, nv);
  if (!(nn > 0.0f) || !(nn < INFINITY)) return o;
  float inv = 1.0f / sqrtf(nn);
  for (int k = 0; k < 3; ++k) o.n[k] = nv[k] * inv;
  float dt = dot3f(tv, o.n);
  float tp[3];
  for (int k = 0; k < 3; ++k) {
    float m = o.n[k] * dt;
    tp[k] = tv[k] - m;
  }
  float tt = dot3f(tp, tp);
  if (!(tt > 0.0f) || !(tt < INFINITY)) return o;
  float invt = 1.0f / sqrtf(tt);
  for (int k = 0; k < 3; ++k) o.t[k] = tp[k] * invt;
  {
    float m0, m1;
    m0 = o.n[1] * o.t[2]; m1 = o.n[2] * o.t[1]; o.b[0] = m0 - m1;
    m0 = o.n[2] * o.t[0]; m1 = o.n[0] * o.t[2]; o.b[1] = m0 - m1;
    m0 = o.n[0] * o.t[1]; m1 = o.n[1] * o.t[0]; o.b[2] = m0 - m1;
  }
  float ec = -o.c[2];
  float reach = a + b;
  if (!(ec - reach >= near)) return o;
  o.nc = dot3f(o.n, o.c);
  o.ct = dot3f(o.c, o.t);
  o.cb = dot3f(o.c, o.b);
  float a2 = a * a, b2 = b * b;
  o.ia2 = 1.0f / a2;
  o.ib2 = 1.0f / b2;
  /* world-space unit normal for the sums */
  double ln = sqrt(rec[4] * rec[4] + rec[5] * rec[5] + rec[6] * rec[6]);
  for (int k = 0; k < 3; ++k) o.nw[k] = rec[4 + k] / ln;
  /* pixel box: projected corners c +- a t^ +- b b^ (FP64), widened by two pixels */
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
  for (int sa = -1; sa <= 1; sa += 2)
    for (int sb = -1; sb <= 1; sb += 2) {
      double q[3];
      for (int k = 0; k < 3; ++k) q[k] = (double)o.c[k] + sa * (double)a * o.t[k] + sb * (double)b * o.b[k];
      double e = -q[2];
      double X = hw * (1.0 + q[0] / e * kx), Y = hh * (1.0 - q[1] / e * ky);
      if (X < xmin) xmin = X;
      if (X > xmax) xmax = X;
      if (Y < ymin) ymin = Y;
      if (Y > ymax) ymax = Y;
    }
  o.box[0] = floor(xmin - 0.5) - 2.0;
  o.box[1] = floor(ymin - 0.5) - 2.0;
  o.box[2] = ceil(xmax - 0.5) + 2.0;
  o.box[3] = ceil(ymax - 0.5) + 2.0;
  o.ok = 1;
  return o;
}

/* eye depth at which the ray (ux, uy, -1) meets the surfel inside its ellipse, else 0 */
static float surfel_hit(const or_surfel* s, float ux, float uy) {
  float m0, m1;
  m0 = s->n[0] * ux; m1 = s->n[1] * uy; float nd = m0 + m1; nd = nd - s->n[2]; /* n^ . d */
  m0 = s->t[0] * ux; m1 = s->t[1] * uy; float dt = m0 + m1; dt = dt - s->t[2]; /* d . t^ */
  m0 = s->b[0] * ux; m1 = s->b[1] * uy; float db = m0 + m1; db = db - s->b[2]; /* d . b^ */
  float sign = s->nc * nd;
  if (!(sign > 0.0f)) return 0.0f;
  m0 = s->nc * dt; m1 = nd * s->ct; float U = m0 - m1;
  m0 = s->nc * db; m1 = nd * s->cb; float V = m0 - m1;
  float pu = U * U, pv = V * V;
  pu = pu * s->ia2;
  pv = pv * s->ib2;
  float e = pu + pv;
  float n2 = nd * nd;
  if (!(e <= n2)) return 0.0f;
  float sd = s->nc / nd;
  return (sd > 0.0f && sd < INFINITY) ? sd : 0.0f;
}

/* recs: N*16.  gb: W*H*9 as or_raster; weight: W*H (NULL allowed). */
int or_surfels(const double* recs, long N, const or_camera* cam, double near, double tol, double* gb, double* weight) {
  int W = cam->W, H = cam->H;
  double t = tan(0.5 * cam->fov_y);
  float ky = (float)(1.0 / t), kx = (float)((double)H / ((double)W * t));
  float hw = (float)(0.5 * W), hh = (float)(0.5 * H), nearf = (float)near;
  float f = 1.0f + (float)tol;
  float axes[9], eye[3];
  for (int c = 0; c < 3; ++c) {
    for (int i = 0; i < 3; ++i) axes[3 * c + i] = (float)cam->v2w[4 * c + i];
    eye[c] = (float)cam->v2w[12 + c];
  }
  float* ux = (float*)malloc(sizeof(float) * W);
  float* uy = (float*)malloc(sizeof(float) * H);
  for (int x = 0; x < W; ++x) {
    float q = ((float)x + 0.5f) / hw;
    q = q - 1.0f;
    ux[x] = q / kx;
  }
  for (int y = 0; y < H; ++y) {
    float q = ((float)y + 0.5f) / hh;
    q = 1.0f - q;
    uy[y] = q / ky;
  }
  float* emin = (float*)malloc(sizeof(float) * (size_t)W * H);
  double* acc = (double*)calloc((size_t)W * H * 9, sizeof(double));
  for (long p = 0; p < (long)W * H; ++p) emin[p] = INFINITY;
  or_surfel* S = (or_surfel*)malloc(sizeof(or_surfel) * (N > 0 ? N : 1));
  for (long i = 0; i < N; ++i) S[i] = surfel_setup(recs + 16 * i, axes, eye, nearf, kx, ky, hw, hh);
  for (int pass = 0; pass < 2; ++pass)
    for (long i = 0; i < N; ++i) {
      const or_surfel* s = &S[i];
      if (!s->ok) continue;
      long x0 = s->box[0] < 0 ? 0 : (long)s->box[0], y0 = s->box[1] < 0 ? 0 : (long)s->box[1];
      long x1 = s->box[2] > W - 1 ? W - 1 : (long)s->box[2], y1 = s->box[3] > H - 1 ? H - 1 : (long)s->box[3];
      for (long y = y0; y <= y1; ++y)
        for (long x = x0; x <= x1; ++x) {
          float sd = surfel_hit(s, ux[x], uy[y]);
          if (sd == 0.0f) continue;
          long p = y * W + x;
          if (pass == 0) {
            if (sd < emin[p]) emin[p] = sd;
            continue;
          }
          float thr = emin[p] * f;
          if (!(sd <= thr)) continue;
          const double* r = recs + 16 * i;
          double* a = acc + 9 * p;
          a[0] += r[12];
          a[1] += r[13];
          a[2] += r[14];
          a[3] += r[11];
          a[4] += s->nw[0];
          a[5] += s->nw[1];
          a[6] += s->nw[2];
          a[7] += r[15];
          a[8] += 1.0;
        }
    }
  for (long p = 0; p < (long)W * H; ++p) {
    double* o = gb + 9 * p;
    const double* a = acc + 9 * p;
    if (weight) weight[p] = a[8];
    if (a[8] == 0.0) {
      for (int q = 0; q < 8; ++q) o[q] = 0.0;
      o[8] = INFINITY;
      continue;
    }
    for (int q = 0; q < 4; ++q) o[q] = a[q] / a[8];
    double n[3] = {a[4], a[5], a[6]};
    double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int k = 0; k < 3; ++k) o[4 + k] = ln > 0.0 ? n[k] / ln : 0.0;
    o[7] = a[7] / a[8];
    o[8] = emin[p];
  }
  free(S);
  free(acc);
  free(emin);
  free(uy);
  free(ux);
  return 0;
}
