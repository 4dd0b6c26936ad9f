/*
 * flame_oracle.c -- plain FP64 CPU oracle for the render / compare / adjust
 * loop of Shen et al., "Radiative Transport Based Flame Volume Reconstruction
 * from Videos" (arXiv 1809.06417).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  The GPU library shares no
 * source, header, table or helper with it.  Everything here is a direct,
 * unblocked restatement of the paper's steps in double precision, written for a
 * reader to check against the paper by eye; nothing is tuned.
 *
 * Conventions (the paper leaves them open; each is a stated reading):
 *  - Key points (Sec. 3.3 definitions) are grid nodes.  Node (i,j,k) sits at
 *    world position origin + h*(i,j,k); values at any other point are the
 *    trilinear blend of the 8 surrounding key points.  All ray arithmetic is
 *    done in voxel coordinates (world / h), so lengths, the sampling step and
 *    the key-point distance D of Eq. 10 are in voxel edge lengths.
 *  - A node record holds {S_r, S_g, S_b, sigma_t}: the emitted radiance source
 *    per voxel length of Eq. 5 and the extinction coefficient per voxel length.
 *  - Rays start at the pinhole, pass through pixel centres (row 0 on top), are
 *    clipped to the node box [0, n-1]^3, and are cut into segments of length
 *    `step`; each segment is sampled at its midpoint (the last one is shorter).
 *  - Field mode integrates Eq. 6 exactly for piecewise-constant samples:
 *    a segment of length l with source S and extinction s adds
 *    T * S * (1 - exp(-s l)) / s and multiplies T by exp(-s l).
 *  - Constant-tau mode (tau > 0) is the paper-literal under blending of
 *    Eqs. 7-8 with every sample's opacity equal to tau, so that the k-th sample
 *    (1-based) sees T = (1 - tau)^(k-1) (Eq. 12).
 *  - The background E(s_b) of Eq. 6 is black (Sec. 4.1).
 *
 * Parity pins: see tests/test_oracle_*.py.  The in-scattering estimate
 * (orc_scatter_J) has no algorithm in the paper: parity unpinned against the
 * paper; it is pinned only by the homogeneous-slab closed form and by the
 * albedo-zero reduction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#define ORC_THREAD() omp_get_thread_num()
#else
#define ORC_THREAD() 0
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    int32_t nx, ny, nz, pad_;
    double origin[3];
    double h;
} orc_grid;

typedef struct {
    double pos[3], right[3], up[3], fwd[3];
    double tan_half_fov; /* tan of half the vertical field of view */
    int32_t width, height;
} orc_cam;

typedef struct {
    double step;         /* sampling step, voxel edge lengths (Sec. 4.2) */
    double alpha_l;      /* Eq. 10 residual scale */
    double alpha_d;      /* Eq. 10 distance scale */
    double tau;          /* > 0: constant sample opacity (Eqs. 7, 8, 12) */
    double g_std;        /* spread of G(s) around its mean of 1 (Eq. 11) */
    double flame_thresh; /* flame-pixel threshold (Sec. 4.1), image units */
    uint64_t seed;       /* key of the G(s) stream */
    int32_t clamp_nonneg;/* clamp updated values at 0 */
    int32_t pad_;
    double hg_g;         /* Henyey-Greenstein asymmetry of the in-scattering (Eq. 9); 0: isotropic */
    int32_t sequential;  /* 1: views update the volume one after another (Kaczmarz order) */
    int32_t storage;     /* orc_reconstruct: 0 records held in double; ORC_BF16 / ORC_F16: every
                            record the loop stores (volume, in-scattering source) is rounded to
                            that type, as a volume kept in 16-bit storage is */
} orc_params;

enum { ORC_STORE_F64 = 0, ORC_BF16 = 1, ORC_F16 = 2 };

/* Temperature-to-RGB table (Sec. 3.3.3): m entries over [t_min, t_max]. */
typedef struct {
    const double *lut;   /* m x 3, row i at t_min + i*(t_max-t_min)/(m-1) */
    int32_t m, pad_;
    double t_min, t_max;
} orc_lut;

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

static int64_t node_index(const orc_grid *g, int i, int j, int k)
{
    return ((int64_t)k * g->ny + j) * g->nx + i;
}

/* Pinhole ray through the centre of pixel (px, py) in voxel coordinates. */
static void camera_ray(const orc_grid *g, const orc_cam *c, int px, int py,
                       double o[3], double d[3])
{
    double aspect = (double)c->width / (double)c->height;
    double x = (2.0 * (px + 0.5) / c->width - 1.0) * c->tan_half_fov * aspect;
    double y = (1.0 - 2.0 * (py + 0.5) / c->height) * c->tan_half_fov;
    double n2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        d[a] = c->fwd[a] + x * c->right[a] + y * c->up[a];
        n2 += d[a] * d[a];
        o[a] = (c->pos[a] - g->origin[a]) / g->h;
    }
    double inv = 1.0 / sqrt(n2);
    for (int a = 0; a < 3; ++a) d[a] *= inv;
}

/* Slab clip of o + t d against the node box [0, n-1]^3; t >= 0 only.
 * Returns 1 and [t0, t1] with t1 > t0 when the ray enters the box. */
static int clip_ray(const orc_grid *g, const double o[3], const double d[3],
                    double *t0, double *t1)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    double tin = -INFINITY, tout = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = 0.0, hi = (double)(n[a] - 1);
        if (d[a] == 0.0) {
            if (o[a] < lo || o[a] > hi) return 0;
            continue;
        }
        double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
        if (ta > tb) { double s = ta; ta = tb; tb = s; }
        if (ta > tin) tin = ta;
        if (tb < tout) tout = tb;
    }
    if (tin < 0.0) tin = 0.0;
    if (!(tout > tin)) return 0;
    *t0 = tin;
    *t1 = tout;
    return 1;
}

static int64_t segment_count(double t0, double t1, double step)
{
    return (int64_t)ceil((t1 - t0) / step);
}

/* Segment k of a clipped ray: its length and midpoint. */
static void segment(const double o[3], const double d[3], double t0, double t1,
                    double step, int64_t k, double *len, double p[3])
{
    double ta = t0 + (double)k * step;
    double tb = ta + step;
    if (tb > t1) tb = t1;
    *len = tb - ta;
    double tm = 0.5 * (ta + tb);
    for (int a = 0; a < 3; ++a) p[a] = o[a] + tm * d[a];
}

/* Cell of the sample point and its fractional position in it.  The cell
 * index is clamped to [0, n-2] so that points on the upper face use the last
 * cell with fraction 1. */
static void locate(const orc_grid *g, const double p[3], int c[3], double f[3])
{
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) {
        int i = (int)floor(p[a]);
        if (i < 0) i = 0;
        if (i > n[a] - 2) i = n[a] - 2;
        double fr = p[a] - (double)i;
        if (fr < 0.0) fr = 0.0;
        if (fr > 1.0) fr = 1.0;
        c[a] = i;
        f[a] = fr;
    }
}

/* The eight key points around a sample (Sec. 3.3, sample points): node
 * indices and trilinear weights, corner b = dx + 2 dy + 4 dz. */
static void corners(const orc_grid *g, const int c[3], const double f[3],
                    int64_t idx[8], double w[8])
{
    for (int b = 0; b < 8; ++b) {
        int dx = b & 1, dy = (b >> 1) & 1, dz = (b >> 2) & 1;
        idx[b] = node_index(g, c[0] + dx, c[1] + dy, c[2] + dz);
        w[b] = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) *
               (dz ? f[2] : 1.0 - f[2]);
    }
}

/* ------------------------------------------------------------------------ */
/* Threads and storage types                                                 */
/* ------------------------------------------------------------------------ */

/* Threads the pixel loops of rendering and adjustment and the node loop of
 * the visual hull run on (1 unless set; OpenMP builds only).  Pixels are
 * independent, so renders do not depend on it; the adjustment sums each
 * thread's share in its own buffer and adds the buffers in thread order, so
 * its sums are regrouped (FP64 rounding only) when the count changes. */
static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 1 ? n : 1; }

/* Threads the next parallel loop can use (1 in a build without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return g_threads;
#else
    return 1;
#endif
}

/* x rounded to the nearest value with `bits` significant binary digits
 * (ties to even), whose exponent is at least e_min (below it, numbers are
 * spaced 2^(e_min - bits + 1) apart, the subnormals of the type): the
 * rounding of a binary floating-point type with that many digits and that
 * smallest normal exponent.  Overflow is not handled (the fields here stay
 * far below the types' largest values). */
static double round_digits(double x, int bits, int e_min)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e);                    /* |x| in [2^(e-1), 2^e) */
    if (e - 1 < e_min) e = e_min + 1;
    const double q = ldexp(1.0, e - bits);   /* spacing of the representable values there */
    return nearbyint(x / q) * q;     /* the default rounding mode: to nearest, ties to even */
}

/* Round n values to a 16-bit storage type: bfloat16 (8 significant digits,
 * the exponent range of float32, smallest normal 2^-126) or IEEE binary16
 * (11 digits, smallest normal 2^-14).  mode 0 leaves them. */
void orc_round_storage(int64_t n, double *x, int mode)
{
    if (mode == ORC_STORE_F64) return;
    const int bits = mode == ORC_BF16 ? 8 : 11, e_min = mode == ORC_BF16 ? -126 : -14;
    for (int64_t i = 0; i < n; ++i) x[i] = round_digits(x[i], bits, e_min);
}

/* ------------------------------------------------------------------------ */
/* Colour-temperature mapping (Sec. 3.3.3)                                   */
/* ------------------------------------------------------------------------ */

static const double PLANCK_H = 6.62607015e-34;
static const double LIGHT_C = 299792458.0;
static const double BOLTZMANN_K = 1.380649e-23;

/* Planck's law, spectral radiance per metre of wavelength (Sec. 3.3.3). */
double orc_planck(double lambda_m, double temp_k)
{
    double x = PLANCK_H * LIGHT_C / (lambda_m * BOLTZMANN_K * temp_k);
    return 2.0 * PLANCK_H * LIGHT_C * LIGHT_C / pow(lambda_m, 5.0) / expm1(x);
}

/* Camera response of channel ch (0 R, 1 G, 2 B): a Gaussian in wavelength. */
static double response(int ch, double lambda_nm)
{
    static const double mu[3] = {600.0, 540.0, 460.0};
    const double w = 40.0;
    double u = (lambda_nm - mu[ch]) / w;
    return exp(-0.5 * u * u);
}

/* Unnormalised channel value: trapezoid rule over 380..780 nm in 1 nm steps. */
static double channel_raw(int ch, double temp_k)
{
    double acc = 0.0;
    for (int i = 0; i <= 400; ++i) {
        double lam = 380.0 + i;
        double wgt = (i == 0 || i == 400) ? 0.5 : 1.0;
        acc += wgt * orc_planck(lam * 1e-9, temp_k) * response(ch, lam);
    }
    return acc * 1e-9; /* d(lambda) = 1 nm */
}

/* RGB of a black body at temp_k, scaled so the green value at 2000 K is 1. */
void orc_temp_rgb(double temp_k, double out[3])
{
    double s = 1.0 / channel_raw(1, 2000.0);
    for (int ch = 0; ch < 3; ++ch) out[ch] = s * channel_raw(ch, temp_k);
}

void orc_lut_build(double t_min, double t_max, int m, double *lut)
{
    for (int i = 0; i < m; ++i) {
        double t = t_min + (t_max - t_min) * (double)i / (double)(m - 1);
        orc_temp_rgb(t, lut + 3 * (int64_t)i);
    }
}

/* Piecewise-linear table lookup and the derivative of that interpolant;
 * clamped (derivative 0) outside [t_min, t_max]. */
static void lut_eval(const orc_lut *L, double t, double q[3], double dq[3])
{
    double span = L->t_max - L->t_min;
    double u = (t - L->t_min) / span * (double)(L->m - 1);
    int inside = 1;
    if (u < 0.0) { u = 0.0; inside = 0; }
    if (u > (double)(L->m - 1)) { u = (double)(L->m - 1); inside = 0; }
    int i = (int)floor(u);
    if (i > L->m - 2) i = L->m - 2;
    double f = u - (double)i;
    for (int ch = 0; ch < 3; ++ch) {
        double a = L->lut[3 * (int64_t)i + ch], b = L->lut[3 * (int64_t)(i + 1) + ch];
        q[ch] = a + f * (b - a);
        dq[ch] = inside ? (b - a) * (double)(L->m - 1) / span : 0.0;
    }
}

/* Temperature from a green value (Sec. 3.3.3: the temperature is recovered
 * through the green channel, which grows with temperature over the table's
 * range): the inverse of the table's piecewise-linear green interpolant.  The
 * segment i with g_i <= g <= g_{i+1} is found by bisection; values below the
 * first entry give t_min, above the last t_max.  The green column must be
 * strictly increasing. */
double orc_green_to_temp(const orc_lut *L, double green)
{
    const double *lut = L->lut;
    const int m = L->m;
    if (!(green > lut[1])) return L->t_min;
    if (!(green < lut[3 * (int64_t)(m - 1) + 1])) return L->t_max;
    int lo = 0, hi = m - 1;   /* lut_g[lo] < green < lut_g[hi] */
    while (hi - lo > 1) {
        const int mid = lo + (hi - lo) / 2;
        if (lut[3 * (int64_t)mid + 1] <= green) lo = mid;
        else hi = mid;
    }
    const double a = lut[3 * (int64_t)lo + 1], b = lut[3 * (int64_t)hi + 1];
    const double f = (green - a) / (b - a);
    return L->t_min + ((double)lo + f) * (L->t_max - L->t_min) / (double)(m - 1);
}

/* Henyey-Greenstein phase function, Eq. 9; cos_wi = omega . omega_i. */
double orc_hg_phase(double g, double cos_wi)
{
    double den = 1.0 + g * g + 2.0 * g * cos_wi;
    return (1.0 - g * g) / (4.0 * ORC_PI * den * sqrt(den));
}

/* ------------------------------------------------------------------------ */
/* G(s) of Eq. 11: Gaussian with mean 1 from a counter-based stream.         */
/* The draw for sample k of pixel p in view v at iteration it uses outputs   */
/* 2c+1 and 2c+2 of the SplitMix64 sequence (Steele, Lea and Flood, OOPSLA   */
/* 2014) started at `seed`, where c packs (it, v, p, k) into 64 bits, and    */
/* turns them into a normal deviate by the Box-Muller transform.             */
/* ------------------------------------------------------------------------ */

static uint64_t splitmix_out(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_g_counter(int iteration, int view, int64_t pixel, int64_t k)
{
    return ((uint64_t)iteration << 44) | ((uint64_t)view << 36) |
           ((uint64_t)pixel << 14) | (uint64_t)k;
}

double orc_g_draw(uint64_t seed, double g_std, int iteration, int view,
                  int64_t pixel, int64_t k)
{
    if (g_std == 0.0) return 1.0;
    uint64_t c = orc_g_counter(iteration, view, pixel, k);
    uint64_t r1 = splitmix_out(seed, 2 * c + 1), r2 = splitmix_out(seed, 2 * c + 2);
    double u1 = ((double)(r1 >> 40) + 0.5) / 16777216.0;
    double u2 = (double)(r2 >> 40) / 16777216.0;
    return 1.0 + g_std * sqrt(-2.0 * log(u1)) * cos(2.0 * ORC_PI * u2);
}

/* ------------------------------------------------------------------------ */
/* Sampling a node field at a point                                          */
/* ------------------------------------------------------------------------ */

/* Volume kinds: RGB records {S_r,S_g,S_b,sigma}, or temperature records
 * {T, sigma} mapped to RGB through the table. */
enum { ORC_RGB = 0, ORC_TEMP = 1 };

typedef struct {
    int kind;
    const double *vol;
    const orc_lut *lut;
} orc_field;

typedef struct {
    int64_t idx[8];
    double w[8];
    double S[3];     /* source (or colour V in constant-tau mode) */
    double sigma;
    double temp;     /* temperature at the sample (ORC_TEMP) */
    double dS_dT[3]; /* table slope at the sample (ORC_TEMP) */
} orc_sample;

static void sample_field(const orc_grid *g, const orc_field *F, const double p[3],
                         orc_sample *s)
{
    int c[3];
    double f[3];
    locate(g, p, c, f);
    corners(g, c, f, s->idx, s->w);
    s->S[0] = s->S[1] = s->S[2] = 0.0;
    s->sigma = 0.0;
    s->temp = 0.0;
    if (F->kind == ORC_RGB) {
        for (int b = 0; b < 8; ++b) {
            const double *r = F->vol + 4 * s->idx[b];
            for (int ch = 0; ch < 3; ++ch) s->S[ch] += s->w[b] * r[ch];
            s->sigma += s->w[b] * r[3];
        }
    } else {
        for (int b = 0; b < 8; ++b) {
            const double *r = F->vol + 2 * s->idx[b];
            s->temp += s->w[b] * r[0];
            s->sigma += s->w[b] * r[1];
        }
        lut_eval(F->lut, s->temp, s->S, s->dS_dT);
    }
}

/* (1 - exp(-sigma l)) / sigma and its derivative in sigma, evaluated without
 * cancellation for small optical depth. */
static void segment_weight(double sigma, double len, double *beta, double *dbeta)
{
    double a = sigma * len;
    if (fabs(a) < 1e-3) {
        *beta = len * (1.0 - a / 2.0 + a * a / 6.0 - a * a * a / 24.0 + a * a * a * a / 120.0);
        *dbeta = -len * len * (0.5 - a / 3.0 + a * a / 8.0 - a * a * a / 30.0);
    } else {
        *beta = -expm1(-a) / sigma;
        *dbeta = (len * exp(-a) - *beta) / sigma;
    }
}

/* ------------------------------------------------------------------------ */
/* Forward rendering (Eqs. 5-8, 12; Algorithm 2, rendering half)             */
/* ------------------------------------------------------------------------ */

/* Radiance of one pixel; returns the number of samples taken. */
static int64_t render_pixel(const orc_grid *g, const orc_field *F, const orc_cam *c,
                            const orc_params *P, int px, int py, double L[3],
                            double *t_final)
{
    double o[3], d[3], t0, t1;
    L[0] = L[1] = L[2] = 0.0;
    if (t_final) *t_final = 1.0;
    camera_ray(g, c, px, py, o, d);
    if (!clip_ray(g, o, d, &t0, &t1)) return 0;
    int64_t n = segment_count(t0, t1, P->step);
    double T = 1.0;
    for (int64_t k = 0; k < n; ++k) {
        double len, p[3];
        orc_sample s;
        segment(o, d, t0, t1, P->step, k, &len, p);
        sample_field(g, F, p, &s);
        if (P->tau > 0.0) {
            for (int ch = 0; ch < 3; ++ch) L[ch] += T * P->tau * s.S[ch];
            T *= 1.0 - P->tau;
        } else {
            double beta, dbeta;
            segment_weight(s.sigma, len, &beta, &dbeta);
            for (int ch = 0; ch < 3; ++ch) L[ch] += T * s.S[ch] * beta;
            T *= exp(-s.sigma * len);
        }
    }
    if (t_final) *t_final = T;
    return n;
}

static int64_t render_views(const orc_grid *g, const orc_field *F, const orc_cam *cams,
                            int ncam, const orc_params *P, double *out, double *t_out)
{
    int64_t total = 0, off = 0;
    for (int v = 0; v < ncam; ++v) {
        const orc_cam *c = cams + v;
        int64_t view_total = 0;
#pragma omp parallel for num_threads(g_threads) schedule(static, 1) reduction(+ : view_total)
        for (int py = 0; py < c->height; ++py)
            for (int px = 0; px < c->width; ++px) {
                int64_t pix = off + (int64_t)py * c->width + px;
                view_total += render_pixel(g, F, c, P, px, py, out + 3 * pix,
                                           t_out ? t_out + pix : NULL);
            }
        total += view_total;
        off += (int64_t)c->width * c->height;
    }
    return total;
}

/* Render every pixel of every view.  vol: N^3 x 4 records.  out: 3 values per
 * pixel, views concatenated, rows top to bottom.  t_out (nullable): final
 * transmittance per pixel.  Returns the number of samples taken. */
int64_t orc_render(const orc_grid *g, const double *vol, const orc_cam *cams, int ncam,
                   const orc_params *P, double *out, double *t_out)
{
    orc_field F = {ORC_RGB, vol, NULL};
    return render_views(g, &F, cams, ncam, P, out, t_out);
}

int64_t orc_render_temp(const orc_grid *g, const double *vol_ts, const orc_lut *lut,
                        const orc_cam *cams, int ncam, const orc_params *P, double *out)
{
    orc_field F = {ORC_TEMP, vol_ts, lut};
    return render_views(g, &F, cams, ncam, P, out, NULL);
}

/* One ray, sample by sample: for each segment k its length, midpoint (voxel
 * coordinates) and the transmittance T_k in front of it.  Returns the number
 * of segments (at most max_n are written). */
int64_t orc_trace_pixel(const orc_grid *g, const double *vol, const orc_cam *c,
                        const orc_params *P, int px, int py, int64_t max_n,
                        double *t_before, double *len_out, double *pos_out)
{
    orc_field F = {ORC_RGB, vol, NULL};
    double o[3], d[3], t0, t1;
    camera_ray(g, c, px, py, o, d);
    if (!clip_ray(g, o, d, &t0, &t1)) return 0;
    int64_t n = segment_count(t0, t1, P->step);
    double T = 1.0;
    for (int64_t k = 0; k < n; ++k) {
        double len, p[3];
        orc_sample s;
        segment(o, d, t0, t1, P->step, k, &len, p);
        sample_field(g, &F, p, &s);
        if (k < max_n) {
            t_before[k] = T;
            len_out[k] = len;
            for (int a = 0; a < 3; ++a) pos_out[3 * k + a] = p[a];
        }
        T *= P->tau > 0.0 ? 1.0 - P->tau : exp(-s.sigma * len);
    }
    return n;
}

/* Render chosen pixels only: vpx holds n triples (view, px, py). */
int64_t orc_render_pixels(const orc_grid *g, const double *vol, const orc_cam *cams,
                          const orc_params *P, int64_t n, const int32_t *vpx, double *out)
{
    orc_field F = {ORC_RGB, vol, NULL};
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i)
        total += render_pixel(g, &F, cams + vpx[3 * i], P, vpx[3 * i + 1], vpx[3 * i + 2],
                              out + 3 * i, NULL);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Pre-processing and residual (Sec. 4.1, Sec. 3.3.2 colour constraint,      */
/* Sec. 5.1 error measure)                                                    */
/* ------------------------------------------------------------------------ */

/* Pixels whose largest channel exceeds the threshold are flame pixels; the
 * others are set to black.  bbox (per view): x0, y0, x1, y1 inclusive, the
 * tight box of the flame pixels; an empty view gets x0 > x1. */
void orc_prepare_targets(int ncam, int height, int width, double *targets,
                         double thresh, uint8_t *mask, int32_t *bbox)
{
    for (int v = 0; v < ncam; ++v) {
        int32_t *bb = bbox + 4 * v;
        bb[0] = width; bb[1] = height; bb[2] = -1; bb[3] = -1;
        for (int py = 0; py < height; ++py)
            for (int px = 0; px < width; ++px) {
                int64_t pix = ((int64_t)v * height + py) * width + px;
                double *t = targets + 3 * pix;
                double mx = t[0];
                if (t[1] > mx) mx = t[1];
                if (t[2] > mx) mx = t[2];
                int flame = mx > thresh;
                mask[pix] = (uint8_t)flame;
                if (!flame) {
                    t[0] = t[1] = t[2] = 0.0;
                    continue;
                }
                if (px < bb[0]) bb[0] = px;
                if (py < bb[1]) bb[1] = py;
                if (px > bb[2]) bb[2] = px;
                if (py > bb[3]) bb[3] = py;
            }
    }
}

/* residual = target - rendered for every pixel; rmse3 = 255 * RMS of the
 * residual over the union of the per-view boxes, per channel. */
void orc_residual(int ncam, int height, int width, const double *rendered,
                  const double *targets, const int32_t *bbox, double *residual,
                  double *rmse3)
{
    double acc[3] = {0.0, 0.0, 0.0};
    int64_t count = 0;
    for (int v = 0; v < ncam; ++v) {
        const int32_t *bb = bbox + 4 * v;
        for (int py = 0; py < height; ++py)
            for (int px = 0; px < width; ++px) {
                int64_t pix = ((int64_t)v * height + py) * width + px;
                int in_box = px >= bb[0] && px <= bb[2] && py >= bb[1] && py <= bb[3];
                for (int ch = 0; ch < 3; ++ch) {
                    double r = targets[3 * pix + ch] - rendered[3 * pix + ch];
                    residual[3 * pix + ch] = r;
                    if (in_box) acc[ch] += r * r;
                }
                count += in_box;
            }
    }
    for (int ch = 0; ch < 3; ++ch)
        rmse3[ch] = count ? 255.0 * sqrt(acc[ch] / (double)count) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Volume adjustment, paper rule (Eqs. 10-12; Algorithm 2, adjustment half)  */
/* ------------------------------------------------------------------------ */

/* For every flame pixel, every sample on its ray and each of the sample's
 * eight key points j:
 *     dV_j += G(s) * alpha_l * dL * T(s, s_e) * exp(-alpha_d * D(j, s)),
 * where T(s, s_e) is the transmittance between the eye and the sample (Eq. 12
 * in constant-tau mode, exp(-sum of preceding optical depths) in field mode)
 * and D the Euclidean key-point distance in voxel edge lengths.  All views
 * accumulate into one dV (N^3 x 3).  Returns the number of samples visited.
 *
 * Which eight key points a sample has is an integer decision (its cell), and
 * so is the number of samples on a ray (ceil(chord / step)): an evaluation in
 * another precision may take either when the sample lies within its rounding
 * error of a cell face, or chord / step within it of an integer.  undecided
 * (nullable, one value per node) then receives, for each such sample, its
 * largest possible contribution G alpha_l T max_c |dL_c| (exp(-alpha_d D) <= 1)
 * at every node of the cells it may belong to: a bound on how much that
 * decision can move the node's sum.  The margins are set by
 * orc_set_undecided_margins. */
static double g_face_eps = 2e-4;    /* voxels */
static double g_count_eps = 1e-3;   /* segments */

void orc_set_undecided_margins(double face_voxels, double count_segments)
{
    g_face_eps = face_voxels;
    g_count_eps = count_segments;
}

/* w added to every node of the cells [c + lo, c + hi] (clamped to the grid). */
static void add_to_cells(const orc_grid *g, const int c[3], const int lo[3], const int hi[3], double w,
                         double *und)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    int a0[3], a1[3];
    for (int a = 0; a < 3; ++a) {
        a0[a] = c[a] + lo[a] < 0 ? 0 : c[a] + lo[a];
        a1[a] = c[a] + hi[a] + 1 > n[a] - 1 ? n[a] - 1 : c[a] + hi[a] + 1;
    }
    for (int k = a0[2]; k <= a1[2]; ++k)
        for (int j = a0[1]; j <= a1[1]; ++j)
            for (int i = a0[0]; i <= a1[0]; ++i) und[node_index(g, i, j, k)] += w;
}

static int64_t update_paper_views(const orc_grid *g, const double *vol, const orc_cam *cams,
                                  int ncam, const orc_params *P, const double *residual,
                                  const uint8_t *mask, int iteration, int view_base, double *dV,
                                  double *undecided);

int64_t orc_update_paper(const orc_grid *g, const double *vol, const orc_cam *cams,
                         int ncam, const orc_params *P, const double *residual,
                         const uint8_t *mask, int iteration, double *dV, double *undecided)
{
    return update_paper_views(g, vol, cams, ncam, P, residual, mask, iteration, 0, dV, undecided);
}

/* The views of cams are views view_base, view_base + 1, ... of the problem:
 * their index keys the G(s) stream. */
static int64_t update_paper_views(const orc_grid *g, const double *vol, const orc_cam *cams,
                                  int ncam, const orc_params *P, const double *residual,
                                  const uint8_t *mask, int iteration, int view_base, double *dV,
                                  double *undecided)
{
    orc_field F = {ORC_RGB, vol, NULL};
    const int n_ax[3] = {g->nx, g->ny, g->nz};
    const int64_t nodes = (int64_t)g->nx * g->ny * g->nz;
    /* one accumulator per thread (the first is dV itself), added in thread
     * order at the end; the same for the undecided budget */
    int nt = orc_threads();
    double **acc = malloc(sizeof(double *) * (size_t)nt);
    double **und = malloc(sizeof(double *) * (size_t)nt);
    acc[0] = dV;
    und[0] = undecided;
    for (int t = 1; t < nt; ++t) {
        acc[t] = calloc((size_t)(3 * nodes), sizeof(double));
        und[t] = undecided ? calloc((size_t)nodes, sizeof(double)) : NULL;
        if (!acc[t] || (undecided && !und[t])) {   /* out of memory: the work runs on fewer threads */
            free(acc[t]);
            free(und[t]);
            nt = t;
            break;
        }
    }
    int64_t total = 0, off = 0;
    for (int v = 0; v < ncam; ++v) {
        const orc_cam *c = cams + v;
        int64_t view_total = 0;
#pragma omp parallel for num_threads(nt) schedule(static, 1) reduction(+ : view_total)
        for (int py = 0; py < c->height; ++py) {
            double *dst = acc[ORC_THREAD()];
            double *ust = und[ORC_THREAD()];
            for (int px = 0; px < c->width; ++px) {
                int64_t pix = off + (int64_t)py * c->width + px;
                if (!mask[pix]) continue;
                const double *dL = residual + 3 * pix;
                double dl_max = fabs(dL[0]);
                if (fabs(dL[1]) > dl_max) dl_max = fabs(dL[1]);
                if (fabs(dL[2]) > dl_max) dl_max = fabs(dL[2]);
                double o[3], d[3], t0, t1;
                camera_ray(g, c, px, py, o, d);
                if (!clip_ray(g, o, d, &t0, &t1)) continue;
                int64_t n = segment_count(t0, t1, P->step);
                view_total += n;
                double T = 1.0, T_last = 1.0;
                for (int64_t k = 0; k < n; ++k) {
                    double len, p[3];
                    orc_sample s;
                    segment(o, d, t0, t1, P->step, k, &len, p);
                    sample_field(g, &F, p, &s);
                    double G = orc_g_draw(P->seed, P->g_std, iteration, view_base + v,
                                          (int64_t)py * c->width + px, k);
                    for (int b = 0; b < 8; ++b) {
                        int64_t j = s.idx[b];
                        int64_t ji = j % g->nx, jj = (j / g->nx) % g->ny, jk = j / ((int64_t)g->nx * g->ny);
                        double dx = p[0] - (double)ji, dy = p[1] - (double)jj, dz = p[2] - (double)jk;
                        double D = sqrt(dx * dx + dy * dy + dz * dz);
                        double a = G * P->alpha_l * T * exp(-P->alpha_d * D);
                        for (int ch = 0; ch < 3; ++ch) dst[3 * j + ch] += a * dL[ch];
                    }
                    if (ust) {
                        /* a sample within the margin of a face may belong to the cell beyond it */
                        int cc[3], lo[3], hi[3], near = 0;
                        double f[3];
                        locate(g, p, cc, f);
                        for (int a = 0; a < 3; ++a) {
                            lo[a] = f[a] < g_face_eps && cc[a] > 0 ? -1 : 0;
                            hi[a] = f[a] > 1.0 - g_face_eps && cc[a] < n_ax[a] - 2 ? 1 : 0;
                            near |= lo[a] | hi[a];
                        }
                        if (near) add_to_cells(g, cc, lo, hi, fabs(G) * P->alpha_l * T * dl_max, ust);
                    }
                    T_last = T;
                    if (P->tau > 0.0)
                        T *= 1.0 - P->tau;
                    else
                        T *= exp(-s.sigma * len);
                }
                if (ust) {
                    /* chord / step within the margin of an integer m: a sample at the
                     * exit point (index m, a segment of almost no length) may be
                     * added or dropped */
                    const double x = (t1 - t0) / P->step, m = nearbyint(x);
                    if (fabs(x - m) < g_count_eps && m >= 1.0) {
                        double pe[3], f[3];
                        int cc[3];
                        const int lo[3] = {-1, -1, -1}, hi[3] = {1, 1, 1};
                        for (int a = 0; a < 3; ++a) pe[a] = o[a] + t1 * d[a];
                        locate(g, pe, cc, f);
                        const double G = orc_g_draw(P->seed, P->g_std, iteration, view_base + v,
                                                    (int64_t)py * c->width + px, (int64_t)m);
                        add_to_cells(g, cc, lo, hi, fabs(G) * P->alpha_l * T_last * dl_max, ust);
                    }
                }
            }
        }
        total += view_total;
        off += (int64_t)c->width * c->height;
    }
    for (int t = 1; t < nt; ++t) {
        for (int64_t i = 0; i < 3 * nodes; ++i) dV[i] += acc[t][i];
        if (undecided)
            for (int64_t i = 0; i < nodes; ++i) undecided[i] += und[t][i];
        free(acc[t]);
        free(und[t]);
    }
    free(acc);
    free(und);
    return total;
}

/* V_{k+1} = V_k + dV on the three colour components (Eq. 11). */
void orc_apply_update(int64_t nodes, double *vol, const double *dV, int clamp_nonneg)
{
    for (int64_t j = 0; j < nodes; ++j)
        for (int ch = 0; ch < 3; ++ch) {
            double x = vol[4 * j + ch] + dV[3 * j + ch];
            if (clamp_nonneg && x < 0.0) x = 0.0;
            vol[4 * j + ch] = x;
        }
}

/* ------------------------------------------------------------------------ */
/* Exact gradient of the rendered images (the differentiable variant)        */
/* ------------------------------------------------------------------------ */

/* Given gimg = d(loss)/d(rendered pixel) and the rendered radiance L_total of
 * each pixel, accumulate d(loss)/d(node value) into grad (N^3 x 4 for RGB
 * records {S_r,S_g,S_b,sigma}, N^3 x 2 for temperature records {T, sigma}).
 * Along a ray with samples k, L = sum_k T_k c_k with c_k = S_k beta_k and
 * T_{k+1} = T_k exp(-sigma_k l_k), so
 *   dL/dS_k     = T_k beta_k,
 *   dL/dsigma_k = T_k S_k dbeta_k/dsigma - l_k (L - sum_{m<=k} T_m c_m).
 * In constant-tau mode dL/dV_k = T_k tau and sigma does not enter. */
static void grad_views(const orc_grid *g, const orc_field *F, const orc_cam *cams,
                       int ncam, const orc_params *P, const double *L_total,
                       const double *gimg, double *grad)
{
    int rec = F->kind == ORC_RGB ? 4 : 2;
    int64_t off = 0;
    for (int v = 0; v < ncam; ++v) {
        const orc_cam *c = cams + v;
        for (int py = 0; py < c->height; ++py)
            for (int px = 0; px < c->width; ++px) {
                int64_t pix = off + (int64_t)py * c->width + px;
                const double *gp = gimg + 3 * pix, *Lt = L_total + 3 * pix;
                if (gp[0] == 0.0 && gp[1] == 0.0 && gp[2] == 0.0) continue;
                double o[3], d[3], t0, t1;
                camera_ray(g, c, px, py, o, d);
                if (!clip_ray(g, o, d, &t0, &t1)) continue;
                int64_t n = segment_count(t0, t1, P->step);
                double T = 1.0, prefix[3] = {0.0, 0.0, 0.0};
                for (int64_t k = 0; k < n; ++k) {
                    double len, p[3];
                    orc_sample s;
                    segment(o, d, t0, t1, P->step, k, &len, p);
                    sample_field(g, F, p, &s);
                    double gS[3], gsig = 0.0;
                    if (P->tau > 0.0) {
                        for (int ch = 0; ch < 3; ++ch) gS[ch] = gp[ch] * T * P->tau;
                        T *= 1.0 - P->tau;
                    } else {
                        double beta, dbeta;
                        segment_weight(s.sigma, len, &beta, &dbeta);
                        for (int ch = 0; ch < 3; ++ch) {
                            double ck = s.S[ch] * beta;
                            prefix[ch] += T * ck;
                            gS[ch] = gp[ch] * T * beta;
                            gsig += gp[ch] * (T * s.S[ch] * dbeta - len * (Lt[ch] - prefix[ch]));
                        }
                        T *= exp(-s.sigma * len);
                    }
                    if (F->kind == ORC_RGB) {
                        for (int b = 0; b < 8; ++b) {
                            double *gr = grad + 4 * s.idx[b];
                            for (int ch = 0; ch < 3; ++ch) gr[ch] += s.w[b] * gS[ch];
                            gr[3] += s.w[b] * gsig;
                        }
                    } else {
                        double gT = gS[0] * s.dS_dT[0] + gS[1] * s.dS_dT[1] + gS[2] * s.dS_dT[2];
                        for (int b = 0; b < 8; ++b) {
                            double *gr = grad + 2 * s.idx[b];
                            gr[0] += s.w[b] * gT;
                            gr[1] += s.w[b] * gsig;
                        }
                    }
                }
            }
        off += (int64_t)c->width * c->height;
        (void)rec;
    }
}

void orc_grad(const orc_grid *g, const double *vol, const orc_cam *cams, int ncam,
              const orc_params *P, const double *L_total, const double *gimg, double *grad)
{
    orc_field F = {ORC_RGB, vol, NULL};
    grad_views(g, &F, cams, ncam, P, L_total, gimg, grad);
}

void orc_grad_temp(const orc_grid *g, const double *vol_ts, const orc_lut *lut,
                   const orc_cam *cams, int ncam, const orc_params *P,
                   const double *L_total, const double *gimg, double *grad)
{
    orc_field F = {ORC_TEMP, vol_ts, lut};
    grad_views(g, &F, cams, ncam, P, L_total, gimg, grad);
}

/* ------------------------------------------------------------------------ */
/* In-scattering (Eq. 5, third term; isotropic phase, Eq. 9 with g = 0)      */
/* ------------------------------------------------------------------------ */

/* Mean incident radiance J at every node, estimated from the six axis
 * directions: J = (1/6) sum_d L_d, where L_d is the emitted radiance arriving
 * at the node along grid lines travelling in direction d.  Along a line,
 *   L(node i) = L(node i-1) exp(-s) + q (1 - exp(-s)) / s,
 * with s and q the averages of the two end nodes (the midpoint sample of the
 * unit-length segment between them) and L = 0 at the first node.  This is
 * single scattering of the emitted light.  vol: N^3 x 4 records holding the
 * emission q (RGB) and sigma; J: N^3 x 3. */
void orc_scatter_J(const orc_grid *g, const double *vol, double *J)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    int64_t nodes = (int64_t)n[0] * n[1] * n[2];
    memset(J, 0, sizeof(double) * 3 * (size_t)nodes);
    for (int axis = 0; axis < 3; ++axis) {
        int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
        for (int u = 0; u < n[a1]; ++u)
            for (int w = 0; w < n[a2]; ++w)
                for (int dir = 0; dir < 2; ++dir) {
                    double L[3] = {0.0, 0.0, 0.0};
                    int64_t prev = -1;
                    for (int s = 0; s < n[axis]; ++s) {
                        int pos = dir == 0 ? s : n[axis] - 1 - s;
                        int ijk[3];
                        ijk[axis] = pos; ijk[a1] = u; ijk[a2] = w;
                        int64_t j = node_index(g, ijk[0], ijk[1], ijk[2]);
                        if (prev >= 0) {
                            const double *r0 = vol + 4 * prev, *r1 = vol + 4 * j;
                            double sig = 0.5 * (r0[3] + r1[3]);
                            double beta, dbeta;
                            segment_weight(sig, 1.0, &beta, &dbeta);
                            double att = exp(-sig);
                            for (int ch = 0; ch < 3; ++ch)
                                L[ch] = L[ch] * att + 0.5 * (r0[ch] + r1[ch]) * beta;
                        }
                        for (int ch = 0; ch < 3; ++ch) J[3 * j + ch] += L[ch] / 6.0;
                        prev = j;
                    }
                }
    }
}

/* Source records for rendering with in-scattering (Eq. 5):
 * S = q + albedo * sigma * J, sigma unchanged.  out may alias nothing. */
void orc_scatter_source(int64_t nodes, const double *vol, const double *albedo,
                        const double *J, double *out)
{
    for (int64_t j = 0; j < nodes; ++j) {
        double s = vol[4 * j + 3];
        for (int ch = 0; ch < 3; ++ch)
            out[4 * j + ch] = vol[4 * j + ch] + albedo[j] * s * J[3 * j + ch];
        out[4 * j + 3] = s;
    }
}

/* The six directional radiances of orc_scatter_J kept apart: L6 (N^3 x 6 x 3)
 * holds, for propagation direction d = 2 axis + dir (dir 0: towards +axis,
 * 1: towards -axis), the radiance arriving at each node along the grid line
 * (same recurrence, L = 0 at the line's first node). */
void orc_scatter_L6(const orc_grid *g, const double *vol, double *L6)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    int64_t nodes = (int64_t)n[0] * n[1] * n[2];
    memset(L6, 0, sizeof(double) * 18 * (size_t)nodes);
    for (int axis = 0; axis < 3; ++axis) {
        int a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
        for (int u = 0; u < n[a1]; ++u)
            for (int w = 0; w < n[a2]; ++w)
                for (int dir = 0; dir < 2; ++dir) {
                    double L[3] = {0.0, 0.0, 0.0};
                    int64_t prev = -1;
                    for (int s = 0; s < n[axis]; ++s) {
                        int pos = dir == 0 ? s : n[axis] - 1 - s;
                        int ijk[3];
                        ijk[axis] = pos; ijk[a1] = u; ijk[a2] = w;
                        int64_t j = node_index(g, ijk[0], ijk[1], ijk[2]);
                        if (prev >= 0) {
                            const double *r0 = vol + 4 * prev, *r1 = vol + 4 * j;
                            double sig = 0.5 * (r0[3] + r1[3]);
                            double beta, dbeta;
                            segment_weight(sig, 1.0, &beta, &dbeta);
                            double att = exp(-sig);
                            for (int ch = 0; ch < 3; ++ch)
                                L[ch] = L[ch] * att + 0.5 * (r0[ch] + r1[ch]) * beta;
                        }
                        for (int ch = 0; ch < 3; ++ch) L6[18 * j + 3 * (2 * axis + dir) + ch] = L[ch];
                        prev = j;
                    }
                }
    }
}

/* Weights of the six directional radiances in the light scattered towards
 * unit direction omega (Eq. 9): light propagating along direction d arrives
 * from omega_i = -e_d, so w_d is proportional to p(omega, -e_d); the six
 * weights are normalised to sum to 1 (each direction stands for a sixth of the
 * sphere).  g = 0 gives 1/6 each. */
void orc_hg_weights(double g, const double omega[3], double w[6])
{
    double sum = 0.0;
    for (int d = 0; d < 6; ++d) {
        const int axis = d / 2;
        const double sign = (d & 1) ? -1.0 : 1.0;   /* e_d along +axis for dir 0 */
        const double cos_wi = -sign * omega[axis];  /* omega . (-e_d) */
        w[d] = orc_hg_phase(g, cos_wi);
        sum += w[d];
    }
    for (int d = 0; d < 6; ++d) w[d] /= sum;
}

/* Source records towards one view: S = q + albedo sigma sum_d w_d L_d. */
void orc_scatter_source_hg(int64_t nodes, const double *vol, const double *albedo, const double *L6,
                           const double w[6], double *out)
{
    for (int64_t j = 0; j < nodes; ++j) {
        double s = vol[4 * j + 3];
        for (int ch = 0; ch < 3; ++ch) {
            double in = 0.0;
            for (int d = 0; d < 6; ++d) in += w[d] * L6[18 * j + 3 * d + ch];
            out[4 * j + ch] = vol[4 * j + ch] + albedo[j] * s * in;
        }
        out[4 * j + 3] = s;
    }
}

/* Unit direction from the volume's centre to camera c, in world axes (the
 * grid's axes): the direction towards which view c sees scattered light. */
static void view_direction(const orc_grid *g, const orc_cam *c, double omega[3])
{
    double d[3], len = 0.0;
    const int n[3] = {g->nx, g->ny, g->nz};
    for (int a = 0; a < 3; ++a) {
        d[a] = c->pos[a] - (g->origin[a] + 0.5 * (double)(n[a] - 1) * g->h);
        len += d[a] * d[a];
    }
    len = sqrt(len);
    for (int a = 0; a < 3; ++a) omega[a] = d[a] / len;
}

/* ------------------------------------------------------------------------ */
/* Visual hull (Sec. 4.3.1, Algorithm 1)                                     */
/* ------------------------------------------------------------------------ */

/* Algorithm 1 tags the key points near every flame ray of view v with bit
 * v; a key point is inside the hull when all K bits are set.  Reading: key
 * point j is near a flame ray of view v when the centre of a flame pixel
 * lies in the image rectangle that bounds the projection of the box of the
 * eight cells sharing j ([j-1, j+1] per axis, clipped to the volume) -- every
 * ray that can sample one of those cells passes through that rectangle, so
 * the tags are conservative.  The corners are projected in double precision:
 *   u = (x_c / z_c / t_x + 1) W / 2 - 1/2,  t_x = tan_half W / H,
 *   v = (1 - y_c / z_c / t_y) H / 2 - 1/2,  t_y = tan_half,
 * (x_c, y_c, z_c) the corner relative to the camera along right, up, fwd, in
 * voxel units; the pixel centres inside are columns ceil(u_min)..floor(u_max)
 * and rows ceil(v_min)..floor(v_max), clipped to the image; a corner with
 * z_c <= 0 (beside or behind the camera) makes it the whole image.
 *
 * Whether a pixel centre lies in the rectangle is an integer decision, which
 * an evaluation in another precision may take differently when a rectangle
 * edge lies within its rounding error of a pixel centre.  amb (nullable)
 * receives, per node, the views whose bit changes when every edge of the
 * rectangle moves in or out by eps pixels, or when a corner lies within eps_z
 * voxels of the camera plane: the decisions that are not fixed to that
 * margin. */

/* 1 when a flame pixel of view v has its centre in [u0, u1] x [w0, w1]. */
static int flame_in_rect(const uint8_t *mask, const orc_cam *c, int v, double u0, double u1,
                         double w0, double w1)
{
    double x0 = ceil(u0), x1 = floor(u1), y0 = ceil(w0), y1 = floor(w1);
    if (x0 < 0.0) x0 = 0.0;
    if (y0 < 0.0) y0 = 0.0;
    if (x1 > (double)(c->width - 1)) x1 = (double)(c->width - 1);
    if (y1 > (double)(c->height - 1)) y1 = (double)(c->height - 1);
    if (!(x0 <= x1) || !(y0 <= y1)) return 0;
    for (int py = (int)y0; py <= (int)y1; ++py)
        for (int px = (int)x0; px <= (int)x1; ++px)
            if (mask[((int64_t)v * c->height + py) * c->width + px]) return 1;
    return 0;
}

void orc_visual_hull(const orc_grid *g, const orc_cam *cams, int ncam, const uint8_t *mask,
                     uint32_t *tags, uint32_t *amb, double eps, double eps_z)
{
    const int n[3] = {g->nx, g->ny, g->nz};
#pragma omp parallel for num_threads(g_threads) schedule(static, 1)
    for (int k = 0; k < n[2]; ++k)
        for (int j = 0; j < n[1]; ++j)
            for (int i = 0; i < n[0]; ++i) {
                uint32_t tag = 0, unsure = 0;
                const int lo[3] = {i > 0 ? i - 1 : 0, j > 0 ? j - 1 : 0, k > 0 ? k - 1 : 0};
                const int hi[3] = {i < n[0] - 1 ? i + 1 : n[0] - 1, j < n[1] - 1 ? j + 1 : n[1] - 1,
                                   k < n[2] - 1 ? k + 1 : n[2] - 1};
                for (int v = 0; v < ncam; ++v) {
                    const orc_cam *c = cams + v;
                    const double ty = c->tan_half_fov;
                    const double tx = ty * (double)c->width / (double)c->height;
                    double umin = INFINITY, umax = -INFINITY, wmin = INFINITY, wmax = -INFINITY;
                    int behind = 0, near_plane = 0;
                    for (int b = 0; b < 8; ++b) {
                        const int corner[3] = {(b & 1) ? hi[0] : lo[0], (b & 2) ? hi[1] : lo[1],
                                               (b & 4) ? hi[2] : lo[2]};
                        double xc = 0.0, yc = 0.0, zc = 0.0;
                        for (int a = 0; a < 3; ++a) {
                            const double X = (double)corner[a] - (c->pos[a] - g->origin[a]) / g->h;
                            xc += X * c->right[a];
                            yc += X * c->up[a];
                            zc += X * c->fwd[a];
                        }
                        if (fabs(zc) <= eps_z) near_plane = 1;
                        if (!(zc > 0.0)) {
                            behind = 1;
                            continue;
                        }
                        const double u = (xc / zc / tx + 1.0) * 0.5 * (double)c->width - 0.5;
                        const double w = (1.0 - yc / zc / ty) * 0.5 * (double)c->height - 0.5;
                        if (u < umin) umin = u;
                        if (u > umax) umax = u;
                        if (w < wmin) wmin = w;
                        if (w > wmax) wmax = w;
                    }
                    int hit, shrunk, grown;
                    if (behind) {
                        hit = shrunk = grown = flame_in_rect(mask, c, v, -INFINITY, INFINITY, -INFINITY, INFINITY);
                    } else {
                        hit = flame_in_rect(mask, c, v, umin, umax, wmin, wmax);
                        shrunk = flame_in_rect(mask, c, v, umin + eps, umax - eps, wmin + eps, wmax - eps);
                        grown = flame_in_rect(mask, c, v, umin - eps, umax + eps, wmin - eps, wmax + eps);
                    }
                    if (hit) tag |= 1u << v;
                    if (shrunk != grown || near_plane) unsure |= 1u << v;
                }
                tags[node_index(g, i, j, k)] = tag;
                if (amb) amb[node_index(g, i, j, k)] = unsure;
            }
}

/* Volume dimensions (Sec. 4.2): project the 8 corners of the world box
 * [lo, lo + len] into every image; for each of the 12 edges (along axis d) the
 * pixels it spans are the larger of |du| and |dv|; n_d is the largest over
 * edges and images; the voxel edge along d is alpha len_d / n_d.  Reading for
 * cubic voxels: h = the smallest of the three, dims_d = ceil(len_d / h) + 1
 * nodes.  Returns 0, or -1 when a corner is not in front of a camera. */
int orc_volume_dims(const orc_cam *cams, int ncam, const double lo[3], const double len[3], double alpha,
                    int dims[3], double *h, double nmax[3])
{
    for (int d = 0; d < 3; ++d) nmax[d] = 0.0;
    for (int v = 0; v < ncam; ++v) {
        const orc_cam *c = cams + v;
        const double ty = c->tan_half_fov, tx = ty * (double)c->width / (double)c->height;
        double u[8], w[8];
        for (int b = 0; b < 8; ++b) {
            double rel[3];
            for (int d = 0; d < 3; ++d) rel[d] = lo[d] + (((b >> d) & 1) ? len[d] : 0.0) - c->pos[d];
            const double xc = rel[0] * c->right[0] + rel[1] * c->right[1] + rel[2] * c->right[2];
            const double yc = rel[0] * c->up[0] + rel[1] * c->up[1] + rel[2] * c->up[2];
            const double zc = rel[0] * c->fwd[0] + rel[1] * c->fwd[1] + rel[2] * c->fwd[2];
            if (!(zc > 0.0)) return -1;
            u[b] = (xc / zc / tx + 1.0) * 0.5 * c->width - 0.5;
            w[b] = (1.0 - yc / zc / ty) * 0.5 * c->height - 0.5;
        }
        for (int b = 0; b < 8; ++b)
            for (int d = 0; d < 3; ++d) {
                if ((b >> d) & 1) continue;
                const int e = b | (1 << d);
                double span = fabs(u[e] - u[b]);
                if (fabs(w[e] - w[b]) > span) span = fabs(w[e] - w[b]);
                if (span > nmax[d]) nmax[d] = span;
            }
    }
    double best = INFINITY;
    for (int d = 0; d < 3; ++d) {
        if (!(nmax[d] > 0.0)) return -1;
        const double e = alpha * len[d] / nmax[d];
        if (e < best) best = e;
    }
    *h = best;
    for (int d = 0; d < 3; ++d) dims[d] = (int)ceil(len[d] / best - 1e-9) + 1;
    return 0;
}

/* Volume data error (Sec. 5.1): per colour channel, the root mean square of
 * the difference between two volumes' emission over the key points inside the
 * visual hull (tags == full; every key point when tags is NULL), in the
 * volumes' own units.  Returns the number of key points compared (rmse3 = 0
 * when there are none). */
int64_t orc_volume_rmse(int64_t nodes, const double *a, const double *b, const uint32_t *tags,
                        uint32_t full, double *rmse3)
{
    double acc[3] = {0.0, 0.0, 0.0};
    int64_t count = 0;
    for (int64_t j = 0; j < nodes; ++j) {
        if (tags && tags[j] != full) continue;
        for (int ch = 0; ch < 3; ++ch) {
            const double d = a[4 * j + ch] - b[4 * j + ch];
            acc[ch] += d * d;
        }
        ++count;
    }
    for (int ch = 0; ch < 3; ++ch) rmse3[ch] = count ? sqrt(acc[ch] / (double)count) : 0.0;
    return count;
}

/* ------------------------------------------------------------------------ */
/* The iteration (Sec. 3, Algorithm 2): render, compare, adjust.             */
/* ------------------------------------------------------------------------ */

/* Squared residual sums of one view inside its flame box: residual =
 * target - rendered everywhere, acc[0..2] += the squares in the box, returns
 * the number of box pixels (Sec. 5.1). */
static int64_t view_residual(int height, int width, const double *rendered, const double *targets,
                             const int32_t *bb, double *residual, double acc[3])
{
    int64_t count = 0;
    for (int py = 0; py < height; ++py)
        for (int px = 0; px < width; ++px) {
            int64_t pix = (int64_t)py * width + px;
            int in_box = px >= bb[0] && px <= bb[2] && py >= bb[1] && py <= bb[3];
            for (int ch = 0; ch < 3; ++ch) {
                double r = targets[3 * pix + ch] - rendered[3 * pix + ch];
                residual[3 * pix + ch] = r;
                if (in_box) acc[ch] += r * r;
            }
            count += in_box;
        }
    return count;
}

/* Runs `iters` iterations of the paper rule on vol (N^3 x 4, colour updated
 * in place); with stop_delta >= 0, stops earlier after the first iteration
 * k >= 1 whose image error differs from iteration k-1's by less than
 * stop_delta in every channel (Sec. 3 stop criterion), and *iters_done
 * (nullable) gets the iterations run.  albedo (nullable) turns on the
 * in-scattering source, recomputed from the current volume at the start of
 * each iteration.  targets must have been through orc_prepare_targets (mask,
 * bbox).  rmse (iters x 3) gets the error of the images rendered in each
 * iteration.  samples[0..1] accumulate forward and adjustment sample counts.
 * undecided (nullable, one value per node) accumulates over the iterations
 * the adjustment's undecided budget (see update_paper_views).
 * P->storage != 0 keeps the records in a 16-bit type: the volume is rounded
 * to it on entry and after every update, the in-scattering source each time it
 * is formed (orc_round_storage).
 *
 * Variants the paper mentions without using (Sec. 3.3.1, Eq. 9; Sec. 3.3.2):
 * P->hg_g != 0 scatters with the Henyey-Greenstein phase function: each view
 * renders its own source, with the six directional radiances weighted
 * towards the direction from the volume's centre to its camera;
 * P->sequential = 1 updates the volume after each view in turn (Kaczmarz
 * order), the source recomputed from the current volume before each view.
 * Either way the views are rendered and adjusted one at a time and the
 * iteration's error pools every view's box. */
void orc_reconstruct(const orc_grid *g, double *vol, const double *albedo,
                     const orc_cam *cams, int ncam, const orc_params *P,
                     const double *targets, const uint8_t *mask, const int32_t *bbox,
                     int iters, int first_iteration, double *rmse, int64_t *samples,
                     const uint32_t *hull, double stop_delta, int *iters_done, double *undecided)
{
    int64_t nodes = (int64_t)g->nx * g->ny * g->nz;
    int64_t npix = 0;
    for (int v = 0; v < ncam; ++v) npix += (int64_t)cams[v].width * cams[v].height;
    const int per_view = P->hg_g != 0.0 || P->sequential;
    double *img = malloc(sizeof(double) * 3 * (size_t)npix);
    double *res = malloc(sizeof(double) * 3 * (size_t)npix);
    double *dV = malloc(sizeof(double) * 3 * (size_t)nodes);
    double *J = albedo ? malloc(sizeof(double) * 18 * (size_t)nodes) : NULL;   /* J or L6 */
    double *src = albedo ? malloc(sizeof(double) * 4 * (size_t)nodes) : NULL;
    /* key points outside the visual hull are not reconstructed: they hold no
     * flame, so their whole record (emission and extinction) is 0 and stays 0
     * (Sec. 4.3.1 marks them with a non-flame value, slightly below zero;
     * 0 here, which leaves the rays through them unchanged) */
    const uint32_t full = ncam >= 32 ? 0xffffffffu : ((1u << ncam) - 1u);
    if (hull)
        for (int64_t j = 0; j < nodes; ++j)
            if (hull[j] != full) vol[4 * j] = vol[4 * j + 1] = vol[4 * j + 2] = vol[4 * j + 3] = 0.0;
    /* a volume in 16-bit storage holds only values of that type: the records
     * the loop keeps (the volume after each update and the source records it
     * renders) are rounded to it */
    orc_round_storage(4 * nodes, vol, P->storage);
    for (int it = 0; it < iters; ++it) {
        if (!per_view) {
            const double *rvol = vol;
            if (albedo) {
                orc_scatter_J(g, vol, J);
                orc_scatter_source(nodes, vol, albedo, J, src);
                orc_round_storage(4 * nodes, src, P->storage);
                rvol = src;
            }
            samples[0] += orc_render(g, rvol, cams, ncam, P, img, NULL);
            orc_residual(ncam, cams[0].height, cams[0].width, img, targets, bbox, res, rmse + 3 * it);
            memset(dV, 0, sizeof(double) * 3 * (size_t)nodes);
            samples[1] += orc_update_paper(g, rvol, cams, ncam, P, res, mask, first_iteration + it, dV, undecided);
            orc_apply_update(nodes, vol, dV, P->clamp_nonneg);
            orc_round_storage(4 * nodes, vol, P->storage);
            if (hull)
                for (int64_t j = 0; j < nodes; ++j)
                    if (hull[j] != full) vol[4 * j] = vol[4 * j + 1] = vol[4 * j + 2] = vol[4 * j + 3] = 0.0;
        } else {
            double acc[3] = {0.0, 0.0, 0.0};
            int64_t count = 0, off = 0;
            memset(dV, 0, sizeof(double) * 3 * (size_t)nodes);
            for (int v = 0; v < ncam; ++v) {
                const orc_cam *c = cams + v;
                const double *rvol = vol;
                if (albedo) {
                    if (P->hg_g != 0.0) {
                        if (v == 0 || P->sequential) orc_scatter_L6(g, vol, J);
                        double omega[3], w[6];
                        view_direction(g, c, omega);
                        orc_hg_weights(P->hg_g, omega, w);
                        orc_scatter_source_hg(nodes, vol, albedo, J, w, src);
                        orc_round_storage(4 * nodes, src, P->storage);
                    } else if (v == 0 || P->sequential) {
                        orc_scatter_J(g, vol, J);
                        orc_scatter_source(nodes, vol, albedo, J, src);
                        orc_round_storage(4 * nodes, src, P->storage);
                    }
                    rvol = src;
                }
                samples[0] += orc_render(g, rvol, c, 1, P, img + 3 * off, NULL);
                count += view_residual(c->height, c->width, img + 3 * off, targets + 3 * off, bbox + 4 * v,
                                       res + 3 * off, acc);
                samples[1] += update_paper_views(g, rvol, c, 1, P, res + 3 * off, mask + off,
                                                 first_iteration + it, v, dV, undecided);
                if (P->sequential) {
                    orc_apply_update(nodes, vol, dV, P->clamp_nonneg);
                    orc_round_storage(4 * nodes, vol, P->storage);
                    memset(dV, 0, sizeof(double) * 3 * (size_t)nodes);
                    if (hull)
                        for (int64_t j = 0; j < nodes; ++j)
                            if (hull[j] != full) vol[4 * j] = vol[4 * j + 1] = vol[4 * j + 2] = vol[4 * j + 3] = 0.0;
                }
                off += (int64_t)c->width * c->height;
            }
            if (!P->sequential) {
                orc_apply_update(nodes, vol, dV, P->clamp_nonneg);
                orc_round_storage(4 * nodes, vol, P->storage);
                if (hull)
                    for (int64_t j = 0; j < nodes; ++j)
                        if (hull[j] != full) vol[4 * j] = vol[4 * j + 1] = vol[4 * j + 2] = vol[4 * j + 3] = 0.0;
            }
            for (int ch = 0; ch < 3; ++ch) rmse[3 * it + ch] = count ? 255.0 * sqrt(acc[ch] / (double)count) : 0.0;
        }
        if (iters_done) *iters_done = it + 1;
        if (stop_delta >= 0.0 && it >= 1) {
            int small = 1;
            for (int ch = 0; ch < 3; ++ch)
                if (!(fabs(rmse[3 * it + ch] - rmse[3 * (it - 1) + ch]) < stop_delta)) small = 0;
            if (small) break;
        }
    }
    free(img); free(res); free(dV); free(J); free(src);
}
