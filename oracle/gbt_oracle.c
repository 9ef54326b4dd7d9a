/*
 * gbt_oracle.c -- plain FP64 CPU oracle for Gaussian beam summation (GBS).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or helper with the CUDA
 * library; both sides are written independently from the paper's definitions.
 *
 * It is deliberately slow and direct: loops in the order the method states,
 * double precision throughout, no blocking or fusion.  OpenMP only splits the
 * receiver loop of the sum and the ray loop of the tracer (each receiver's sum
 * and each ray's path are independent and keep their own order).
 *
 * What it computes (paper: "Accelerating Gaussian beam tracing method with
 * dynamic parallelism on GPUs", arXiv 2501.13382):
 *
 *  1. Fan of rays (Sec. 3.3: each ray's initial direction is set by its
 *     take-off angles; Eq. 3 integrates over these take-off parameters).
 *     A Fibonacci sphere: z_i = 1 - (2i+1)/N, phi_i = i * pi (3 - sqrt 5),
 *     each ray carrying the solid-angle weight 4 pi / N; or the paper's grid
 *     of elevation x azimuth angles, each ray carrying its cell's solid angle.
 *  2. Ray tracing (Sec. 2 and Sec. 3.1: rays and their specular interactions
 *     with planar facets).  Homogeneous medium, so rays are straight lines;
 *     nearest hit over the ground plane and the triangles (Moller-Trumbore),
 *     mirror reflection d' = d - 2 (d.n) n, stop at max_path or at the first
 *     hit after max_reflections reflections.  Output: a flat list of straight
 *     segments in ray order (CSR by ray).
 *  3. Beam summation (Eq. 3 with the beam field of Eq. 1 and the dynamic ray
 *     tracing system of Eq. 2).  In a homogeneous medium Eq. 2 gives P = I/c
 *     constant and Q(s) = Q0 + c P s; with an isotropic start Q0 = -i b I/c
 *     the beam stays isotropic across plane mirrors, so for a receiver at
 *     arclength s along the unfolded ray and normal distance n:
 *        E = s - i b,
 *        c = W * Gamma_path * (k b / (8 pi^2)) * (1/E) * exp(i k s + i k n^2 / (2E)),
 *     where k = omega / c_sound, W the ray weight and Gamma_path the product of
 *     the reflection coefficients met before the segment.  The constant
 *     k b / (8 pi^2) is the normalisation for which the sum over a dense fan
 *     tends to the free-field point source exp(ikr) / (4 pi r) (Eq. 3's
 *     weighting function, which the paper leaves as a real constant).
 *     A pair is kept iff its Gaussian exponent k n^2 b / (2 (s^2+b^2)) <= C and
 *     it lies in the segment's window (SEGMENT: 0 <= s_loc < L; LINE: s >= 0).
 *  4. Adjoint of the sum for a real loss L with g = dL/dRe p + i dL/dIm p:
 *     dL/dtheta = sum Re(conj(g) dp/dtheta) for theta = per-material gamma,
 *     per-ray weight and per-frequency beam parameter b (cull mask held fixed).
 *  5. Propagation losses.  The paper's input tables (Sec. 4.5, Tables 2-3) give
 *     the air temperature, relative humidity and pressure and a flow-impedance
 *     setting of the surfaces, and say they shape the field, but give no
 *     formula.  Standard published ones are used: the pure-tone absorption of
 *     air of ISO 9613-1, applied as the amplitude factor exp(-a s) over the
 *     unfolded arclength s of the beam; and, for a porous surface of effective
 *     flow resistivity sigma, the normalised impedance of Delany and Bazley
 *     (1970) with the plane-wave reflection factor of a locally reacting
 *     surface at each reflection's angle of incidence, multiplying the
 *     material's gamma.  A surface with sigma <= 0 is hard (the paper's
 *     negative setting): its reflection is gamma alone.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ fan -- */

/* Fibonacci-sphere take-off directions (the fan of Sec. 3.3 / Eq. 3). */
void orc_fan_fibonacci(int64_t n, double *dirs)
{
    const double golden = ORC_PI * (3.0 - sqrt(5.0));
    for (int64_t i = 0; i < n; ++i) {
        double z = 1.0 - (2.0 * (double)i + 1.0) / (double)n;
        double r = sqrt(1.0 - z * z);
        double phi = (double)i * golden;
        dirs[3 * i + 0] = r * cos(phi);
        dirs[3 * i + 1] = r * sin(phi);
        dirs[3 * i + 2] = z;
    }
}

/* Latitude-longitude fan: the paper sets each ray's initial direction by a
 * pair of take-off angles over an elevation range and an azimuth range (its
 * input tables give 0..180 and 0..360 degrees).  Reading: the elevation is
 * the polar angle from +z; ray g = it * n_phi + ip sits at the centre of its
 * (theta, phi) cell, theta = th0 + (it + 1/2) dth, phi = ph0 + (ip + 1/2) dph,
 * and carries the cell's solid angle, the integral of sin(theta) over the
 * cell:  w = dph * (cos theta_lo - cos theta_hi). */
void orc_fan_latlong(int64_t n_theta, int64_t n_phi, double th0_deg, double th1_deg,
                     double ph0_deg, double ph1_deg, double *dirs, double *w)
{
    const double deg = ORC_PI / 180.0;
    const double th0 = th0_deg * deg, ph0 = ph0_deg * deg;
    const double dth = (th1_deg - th0_deg) * deg / (double)n_theta;
    const double dph = (ph1_deg - ph0_deg) * deg / (double)n_phi;
    for (int64_t it = 0; it < n_theta; ++it) {
        const double th = th0 + ((double)it + 0.5) * dth;
        const double lo = th0 + (double)it * dth, hi = th0 + (double)(it + 1) * dth;
        const double cell = dph * (cos(lo) - cos(hi));
        for (int64_t ip = 0; ip < n_phi; ++ip) {
            const double ph = ph0 + ((double)ip + 0.5) * dph;
            const int64_t g = it * n_phi + ip;
            dirs[3 * g + 0] = sin(th) * cos(ph);
            dirs[3 * g + 1] = sin(th) * sin(ph);
            dirs[3 * g + 2] = cos(th);
            w[g] = cell;
        }
    }
}

/* ---------------------------------------------------------------- trace -- */

typedef struct {
    int ground;            /* ground plane z = ground_z present */
    double ground_z;
    int ground_material;
    int64_t n_tri;
    const double *tri;     /* n_tri * 9 : v0, v1, v2 */
    const int32_t *tri_material;
    const int32_t *tri_face;
} orc_scene;

/* Moller-Trumbore ray/triangle test; returns t or -1 when there is no hit.
 * Barycentric bounds are inclusive. */
static double orc_ray_triangle(const double *o, const double *d, const double *v)
{
    double e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
    double e2x = v[6] - v[0], e2y = v[7] - v[1], e2z = v[8] - v[2];
    /* p = d x e2 */
    double px = d[1] * e2z - d[2] * e2y;
    double py = d[2] * e2x - d[0] * e2z;
    double pz = d[0] * e2y - d[1] * e2x;
    double det = e1x * px + e1y * py + e1z * pz;
    if (det == 0.0) return -1.0;
    double inv = 1.0 / det;
    double tx = o[0] - v[0], ty = o[1] - v[1], tz = o[2] - v[2];
    double u = (tx * px + ty * py + tz * pz) * inv;
    if (u < 0.0 || u > 1.0) return -1.0;
    /* q = tvec x e1 */
    double qx = ty * e1z - tz * e1y;
    double qy = tz * e1x - tx * e1z;
    double qz = tx * e1y - ty * e1x;
    double v_ = (d[0] * qx + d[1] * qy + d[2] * qz) * inv;
    if (v_ < 0.0 || u + v_ > 1.0) return -1.0;
    return (e2x * qx + e2y * qy + e2z * qz) * inv;
}

/* Unit normal of a triangle: (v1-v0) x (v2-v0) normalised. */
static void orc_triangle_normal(const double *v, double *n)
{
    double e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
    double e2x = v[6] - v[0], e2y = v[7] - v[1], e2z = v[8] - v[2];
    double nx = e1y * e2z - e1z * e2y;
    double ny = e1z * e2x - e1x * e2z;
    double nz = e1x * e2y - e1y * e2x;
    double len = sqrt(nx * nx + ny * ny + nz * nz);
    n[0] = nx / len; n[1] = ny / len; n[2] = nz / len;
}

/*
 * Trace one fan.  For ray i the segments are written at rows
 * [i*(R+1), i*(R+1) + cnt[i]) of the padded output arrays (R = max_refl).
 * Per segment: origin o, direction t, length L, start arclength s0,
 * material of the reflection that starts it (-1 for the first), and the
 * primitive that ends it (0 = ground, 1+k = triangle k, -1 = none).
 *
 * Primitive order for ties is ground first, then triangles by index; a hit
 * must have t > t_min and may not lie on the facet the ray just left
 * (ground facet = -2, triangle facet = tri_face[k]).
 */
void orc_trace(const orc_scene *sc, const double *src, const double *dirs,
               int64_t n_rays, int max_refl, double max_path, double t_min,
               int32_t *cnt, double *seg_o, double *seg_t, double *seg_L,
               double *seg_s0, int32_t *seg_bmat, int32_t *seg_hit)
{
    const int64_t stride = max_refl + 1;
    /* rays are independent: each writes only its own padded rows */
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n_rays; ++i) {
        double o[3] = {src[0], src[1], src[2]};
        double d[3] = {dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]};
        double s0 = 0.0;
        int last_face = -1;     /* no facet yet */
        int bmat = -1;
        int nref = 0, nseg = 0;
        for (;;) {
            double tbest = INFINITY;
            int best = -1;
            if (sc->ground && last_face != -2 && d[2] != 0.0) {
                double t = (sc->ground_z - o[2]) / d[2];
                if (t > t_min && t < tbest) { tbest = t; best = 0; }
            }
            for (int64_t k = 0; k < sc->n_tri; ++k) {
                int face = sc->tri_face ? sc->tri_face[k] : (int)k;
                if (face == last_face) continue;
                double t = orc_ray_triangle(o, d, sc->tri + 9 * k);
                if (t > t_min && t < tbest) { tbest = t; best = (int)(k + 1); }
            }
            double remaining = max_path - s0;
            int64_t row = i * stride + nseg;
            seg_o[3 * row + 0] = o[0]; seg_o[3 * row + 1] = o[1]; seg_o[3 * row + 2] = o[2];
            seg_t[3 * row + 0] = d[0]; seg_t[3 * row + 1] = d[1]; seg_t[3 * row + 2] = d[2];
            seg_s0[row] = s0;
            seg_bmat[row] = bmat;
            ++nseg;
            if (best < 0 || tbest >= remaining) {
                seg_L[row] = remaining;
                seg_hit[row] = -1;
                break;
            }
            seg_L[row] = tbest;
            seg_hit[row] = best;
            if (nref == max_refl) break;
            /* specular reflection at the hit point */
            double nrm[3];
            int face, mat;
            if (best == 0) {
                nrm[0] = 0.0; nrm[1] = 0.0; nrm[2] = 1.0;
                face = -2; mat = sc->ground_material;
            } else {
                const int64_t k = best - 1;
                orc_triangle_normal(sc->tri + 9 * k, nrm);
                face = sc->tri_face ? sc->tri_face[k] : (int)k;
                mat = sc->tri_material[k];
            }
            o[0] = o[0] + tbest * d[0];
            o[1] = o[1] + tbest * d[1];
            o[2] = o[2] + tbest * d[2];
            double dn = d[0] * nrm[0] + d[1] * nrm[1] + d[2] * nrm[2];
            d[0] = d[0] - 2.0 * dn * nrm[0];
            d[1] = d[1] - 2.0 * dn * nrm[1];
            d[2] = d[2] - 2.0 * dn * nrm[2];
            s0 = s0 + tbest;
            last_face = face;
            bmat = mat;
            ++nref;
        }
        cnt[i] = nseg;
    }
}

/* ---------------------------------------------------- propagation losses -- */

/* Pure-tone attenuation coefficient of air in dB per metre (ISO 9613-1): the
 * saturation vapour pressure over the triple-point temperature, the molar
 * concentration h of water vapour from the relative humidity, the relaxation
 * frequencies of oxygen and nitrogen, and the classical-plus-rotational term
 * with the two vibrational relaxation terms.  T_c in degrees Celsius, rh in
 * percent, p_kpa the ambient pressure in kPa. */
double orc_air_absorption_db(double f, double T_c, double rh, double p_kpa)
{
    const double T0 = 293.15;            /* reference temperature, K */
    const double T01 = 273.16;           /* triple-point isotherm temperature, K */
    const double pr = 101.325;           /* reference pressure, kPa */
    const double T = T_c + 273.15;
    const double prel = p_kpa / pr;
    const double C = -6.8346 * pow(T01 / T, 1.261) + 4.6151;
    const double psat_rel = pow(10.0, C);               /* p_sat / p_r */
    const double h = rh * psat_rel / prel;              /* percent */
    const double frO = prel * (24.0 + 4.04e4 * h * (0.02 + h) / (0.391 + h));
    const double frN = prel * pow(T / T0, -0.5) *
                       (9.0 + 280.0 * h * exp(-4.170 * (pow(T / T0, -1.0 / 3.0) - 1.0)));
    const double classical = 1.84e-11 / prel * sqrt(T / T0);
    const double oxygen = 0.01275 * exp(-2239.1 / T) / (frO + f * f / frO);
    const double nitrogen = 0.1068 * exp(-3352.0 / T) / (frN + f * f / frN);
    return 8.686 * f * f * (classical + pow(T / T0, -2.5) * (oxygen + nitrogen));
}

/* The same attenuation as a pressure-amplitude decay rate a (Np/m): the amplitude
 * falls as exp(-a s) over a path of length s, and 20 log10(e) dB = 1 Np. */
double orc_air_absorption_np(double f, double T_c, double rh, double p_kpa)
{
    return orc_air_absorption_db(f, T_c, rh, p_kpa) / (20.0 / log(10.0));
}

/* Normalised surface impedance Z / (rho c) of a porous surface of effective flow
 * resistivity sigma (kPa s m^-2) at frequency f (Hz): Delany and Bazley's
 * one-parameter model, written for the exp(-i omega t) convention. */
static double complex orc_delany_bazley(double f, double sigma)
{
    const double x = f / sigma;
    return 1.0 + 9.08 * pow(x, -0.75) + I * 11.9 * pow(x, -0.73);
}

void orc_delany_bazley_z(double f, double sigma, double *z)
{
    const double complex Z = orc_delany_bazley(f, sigma);
    z[0] = creal(Z);
    z[1] = cimag(Z);
}

/* Reflection factor of a plane wave meeting a locally reacting surface of
 * normalised impedance Z at incidence angle theta (cos_theta = cos theta). */
static double complex orc_plane_wave_reflection(double complex Z, double cos_theta)
{
    return (Z * cos_theta - 1.0) / (Z * cos_theta + 1.0);
}

void orc_plane_wave_reflection_r(const double *z, double cos_theta, double *r)
{
    const double complex R = orc_plane_wave_reflection(z[0] + I * z[1], cos_theta);
    r[0] = creal(R);
    r[1] = cimag(R);
}

/* Cosine of the angle of incidence at the reflection that starts each segment:
 * |t_j . n| with n the unit normal of the primitive that ended segment j - 1
 * (a mirror reflection keeps |d . n|, so the reflected direction gives it);
 * 1 for the first segment of a ray. */
void orc_incidence_cos(const orc_scene *sc, int64_t n_seg, const double *t,
                       const int32_t *depth, const int32_t *hit, double *cosi)
{
    for (int64_t j = 0; j < n_seg; ++j) {
        if (depth[j] == 0) { cosi[j] = 1.0; continue; }
        const int32_t prim = hit[j - 1];
        double nrm[3] = {0.0, 0.0, 1.0};
        if (prim >= 1) orc_triangle_normal(sc->tri + 9 * (int64_t)(prim - 1), nrm);
        cosi[j] = fabs(t[3 * j] * nrm[0] + t[3 * j + 1] * nrm[1] + t[3 * j + 2] * nrm[2]);
    }
}

/* Per frequency f and segment j: the product, over the reflections before j off a
 * porous material (sigma[m] > 0), of the plane-wave reflection factor of the
 * material's Delany-Bazley impedance at that reflection's incidence; 1 where the
 * path met none.  out: interleaved complex, [n_freq][n_seg]. */
void orc_path_factor(int64_t n_seg, const int32_t *depth, const int32_t *bmat,
                     const double *cosi, const double *sigma, const double *freq, int n_freq,
                     double *out)
{
    for (int f = 0; f < n_freq; ++f) {
        for (int64_t j = 0; j < n_seg; ++j) {
            double complex F = 1.0;
            const int64_t first = j - depth[j];
            for (int64_t q = first + 1; q <= j; ++q) {
                const double sg = sigma[bmat[q]];
                if (sg > 0.0)
                    F *= orc_plane_wave_reflection(orc_delany_bazley(freq[f], sg), cosi[q]);
            }
            out[2 * ((int64_t)f * n_seg + j) + 0] = creal(F);
            out[2 * ((int64_t)f * n_seg + j) + 1] = cimag(F);
        }
    }
}

/* ------------------------------------------------------------------ sum -- */

typedef struct {
    int64_t n_seg;
    const double *o;        /* n_seg*3 */
    const double *t;        /* n_seg*3 */
    const double *L;
    const double *s0;
    const int32_t *ray;     /* ray index of each segment */
    const int32_t *depth;   /* index of the segment within its ray */
    const int32_t *bmat;    /* material of the reflection starting the segment, -1 first */
} orc_segments;

typedef struct {
    double c;               /* speed of sound */
    int n_freq;
    const double *freq;     /* Hz */
    const double *b;        /* beam parameter per frequency (m) */
    const double *b_mask;   /* b used by the cull test (NULL -> b) */
    double cutoff;          /* C */
    int window;             /* 0 SEGMENT, 1 LINE */
    const double *absorb;   /* amplitude attenuation of air per frequency, Np/m (NULL: none) */
    const double *seg_factor; /* complex reflection factors of porous surfaces per frequency and
                                 segment, interleaved [n_freq][n_seg] (NULL: none) */
} orc_sum_args;

/* Gamma_path of segment j: product of gamma over the reflections before it. */
static double orc_gamma_path(const orc_segments *S, int64_t j, const double *gamma)
{
    double g = 1.0;
    int64_t first = j - S->depth[j];
    for (int64_t q = first + 1; q <= j; ++q) g *= gamma[S->bmat[q]];
    return g;
}

/* Geometry of receiver x against segment j: s_loc, s, n^2.  n^2 uses the
 * cross product |(x-o) x t|^2. */
static void orc_geometry(const orc_segments *S, int64_t j, const double *x,
                         double *s_loc, double *s, double *n2)
{
    const double *o = S->o + 3 * j, *t = S->t + 3 * j;
    double dx = x[0] - o[0], dy = x[1] - o[1], dz = x[2] - o[2];
    double sl = dx * t[0] + dy * t[1] + dz * t[2];
    double cx = dy * t[2] - dz * t[1];
    double cy = dz * t[0] - dx * t[2];
    double cz = dx * t[1] - dy * t[0];
    *s_loc = sl;
    *s = S->s0[j] + sl;
    *n2 = cx * cx + cy * cy + cz * cz;
}

static int orc_keep(const orc_segments *S, int64_t j, const orc_sum_args *A,
                    double k, double bm, double s_loc, double s, double n2)
{
    if (A->window == 0) {
        if (!(s_loc >= 0.0 && s_loc < S->L[j])) return 0;
    } else {
        if (!(s >= 0.0)) return 0;
    }
    return k * n2 * bm / (2.0 * (s * s + bm * bm)) <= A->cutoff;
}

/* Gaussian beam contribution with unit weight and unit Gamma_path. */
static double complex orc_beam(double k, double b, double s, double n2)
{
    double complex E = s - I * b;
    return (k * b / (8.0 * ORC_PI * ORC_PI)) / E * cexp(I * k * s + I * k * n2 / (2.0 * E));
}

/* Neumaier-compensated complex accumulator. */
typedef struct { double sr, cr, si, ci; } orc_acc;
static void orc_acc_add1(double *sum, double *comp, double v)
{
    double t = *sum + v;
    if (fabs(*sum) >= fabs(v)) *comp += (*sum - t) + v;
    else *comp += (v - t) + *sum;
    *sum = t;
}
static void orc_acc_add(orc_acc *a, double complex v)
{
    orc_acc_add1(&a->sr, &a->cr, creal(v));
    orc_acc_add1(&a->si, &a->ci, cimag(v));
}

/* Losses of segment j at frequency f and arclength s: the porous reflections'
 * factor times the air's amplitude decay exp(-a s) (1 without losses). */
static double complex orc_losses(const orc_segments *S, const orc_sum_args *A, int f, int64_t j,
                                 double s)
{
    double complex L = 1.0;
    if (A->seg_factor) {
        const double *F = A->seg_factor + 2 * ((int64_t)f * S->n_seg + j);
        L = F[0] + I * F[1];
    }
    if (A->absorb) L *= exp(-A->absorb[f] * s);
    return L;
}

/*
 * p[f][r] = sum over segments j (in order) of the kept contributions (Eq. 3).
 * recv: n_recv*3 doubles (the float32 receiver positions widened).
 * gamma: per-material reflection coefficients; weight: per-ray weights.
 * out: n_freq*n_recv complex (interleaved re, im).
 */
void orc_sum(const orc_segments *S, const orc_sum_args *A, const double *recv,
             int64_t n_recv, const double *gamma, const double *weight, double *out)
{
    double *gpath = (double *)malloc(sizeof(double) * (S->n_seg > 0 ? S->n_seg : 1));
    for (int64_t j = 0; j < S->n_seg; ++j) gpath[j] = orc_gamma_path(S, j, gamma);
    for (int f = 0; f < A->n_freq; ++f) {
        const double k = 2.0 * ORC_PI * A->freq[f] / A->c;
        const double b = A->b[f];
        const double bm = A->b_mask ? A->b_mask[f] : b;
        #pragma omp parallel for schedule(dynamic, 16)
        for (int64_t r = 0; r < n_recv; ++r) {
            orc_acc acc = {0, 0, 0, 0};
            for (int64_t j = 0; j < S->n_seg; ++j) {
                double s_loc, s, n2;
                orc_geometry(S, j, recv + 3 * r, &s_loc, &s, &n2);
                if (!orc_keep(S, j, A, k, bm, s_loc, s, n2)) continue;
                double w = weight[S->ray[j]] * gpath[j];
                orc_acc_add(&acc, w * orc_losses(S, A, f, j, s) * orc_beam(k, b, s, n2));
            }
            out[2 * (f * n_recv + r) + 0] = acc.sr + acc.cr;
            out[2 * (f * n_recv + r) + 1] = acc.si + acc.ci;
        }
    }
    free(gpath);
}

/*
 * Adjoint of orc_sum.  g: n_freq*n_recv complex (interleaved), the gradient
 * of a real loss with respect to Re p + i Im p.  Outputs (overwritten):
 * grad_gamma[n_mat], grad_weight[n_rays], grad_b[n_freq].
 *   dc/dW       = c / W
 *   dc/dGamma_m = (sum over bounces on material m of the product of the
 *                  other bounces' gamma) * c / Gamma_path
 *   dc/db       = c * (1/b + i/E - k n^2 / (2 E^2))
 */
void orc_sum_adjoint(const orc_segments *S, const orc_sum_args *A, const double *recv,
                     int64_t n_recv, const double *gamma, int n_mat, const double *weight,
                     int64_t n_rays, const double *g, double *grad_gamma,
                     double *grad_weight, double *grad_b)
{
    memset(grad_gamma, 0, sizeof(double) * n_mat);
    memset(grad_weight, 0, sizeof(double) * n_rays);
    memset(grad_b, 0, sizeof(double) * A->n_freq);
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *pw = (double *)calloc((size_t)nthreads * n_rays + 1, sizeof(double));
    double *pg = (double *)calloc((size_t)nthreads * n_mat + 1, sizeof(double));
    double *pb = (double *)calloc((size_t)nthreads * A->n_freq + 1, sizeof(double));
    double *gpath = (double *)malloc(sizeof(double) * (S->n_seg > 0 ? S->n_seg : 1));
    for (int64_t j = 0; j < S->n_seg; ++j) gpath[j] = orc_gamma_path(S, j, gamma);

    #pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mw = pw + (size_t)tid * n_rays;
        double *mg = pg + (size_t)tid * n_mat;
        double *mb = pb + (size_t)tid * A->n_freq;
        for (int f = 0; f < A->n_freq; ++f) {
            const double k = 2.0 * ORC_PI * A->freq[f] / A->c;
            const double b = A->b[f];
            const double bm = A->b_mask ? A->b_mask[f] : b;
            #pragma omp for schedule(dynamic, 16)
            for (int64_t r = 0; r < n_recv; ++r) {
                double complex gr = g[2 * (f * n_recv + r)] + I * g[2 * (f * n_recv + r) + 1];
                double complex gc = conj(gr);
                for (int64_t j = 0; j < S->n_seg; ++j) {
                    double s_loc, s, n2;
                    orc_geometry(S, j, recv + 3 * r, &s_loc, &s, &n2);
                    if (!orc_keep(S, j, A, k, bm, s_loc, s, n2)) continue;
                    const int32_t ray = S->ray[j];
                    /* W = Gamma = 1; the losses do not depend on W, gamma or b */
                    double complex cu = orc_losses(S, A, f, j, s) * orc_beam(k, b, s, n2);
                    double complex E = s - I * b;
                    /* weight */
                    mw[ray] += creal(gc * gpath[j] * cu);
                    /* beam parameter */
                    double complex dlog = 1.0 / b + I / E - k * n2 / (2.0 * E * E);
                    mb[f] += creal(gc * weight[ray] * gpath[j] * cu * dlog);
                    /* materials: d Gamma_path / d Gamma_m via products of the others */
                    int64_t first = j - S->depth[j];
                    for (int64_t q = first + 1; q <= j; ++q) {
                        double other = 1.0;
                        for (int64_t q2 = first + 1; q2 <= j; ++q2)
                            if (q2 != q) other *= gamma[S->bmat[q2]];
                        mg[S->bmat[q]] += creal(gc * weight[ray] * other * cu);
                    }
                }
            }
        }
    }
    for (int t = 0; t < nthreads; ++t) {
        for (int64_t i = 0; i < n_rays; ++i) grad_weight[i] += pw[(size_t)t * n_rays + i];
        for (int m = 0; m < n_mat; ++m) grad_gamma[m] += pg[(size_t)t * n_mat + m];
        for (int f = 0; f < A->n_freq; ++f) grad_b[f] += pb[(size_t)t * A->n_freq + f];
    }
    free(pw); free(pg); free(pb); free(gpath);
}

/* Count kept pairs (receiver x segment x frequency) -- used for reporting. */
int64_t orc_count_kept(const orc_segments *S, const orc_sum_args *A, const double *recv,
                       int64_t n_recv)
{
    int64_t total = 0;
    for (int f = 0; f < A->n_freq; ++f) {
        const double k = 2.0 * ORC_PI * A->freq[f] / A->c;
        const double bm = A->b_mask ? A->b_mask[f] : A->b[f];
        #pragma omp parallel for reduction(+:total) schedule(dynamic, 16)
        for (int64_t r = 0; r < n_recv; ++r) {
            for (int64_t j = 0; j < S->n_seg; ++j) {
                double s_loc, s, n2;
                orc_geometry(S, j, recv + 3 * r, &s_loc, &s, &n2);
                total += orc_keep(S, j, A, k, bm, s_loc, s, n2);
            }
        }
    }
    return total;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
