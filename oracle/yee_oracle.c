/*
 * Yee FDTD oracle: a plain, slow, FP64 CPU stepper.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no source with the CUDA library.
 *
 * What it computes (arxiv 2502.20610, Sec. 2, Eq. 1, and Fig. 2):
 *   the standard Yee leapfrog on an nx*ny*nz grid, one half-step at a time,
 *   over the whole grid, in the order
 *       H^{n+1/2} = H^{n-1/2} - dt * curl_f E^n          (forward differences)
 *       E^{n+1}   = E^n + ce * curl_b H^{n+1/2}          (backward differences)
 *       E_c[s]   += -ce[s] * J_n                          (point current sources)
 *   Eq. 1 prints the Ex row with backward H differences; the other two E rows
 *   are its cyclic permutations and the H rows are the adjoint (forward
 *   difference) form, the textbook Yee update with dx = dy = dz = 1, mu = 1.
 *   ce = dt / eps per cell (Eq. 1 prints the vacuum case dt/dy; the paper's
 *   implementation carries a per-cell permittivity structure field, Sec. 4).
 *
 * Conductivity (the lossy structure field of Sec. 4, used for absorbing
 *   layers): with sigma > 0 in a cell, the E half-step is the time-centred
 *   discretisation of eps dE/dt + sigma E = curl H - J,
 *       E^{n+1} = ca * E^n + cb * (curl_b H^{n+1/2} - J),
 *       ca = (1 - sigma dt / (2 eps)) / (1 + sigma dt / (2 eps)),
 *       cb = (dt / eps) / (1 + sigma dt / (2 eps)),
 *   which is the lossless update when sigma = 0.  The graded absorber sets
 *   sigma = sigma_max * sum_a (depth_a / L)^m over a layer of L cells at
 *   every wall, depth_a = L - i for i < L, i - (N - 1 - L) for i >= N - L.
 *
 * Grid convention: arrays of nx*ny*nz doubles, index i + nx*(j + ny*k).
 *   Cell (i,j,k) holds Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2),
 *   Hx(i,j+1/2,k+1/2), Hy(i+1/2,j,k+1/2), Hz(i+1/2,j+1/2,k).
 * Boundary:
 *   PEC box [0,N]^3: E at index N reads as 0; tangential E on the low planes
 *   (i=0: Ey,Ez; j=0: Ex,Ez; k=0: Ex,Ey) is never updated.
 *   PERIODIC: every index wraps (oracle-only; used for the dispersion pin).
 *
 * 16-bit field storage (the FP16 / BF16 storage option of the GPU library):
 *   when switched on, every value of field c is kept as s_c * R(v / s_c)
 *   with a power-of-two scale s_c, R rounding to the nearest number of the
 *   16-bit format (ties to even): H values right after the H half-step, E
 *   values after the E half-step and the point sources.  Arithmetic stays
 *   FP64; only what is stored is rounded.
 *
 * Pins (see tests/test_oracle_pins.py): exact energy invariant, Gauss-law
 * invariants, closed-form discrete cavity eigenmodes, the Yee dispersion
 * relation for periodic plane waves, the source work identity and planted
 * mutations that each of those must catch; the storage rounding against
 * numpy's binary16 and torch's bfloat16 conversions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_SOURCES 16

typedef struct {
    int comp;      /* 0,1,2 = Ex,Ey,Ez */
    long idx;      /* linear cell index */
    double *J;     /* J(t_{n+1/2}) for absolute step n */
    long nJ;
} or_source;

typedef struct {
    int nx, ny, nz, periodic;
    double dt;
    double *f[6];  /* Ex Ey Ez Hx Hy Hz */
    double *ce;    /* per-cell E coefficient cb (dt/eps when lossless) */
    double *ca;    /* per-cell E decay ca, NULL when lossless */
    long step;
    int nsrc;
    or_source src[OR_MAX_SOURCES];
    int mutation;  /* 0 = none; >0 plants a known mistake (pin sensitivity tests) */
    int sp, semin, semax;  /* storage rounding: significant bits (0 = off), exponent range */
    double sscale[6];
} yee_oracle;

static long ncell(const yee_oracle *o) { return (long)o->nx * o->ny * o->nz; }

yee_oracle *oracle_create(int nx, int ny, int nz, int periodic, double dt)
{
    if (nx < 1 || ny < 1 || nz < 1) return NULL;
    yee_oracle *o = (yee_oracle *)calloc(1, sizeof(yee_oracle));
    if (!o) return NULL;
    o->nx = nx; o->ny = ny; o->nz = nz; o->periodic = periodic; o->dt = dt;
    long n = ncell(o);
    for (int c = 0; c < 6; ++c) o->f[c] = (double *)calloc((size_t)n, sizeof(double));
    o->ce = (double *)calloc((size_t)n, sizeof(double));
    for (long p = 0; p < n; ++p) o->ce[p] = dt; /* vacuum */
    return o;
}

void oracle_destroy(yee_oracle *o)
{
    if (!o) return;
    for (int c = 0; c < 6; ++c) free(o->f[c]);
    free(o->ce);
    free(o->ca);
    for (int s = 0; s < o->nsrc; ++s) free(o->src[s].J);
    free(o);
}

/* eps per cell; quantize_f32 != 0 rounds dt/eps to float once (the GPU's
 * coefficient), else keeps the FP64 value. */
void oracle_set_eps(yee_oracle *o, const double *eps, int quantize_f32)
{
    long n = ncell(o);
    for (long p = 0; p < n; ++p) {
        double c = o->dt / eps[p];
        o->ce[p] = quantize_f32 ? (double)(float)c : c;
    }
}

/* eps and conductivity sigma per cell: ca and cb as above; quantize_f32 != 0
 * rounds ca and cb to float once (the GPU's coefficients). */
void oracle_set_eps_sigma(yee_oracle *o, const double *eps, const double *sigma, int quantize_f32)
{
    long n = ncell(o);
    if (!o->ca) o->ca = (double *)malloc(sizeof(double) * (size_t)n);
    for (long p = 0; p < n; ++p) {
        double h = sigma[p] * o->dt / (2.0 * eps[p]);
        double a = (1.0 - h) / (1.0 + h), b = (o->dt / eps[p]) / (1.0 + h);
        if (o->mutation == 6) a = (1.0 + h) / (1.0 - h); /* planted: loss with the wrong sign */
        o->ca[p] = quantize_f32 ? (double)(float)a : a;
        o->ce[p] = quantize_f32 ? (double)(float)b : b;
    }
}

/* The graded profile: sigma_max * sum over axes of (depth / L)^m. */
void oracle_graded_sigma(int nx, int ny, int nz, int L, double sigma_max, int m, double *sigma)
{
    int n[3] = {nx, ny, nz};
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int idx[3] = {i, j, k};
                double s = 0.0;
                for (int a = 0; a < 3; ++a) {
                    int d = 0;
                    if (idx[a] < L) d = L - idx[a];
                    else if (idx[a] >= n[a] - L) d = idx[a] - (n[a] - 1 - L);
                    if (d > 0) s += pow((double)d / L, m);
                }
                sigma[i + (long)nx * (j + (long)ny * k)] = sigma_max * s;
            }
}

void oracle_get_ca(const yee_oracle *o, double *dst)
{
    long n = ncell(o);
    for (long p = 0; p < n; ++p) dst[p] = o->ca ? o->ca[p] : 1.0;
}

void oracle_set_field(yee_oracle *o, int comp, const double *src)
{
    memcpy(o->f[comp], src, sizeof(double) * (size_t)ncell(o));
}

void oracle_get_field(const yee_oracle *o, int comp, double *dst)
{
    memcpy(dst, o->f[comp], sizeof(double) * (size_t)ncell(o));
}

void oracle_get_ce(const yee_oracle *o, double *dst)
{
    memcpy(dst, o->ce, sizeof(double) * (size_t)ncell(o));
}

/* Round x to the nearest number with p significant bits whose exponent is
 * at least emin (below 2^emin the spacing stays 2^(emin-p+1): subnormals),
 * ties to even; results of magnitude >= 2^(emax+1) become infinite.
 * IEEE binary16: p = 11, emin = -14, emax = 15.  bfloat16: p = 8,
 * emin = -126, emax = 127.  Scaling by powers of two is exact in FP64 here. */
double oracle_round_to_format(double x, int p, int emin, int emax)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e); /* |x| in [2^(e-1), 2^e) */
    int lead = e - 1;
    if (lead < emin) lead = emin;
    double ulp = ldexp(1.0, lead - (p - 1));
    double r = nearbyint(x / ulp) * ulp; /* default rounding mode: ties to even */
    if (fabs(r) >= ldexp(1.0, emax + 1)) r = copysign(INFINITY, x);
    return r;
}

static void round_field(yee_oracle *o, int c)
{
    if (o->sp <= 0) return;
    long n = ncell(o);
    double s = o->sscale[c];
    /* every element is rounded on its own: threads do not change the result */
#pragma omp parallel for schedule(static)
    for (long q = 0; q < n; ++q) o->f[c][q] = s * oracle_round_to_format(o->f[c][q] / s, o->sp, o->semin, o->semax);
}

/* Switch 16-bit storage rounding on (p > 0) or off (p = 0) with per-component
 * power-of-two scales; the current fields are rounded at once. */
void oracle_set_storage(yee_oracle *o, int p, int emin, int emax, const double *scale)
{
    o->sp = p;
    o->semin = emin;
    o->semax = emax;
    for (int c = 0; c < 6; ++c) {
        o->sscale[c] = scale ? scale[c] : 1.0;
        round_field(o, c);
    }
}

long oracle_current_step(const yee_oracle *o) { return o->step; }
void oracle_set_step(yee_oracle *o, long s) { o->step = s; }
void oracle_set_mutation(yee_oracle *o, int m) { o->mutation = m; }

int oracle_add_source(yee_oracle *o, int comp, int i, int j, int k, const double *J, long nJ)
{
    if (o->nsrc >= OR_MAX_SOURCES || comp < 0 || comp > 2) return -1;
    if (i < 0 || j < 0 || k < 0 || i >= o->nx || j >= o->ny || k >= o->nz) return -1;
    or_source *s = &o->src[o->nsrc++];
    s->comp = comp;
    s->idx = i + (long)o->nx * (j + (long)o->ny * k);
    s->nJ = nJ;
    s->J = (double *)malloc(sizeof(double) * (size_t)(nJ > 0 ? nJ : 1));
    if (nJ > 0) memcpy(s->J, J, sizeof(double) * (size_t)nJ);
    return 0;
}

/* Value of field c at (i,j,k) with the boundary rule applied: PEC reads 0
 * outside [0,N), PERIODIC wraps. */
static double at(const yee_oracle *o, int c, int i, int j, int k)
{
    if (o->periodic) {
        i = (i % o->nx + o->nx) % o->nx;
        j = (j % o->ny + o->ny) % o->ny;
        k = (k % o->nz + o->nz) % o->nz;
    } else if (i < 0 || j < 0 || k < 0 || i >= o->nx || j >= o->ny || k >= o->nz) {
        return 0.0;
    }
    return o->f[c][i + (long)o->nx * (j + (long)o->ny * k)];
}

enum { EX, EY, EZ, HX, HY, HZ };

/* (curl_f E) at the H positions of cell (i,j,k): forward differences. */
static void curl_e(const yee_oracle *o, int i, int j, int k, double out[3])
{
    double ex = at(o, EX, i, j, k), ey = at(o, EY, i, j, k), ez = at(o, EZ, i, j, k);
    out[0] = (at(o, EZ, i, j + 1, k) - ez) - (at(o, EY, i, j, k + 1) - ey);
    out[1] = (at(o, EX, i, j, k + 1) - ex) - (at(o, EZ, i + 1, j, k) - ez);
    out[2] = (at(o, EY, i + 1, j, k) - ey) - (at(o, EX, i, j + 1, k) - ex);
    if (o->mutation == 1) out[1] = (at(o, EX, i, j, k + 1) - ex) + (at(o, EZ, i + 1, j, k) - ez);
    if (o->mutation == 2) out[2] = (at(o, EY, i, j + 1, k) - ey) - (at(o, EX, i, j + 1, k) - ex);
}

/* (curl_b H) at the E positions of cell (i,j,k): backward differences, Eq. 1. */
static void curl_h(const yee_oracle *o, int i, int j, int k, double out[3])
{
    double hx = at(o, HX, i, j, k), hy = at(o, HY, i, j, k), hz = at(o, HZ, i, j, k);
    out[0] = (hz - at(o, HZ, i, j - 1, k)) - (hy - at(o, HY, i, j, k - 1));
    out[1] = (hx - at(o, HX, i, j, k - 1)) - (hz - at(o, HZ, i - 1, j, k));
    out[2] = (hy - at(o, HY, i - 1, j, k)) - (hx - at(o, HX, i, j - 1, k));
    if (o->mutation == 3) out[0] = (hz - at(o, HZ, i - 1, j, k)) - (hy - at(o, HY, i, j, k - 1));
}

/* Is component c (0..2) of cell (i,j,k) a tangential E on a low PEC wall? */
static int pec_fixed(const yee_oracle *o, int c, int i, int j, int k)
{
    if (o->periodic) return 0;
    switch (c) {
    case EX: return j == 0 || k == 0;
    case EY: return i == 0 || k == 0;
    default: return i == 0 || j == 0;
    }
}

static void half_step_h(yee_oracle *o, double **hout)
{
    const int nx = o->nx, ny = o->ny, nz = o->nz;
    const double dt = (o->mutation == 4) ? 0.5 * o->dt : o->dt;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long p = i + (long)nx * (j + (long)ny * k);
                double c[3];
                curl_e(o, i, j, k, c);
                for (int a = 0; a < 3; ++a) hout[a][p] = o->f[HX + a][p] - dt * c[a];
            }
}

static void half_step_e(yee_oracle *o, double **eout)
{
    const int nx = o->nx, ny = o->ny, nz = o->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long p = i + (long)nx * (j + (long)ny * k);
                double c[3];
                curl_h(o, i, j, k, c);
                double decay = o->ca ? o->ca[p] : 1.0;
                for (int a = 0; a < 3; ++a)
                    eout[a][p] = pec_fixed(o, a, i, j, k) ? o->f[EX + a][p]
                                                          : decay * o->f[EX + a][p] + o->ce[p] * c[a];
            }
}

/* Advance n full steps: (E^m, H^{m-1/2}) -> (E^{m+n}, H^{m+n-1/2}). */
/* Threads the parallel loops use from now on (n >= 1); returns the number
 * in effect (1 when built without OpenMP).  Timing only: the results do not
 * depend on it (every loop writes disjoint cells; the energy reduction is
 * not used by the stepper). */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int oracle_step(yee_oracle *o, long n)
{
    long nc = ncell(o);
    double *tmp[3];
    for (int a = 0; a < 3; ++a) {
        tmp[a] = (double *)malloc(sizeof(double) * (size_t)nc);
        if (!tmp[a]) { for (int b = 0; b < a; ++b) free(tmp[b]); return -1; }
    }
    for (long s = 0; s < n; ++s) {
        half_step_h(o, tmp);
        for (int a = 0; a < 3; ++a) { double *t = o->f[HX + a]; o->f[HX + a] = tmp[a]; tmp[a] = t; }
        for (int a = 0; a < 3; ++a) round_field(o, HX + a);
        half_step_e(o, tmp);
        for (int a = 0; a < 3; ++a) { double *t = o->f[EX + a]; o->f[EX + a] = tmp[a]; tmp[a] = t; }
        for (int q = 0; q < o->nsrc; ++q) {
            or_source *src = &o->src[q];
            double J = (o->step < src->nJ) ? src->J[o->step] : 0.0;
            double sign = (o->mutation == 5) ? 1.0 : -1.0;
            o->f[src->comp][src->idx] += sign * o->ce[src->idx] * J;
        }
        for (int a = 0; a < 3; ++a) round_field(o, EX + a);
        o->step += 1;
    }
    for (int a = 0; a < 3; ++a) free(tmp[a]);
    return 0;
}

/* Effective permittivity of cell p for the coefficients in use: from
 * ca = (eps - g)/(eps + g), cb = dt/(eps + g) with g = sigma dt / 2,
 * eps = (dt/cb)(1 + ca)/2 and g = (dt/cb)(1 - ca)/2 (eps = dt/ce when lossless). */
static double eps_eff(const yee_oracle *o, long p)
{
    double a = o->ca ? o->ca[p] : 1.0;
    return o->dt / o->ce[p] * (1.0 + a) * 0.5;
}

/* Q^n = sum eps_eff |E^n|^2 + sum H^{n-1/2} . H^{n+1/2}.
 * Conserved exactly by the leapfrog in a lossless, source-free box; with
 * conductivity, Q^{n+1} - Q^n = -sum g |E^{n+1} + E^n|^2 exactly. */
double oracle_energy(const yee_oracle *o)
{
    const int nx = o->nx, ny = o->ny, nz = o->nz;
    double q = 0.0;
#pragma omp parallel for reduction(+ : q) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long p = i + (long)nx * (j + (long)ny * k);
                double w = eps_eff(o, p);
                double c[3];
                curl_e(o, i, j, k, c);
                for (int a = 0; a < 3; ++a) {
                    double e = o->f[EX + a][p], h = o->f[HX + a][p];
                    q += w * e * e + h * (h - o->dt * c[a]);
                }
            }
    return q;
}

/* Discrete divergence of eps_eff*E at nodes (i,j,k) (backward differences)
 * and of H at dual nodes (i+1/2,j+1/2,k+1/2) (forward differences), written
 * into caller arrays of nx*ny*nz doubles.  PEC reads 0 outside. */
void oracle_div(const yee_oracle *o, double *div_e, double *div_h)
{
    const int nx = o->nx, ny = o->ny, nz = o->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long p = i + (long)nx * (j + (long)ny * k);
                double d = 0.0;
                int ii[3] = {i - 1, i, i}, jj[3] = {j, j - 1, j}, kk[3] = {k, k, k - 1};
                for (int a = 0; a < 3; ++a) {
                    double w0 = eps_eff(o, p);
                    double lo = at(o, EX + a, ii[a], jj[a], kk[a]);
                    double wlo = 0.0;
                    if (o->periodic || (ii[a] >= 0 && jj[a] >= 0 && kk[a] >= 0)) {
                        int i2 = (ii[a] + nx) % nx, j2 = (jj[a] + ny) % ny, k2 = (kk[a] + nz) % nz;
                        wlo = eps_eff(o, i2 + (long)nx * (j2 + (long)ny * k2));
                    }
                    d += w0 * o->f[EX + a][p] - wlo * lo;
                }
                if (div_e) div_e[p] = d;
                if (div_h)
                    div_h[p] = (at(o, HX, i + 1, j, k) - o->f[HX][p]) +
                               (at(o, HY, i, j + 1, k) - o->f[HY][p]) +
                               (at(o, HZ, i, j, k + 1) - o->f[HZ][p]);
            }
}
