/*
 * FP64 CPU oracle of the DC-FSPB dose method (Gu et al., arXiv 1103.1164).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant with the CUDA path: it is a second,
 * independent statement of what the method computes, written for a reader to
 * check against the paper line by line, not for speed.
 *
 * Steps follow Algorithm A1 (Section 2.1) in its order:
 *   step 1        smoothed density rho_hat = Gaussian (x) rho             smooth()
 *   steps 2-4     per beamlet: angle theta, entry/exit on the body surface beamlets(), trace()
 *   steps 5-6     per beamlet: tables t_eq(t) and omega_corr(t)            trace()
 *   steps 7-13    per voxel, per beamlet whose ROI holds it:
 *                 A(t_eq,theta) (9), u^w, omega^w (10), density
 *                 correction (11), eqs. (1)-(4) (12)                        pair_dose(), dose()
 * The loop nesting printed in Algorithm A1 puts the voxel loop inside the
 * beamlet loop; it is read as two phases (beamlet tables, then voxel x
 * beamlet), which is what Algorithm A2 (Kernels 2-4, then Kernel 5) does.
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *  - beam frame: gantry rotates about +z; at gantry 0 the beam travels +y;
 *    couch rotates about +y; collimator rotates the field axes about the beam.
 *  - x, y of eq. (2): components of r - r_s - r_a on the beamlet's own
 *    orthonormal frame (e_x'' = e_x' with its n-component removed, e_y'' =
 *    e_x'' x n), scaled by SAD/|r_a| to the isocentre plane; x0, y0 are the
 *    beamlet half-widths (the |x| <= x0 branch of eq. (4)).
 *  - ROI (Algorithm A1 footnote): physical distance from the beamlet central
 *    axis <= R, inclusive.
 *  - t = |r_a| - L_in where L_in is where the central axis first enters a
 *    voxel of density > rho_surface; pairs with t < 0 or t > t_out = L_out -
 *    L_in contribute nothing; a central axis that meets no such voxel gives a
 *    beamlet with no dose.
 *  - mu/mu_H2O = rho (the input is already relative density); the radiological
 *    depth is the exact integral through voxel-constant rho (Siddon's
 *    parametric ray), sampled every d = min(dx,dy,dz)/2 (Section 2.2) and
 *    linearly interpolated between samples.
 *  - omega_corr is taken per term, omega_i^corr(t) = int b_i(rho) dt'.
 *  - every commissioned function of density takes rho clamped to the
 *    commissioned range (its table's domain); the radiological depth uses the
 *    raw density.
 *  - omega_i = f_omega_i(rho_hat) (omega_i^w + omega_i^corr) as in the text of
 *    Section 2.1, clamped at 0; u_1 uses rho at the voxel, u_2 and omega use
 *    rho_hat at the voxel; u_ix = u_iy = u_i.
 *  - omitting step 11 (density_correction = 0) gives u_i = u_i^w,
 *    omega_i = omega_i^w: the conventional FSPB with 1-D depth correction.
 *  - eq. (4) is evaluated in the algebraically identical overflow-free form
 *      |x| <= x0:  1 - (exp(-u(x0-|x|)) + exp(-u(x0+|x|)))/2
 *      |x| >  x0:  (exp(-u(|x|-x0)) - exp(-u(|x|+x0)))/2
 *  - Gaussian smoothing: 3-D kernel exp(-|r|^2/2 sigma^2) sampled on the
 *    voxel lattice, truncated at ceil(3 sigma/delta) voxels per axis,
 *    normalised to unit sum, clamp-to-edge boundary.
 *
 * Parity aids: a pair whose ROI or depth-range decision lies within a
 * rounding margin of its boundary is reported as "ambiguous" together with its
 * dose, so that a test can accept either decision on those pairs only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EPS_T 1e-4      /* cm: margin on t = 0 and t = t_out          */
#define EPS_Q 1e-3      /* cm^2: margin on |perp|^2 = R^2             */

/* Input descriptor, mirrored field by field by ctypes in oracle.py. */
typedef struct {
    int32_t nx, ny, nz, n_beams;
    double dx, dy, dz, ox, oy, oz;
    const double* rho;        /* [nz][ny][nx] relative density            */
    const double* beams;      /* [n_beams][10]: gantry, couch, coll (deg), SAD,
                                 iso x, y, z, field_x, field_y, unused     */
    double bx, by;            /* beamlet size at the isocentre plane      */
    const double* A;          /* [a_nth][a_nt], A(t_eq = j a_dt, theta = l a_dth) */
    int32_t a_nt, a_nth;
    double a_dt, a_dth;
    const double* water;      /* [4][w_n]: u1w, u2w, w1w, w2w at t = j w_dt */
    int32_t w_n, f_n;
    double w_dt;
    const double* dens;       /* [6][f_n]: f_u1, f_u2, f_w1, f_w2, b1, b2 at rho = f_rho0 + j f_drho */
    double f_rho0, f_drho;
    double roi, sigma, rho_surf;
    int32_t density_correction;
    int32_t lateral_mode;     /* 0: rho(r), rho_hat(r) (Section 2.1); 1: axis stencils */
} OInputs;

typedef struct {
    int beam;
    double n[3], ex[3], ey[3], theta;     /* direction, lateral frame, off-axis angle */
    int hit, K;
    double L_in, L_out;
    double *T, *W1, *W2;                  /* K samples at t = k d                     */
} OBeamlet;

typedef struct {
    double src[3], ez[3], ex[3], ey[3], sad;
    int M, N, first;
} OBeam;

typedef struct {
    OInputs in;
    int64_t V;
    int B;
    double d;
    double *rho, *rhos, *A, *water, *dens, *beamraw;
    OBeam* beam;
    OBeamlet* bl;
} OPlan;

/* ------------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1]*b[2] - a[2]*b[1];
    c[1] = a[2]*b[0] - a[0]*b[2];
    c[2] = a[0]*b[1] - a[1]*b[0];
}
static void normalize3(double* a)
{
    double s = sqrt(dot3(a, a));
    a[0] /= s; a[1] /= s; a[2] /= s;
}

/* Linear interpolation in a table f[j] = f(x0 + j h), j = 0..n-1, clamped to
 * the table's domain (Algorithm A1 steps 9-10 read A, u^w and omega^w from
 * commissioned tables). */
double or_lut1(const double* f, int n, double x0, double h, double x)
{
    double s = (x - x0) / h;
    if (s <= 0.0) return f[0];
    if (s >= n - 1) return f[n - 1];
    int j = (int)floor(s);
    if (j > n - 2) j = n - 2;
    double w = s - j;
    return (1.0 - w) * f[j] + w * f[j + 1];
}

/* Bilinear lookup of A(t_eq, theta) (Algorithm A1 step 9). */
static double lut_A(const OPlan* P, double teq, double theta)
{
    const OInputs* in = &P->in;
    double s = teq / in->a_dt, r = theta / in->a_dth;
    if (s < 0) s = 0;
    if (s > in->a_nt - 1) s = in->a_nt - 1;
    if (r < 0) r = 0;
    if (r > in->a_nth - 1) r = in->a_nth - 1;
    int j = (int)floor(s), l = (int)floor(r);
    if (j > in->a_nt - 2) j = in->a_nt - 2;
    if (l > in->a_nth - 2) l = in->a_nth - 2;
    double wt = s - j, wl = r - l;
    const double* A = P->A;
    double a0 = (1 - wt) * A[(size_t)l * in->a_nt + j] + wt * A[(size_t)l * in->a_nt + j + 1];
    double a1 = (1 - wt) * A[(size_t)(l + 1) * in->a_nt + j] + wt * A[(size_t)(l + 1) * in->a_nt + j + 1];
    return (1 - wl) * a0 + wl * a1;
}

/* Eq. (4), penumbra profile p(x, u, x0), overflow-free form. */
double or_p(double x, double u, double x0)
{
    double ax = fabs(x);
    if (ax <= x0) return 1.0 - 0.5 * (exp(-u * (x0 - ax)) + exp(-u * (x0 + ax)));
    return 0.5 * (exp(-u * (ax - x0)) - exp(-u * (ax + x0)));
}

/* ------------------------------------------------------------------------ */
/* Step 1: rho_hat = normalised truncated 3-D Gaussian (x) rho, clamp-to-edge. */
static void gauss1d(double sigma, double delta, int* r, double** w)
{
    int rr = sigma > 0 ? (int)ceil(3.0 * sigma / delta) : 0;
    double* ww = (double*)malloc(sizeof(double) * (2 * rr + 1));
    for (int j = -rr; j <= rr; ++j)
        ww[j + rr] = sigma > 0 ? exp(-(j * delta) * (j * delta) / (2.0 * sigma * sigma)) : 1.0;
    *r = rr; *w = ww;
}

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

void or_smooth(const double* rho, int nx, int ny, int nz, double dx, double dy, double dz,
               double sigma, double* out, int nthreads)
{
    int rx, ry, rz;
    double *wx, *wy, *wz;
    gauss1d(sigma, dx, &rx, &wx);
    gauss1d(sigma, dy, &ry, &wy);
    gauss1d(sigma, dz, &rz, &wz);
    double norm = 0.0;   /* sum of the 3-D kernel's weights */
    for (int c = -rz; c <= rz; ++c)
        for (int b = -ry; b <= ry; ++b)
            for (int a = -rx; a <= rx; ++a) norm += wx[a + rx] * wy[b + ry] * wz[c + rz];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double s = 0.0;
                for (int c = -rz; c <= rz; ++c)
                    for (int b = -ry; b <= ry; ++b)
                        for (int a = -rx; a <= rx; ++a) {
                            int ii = clampi(i + a, 0, nx - 1), jj = clampi(j + b, 0, ny - 1),
                                kk = clampi(k + c, 0, nz - 1);
                            s += wx[a + rx] * wy[b + ry] * wz[c + rz] *
                                 rho[((size_t)kk * ny + jj) * nx + ii];
                        }
                out[((size_t)k * ny + j) * nx + i] = s / norm;
            }
    free(wx); free(wy); free(wz);
}

/* ------------------------------------------------------------------------ */
/* Beam frame and beamlet geometry (steps 2-3).  The beam's eye frame at
 * gantry 0 is e_x' = +x, e_y' = +z, beam direction e_z' = +y; it is turned by
 * the gantry about +z, then by the couch about +y; the collimator turns e_x',
 * e_y' about e_z'. */
static void rot_z(double a, double* v)
{
    double c = cos(a), s = sin(a), x = v[0], y = v[1];
    v[0] = c * x - s * y; v[1] = s * x + c * y;
}
static void rot_y(double a, double* v)
{
    double c = cos(a), s = sin(a), x = v[0], z = v[2];
    v[0] = c * x + s * z; v[2] = -s * x + c * z;
}

static void beam_frame(const double* bp, OBeam* B)
{
    const double deg = M_PI / 180.0;
    double ex[3] = {1, 0, 0}, ey[3] = {0, 0, 1}, ez[3] = {0, 1, 0};
    rot_z(bp[0] * deg, ex); rot_z(bp[0] * deg, ey); rot_z(bp[0] * deg, ez);
    rot_y(bp[1] * deg, ex); rot_y(bp[1] * deg, ey); rot_y(bp[1] * deg, ez);
    double c = cos(bp[2] * deg), s = sin(bp[2] * deg);
    for (int q = 0; q < 3; ++q) {
        B->ex[q] = c * ex[q] + s * ey[q];
        B->ey[q] = -s * ex[q] + c * ey[q];
        B->ez[q] = ez[q];
    }
    B->sad = bp[3];
    for (int q = 0; q < 3; ++q) B->src[q] = bp[4 + q] - bp[3] * B->ez[q];
}

/* ------------------------------------------------------------------------ */
/* Steps 4-6: Siddon's parametric ray through the voxel grid.  All crossing
 * parameters alpha (distance from the source) of the ray with the x, y and z
 * voxel-boundary planes inside the grid are collected, merged in order, and
 * each interval between consecutive crossings is assigned the voxel that holds
 * its midpoint (Siddon 1985). */
typedef struct { double a0, a1; int64_t vox; } Seg;

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Returns the number of segments (0 if the ray misses the grid); *segs is malloc'ed. */
static int siddon(const OInputs* in, const double* s, const double* n, Seg** segs)
{
    int dims[3] = {in->nx, in->ny, in->nz};
    double del[3] = {in->dx, in->dy, in->dz}, org[3] = {in->ox, in->oy, in->oz};
    double amin = 0.0, amax = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double p0 = org[a] - 0.5 * del[a], p1 = org[a] + (dims[a] - 0.5) * del[a];
        if (fabs(n[a]) < 1e-15) {
            if (s[a] <= p0 || s[a] >= p1) { *segs = NULL; return 0; }
            continue;
        }
        double t0 = (p0 - s[a]) / n[a], t1 = (p1 - s[a]) / n[a];
        double lo = t0 < t1 ? t0 : t1, hi = t0 < t1 ? t1 : t0;
        if (lo > amin) amin = lo;
        if (hi < amax) amax = hi;
    }
    if (!(amin < amax)) { *segs = NULL; return 0; }
    int cap = 2 + dims[0] + dims[1] + dims[2] + 3;
    double* al = (double*)malloc(sizeof(double) * cap);
    int na = 0;
    al[na++] = amin;
    al[na++] = amax;
    for (int a = 0; a < 3; ++a) {
        if (fabs(n[a]) < 1e-15) continue;
        for (int i = 0; i <= dims[a]; ++i) {
            double alpha = (org[a] + (i - 0.5) * del[a] - s[a]) / n[a];
            if (alpha > amin && alpha < amax) al[na++] = alpha;
        }
    }
    qsort(al, na, sizeof(double), cmp_double);
    Seg* sg = (Seg*)malloc(sizeof(Seg) * (na > 0 ? na : 1));
    int ns = 0;
    for (int q = 0; q + 1 < na; ++q) {
        double a0 = al[q], a1 = al[q + 1];
        if (!(a1 > a0)) continue;
        double am = 0.5 * (a0 + a1);
        int idx[3];
        for (int a = 0; a < 3; ++a) {
            double pos = s[a] + am * n[a];
            idx[a] = clampi((int)floor((pos - (org[a] - 0.5 * del[a])) / del[a]), 0, dims[a] - 1);
        }
        sg[ns].a0 = a0; sg[ns].a1 = a1;
        sg[ns].vox = ((int64_t)idx[2] * in->ny + idx[1]) * in->nx + idx[0];
        ++ns;
    }
    free(al);
    *segs = sg;
    return ns;
}

/* Integral over [lo, hi] of a piecewise-constant integrand val[q] on segments. */
static double seg_integral(const Seg* sg, int ns, const double* val, double lo, double hi)
{
    double s = 0.0;
    for (int q = 0; q < ns; ++q) {
        double a = sg[q].a0 > lo ? sg[q].a0 : lo;
        double b = sg[q].a1 < hi ? sg[q].a1 : hi;
        if (b > a) s += val[q] * (b - a);
    }
    return s;
}

/* Steps 4-6 for one ray: entry/exit on the body surface and the tables
 * t_eq(k d) = int rho, omega_i^corr(k d) = int b_i(rho).  The tables are
 * malloc'ed into *T, *W1, *W2 (K samples). */
static void trace(const OPlan* P, const double* s, const double* n, int* hit, double* L_in,
                  double* L_out, int* K, double** T, double** W1, double** W2)
{
    const OInputs* in = &P->in;
    Seg* sg;
    int ns = siddon(in, s, n, &sg);
    int first = -1, last = -1;
    for (int q = 0; q < ns; ++q)
        if (P->rho[sg[q].vox] > in->rho_surf) { if (first < 0) first = q; last = q; }
    *T = *W1 = *W2 = NULL;
    if (first < 0) { *hit = 0; *L_in = *L_out = 0; *K = 0; free(sg); return; }
    *hit = 1;
    *L_in = sg[first].a0;
    *L_out = sg[last].a1;
    double tout = *L_out - *L_in;
    int k = (int)ceil(tout / P->d) + 1;
    if (k < 2) k = 2;
    *K = k;
    double* vr = (double*)malloc(sizeof(double) * (ns > 0 ? ns : 1));
    double* v1 = (double*)malloc(sizeof(double) * (ns > 0 ? ns : 1));
    double* v2 = (double*)malloc(sizeof(double) * (ns > 0 ? ns : 1));
    const double* dens = P->dens;
    for (int q = 0; q < ns; ++q) {
        double r = P->rho[sg[q].vox];
        vr[q] = r;
        v1[q] = or_lut1(dens + 4 * (size_t)in->f_n, in->f_n, in->f_rho0, in->f_drho, r);
        v2[q] = or_lut1(dens + 5 * (size_t)in->f_n, in->f_n, in->f_rho0, in->f_drho, r);
    }
    *T = (double*)malloc(sizeof(double) * k);
    *W1 = (double*)malloc(sizeof(double) * k);
    *W2 = (double*)malloc(sizeof(double) * k);
    for (int j = 0; j < k; ++j) {
        double hi = *L_in + j * P->d;
        (*T)[j] = seg_integral(sg, ns, vr, *L_in, hi);
        (*W1)[j] = seg_integral(sg, ns, v1, *L_in, hi);
        (*W2)[j] = seg_integral(sg, ns, v2, *L_in, hi);
    }
    free(vr); free(v1); free(v2); free(sg);
}

/* Exposed for the tests: trace one arbitrary ray. */
int or_trace_ray(const void* h, const double* s, const double* n, double* L_in, double* L_out,
                 double* T, double* W1, double* W2, int kmax)
{
    const OPlan* P = (const OPlan*)h;
    int hit, K;
    double *t, *w1, *w2;
    trace(P, s, n, &hit, L_in, L_out, &K, &t, &w1, &w2);
    if (!hit) return 0;
    for (int j = 0; j < K && j < kmax; ++j) { T[j] = t[j]; W1[j] = w1[j]; W2[j] = w2[j]; }
    free(t); free(w1); free(w2);
    return K;
}

/* Lookup in a beamlet table at geometric depth t (linear between samples). */
static double lut_tab(const double* tab, int K, double d, double t)
{
    return or_lut1(tab, K, 0.0, d, t);
}

/* ------------------------------------------------------------------------ */
void* or_plan_create(const OInputs* in, int nthreads)
{
    OPlan* P = (OPlan*)calloc(1, sizeof(OPlan));
    P->in = *in;
    P->V = (int64_t)in->nx * in->ny * in->nz;
    P->rho = (double*)malloc(sizeof(double) * P->V);
    memcpy(P->rho, in->rho, sizeof(double) * P->V);
    size_t na = (size_t)in->a_nt * in->a_nth, nw = 4 * (size_t)in->w_n, nf = 6 * (size_t)in->f_n;
    P->A = (double*)malloc(sizeof(double) * na);  memcpy(P->A, in->A, sizeof(double) * na);
    P->water = (double*)malloc(sizeof(double) * nw); memcpy(P->water, in->water, sizeof(double) * nw);
    P->dens = (double*)malloc(sizeof(double) * nf); memcpy(P->dens, in->dens, sizeof(double) * nf);
    P->beamraw = (double*)malloc(sizeof(double) * 10 * in->n_beams);
    memcpy(P->beamraw, in->beams, sizeof(double) * 10 * in->n_beams);
    P->in.rho = P->rho; P->in.A = P->A; P->in.water = P->water; P->in.dens = P->dens;
    P->in.beams = P->beamraw;

    /* step 1 */
    P->rhos = (double*)malloc(sizeof(double) * P->V);
    or_smooth(P->rho, in->nx, in->ny, in->nz, in->dx, in->dy, in->dz, in->sigma, P->rhos, nthreads);

    /* sampling step of Section 2.2 */
    double d = in->dx < in->dy ? in->dx : in->dy;
    d = d < in->dz ? d : in->dz;
    P->d = 0.5 * d;

    /* steps 2-6 */
    P->beam = (OBeam*)calloc(in->n_beams, sizeof(OBeam));
    int B = 0;
    for (int b = 0; b < in->n_beams; ++b) {
        OBeam* bm = &P->beam[b];
        beam_frame(P->beamraw + 10 * b, bm);
        bm->M = (int)lround(P->beamraw[10 * b + 7] / in->bx);
        bm->N = (int)lround(P->beamraw[10 * b + 8] / in->by);
        bm->first = B;
        B += bm->M * bm->N;
    }
    P->B = B;
    P->bl = (OBeamlet*)calloc(B > 0 ? B : 1, sizeof(OBeamlet));
    for (int b = 0; b < in->n_beams; ++b) {
        OBeam* bm = &P->beam[b];
        const double* iso = P->beamraw + 10 * b + 4;
        double fx = P->beamraw[10 * b + 7], fy = P->beamraw[10 * b + 8];
        for (int nn = 0; nn < bm->N; ++nn)
            for (int m = 0; m < bm->M; ++m) {
                OBeamlet* bl = &P->bl[bm->first + nn * bm->M + m];
                bl->beam = b;
                double a = -0.5 * fx + (m + 0.5) * in->bx;
                double c = -0.5 * fy + (nn + 0.5) * in->by;
                double pt[3];
                for (int q = 0; q < 3; ++q) {
                    pt[q] = iso[q] + a * bm->ex[q] + c * bm->ey[q];
                    bl->n[q] = pt[q] - bm->src[q];
                }
                normalize3(bl->n);
                bl->theta = atan2(sqrt(a * a + c * c), bm->sad);      /* step 3 */
                double en = dot3(bm->ex, bl->n);
                for (int q = 0; q < 3; ++q) bl->ex[q] = bm->ex[q] - en * bl->n[q];
                normalize3(bl->ex);
                cross3(bl->ex, bl->n, bl->ey);
            }
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int i = 0; i < B; ++i) {
        OBeamlet* bl = &P->bl[i];
        trace(P, P->beam[bl->beam].src, bl->n, &bl->hit, &bl->L_in, &bl->L_out, &bl->K, &bl->T,
              &bl->W1, &bl->W2);
    }
    return P;
}

void or_plan_destroy(void* h)
{
    OPlan* P = (OPlan*)h;
    if (!P) return;
    for (int i = 0; i < P->B; ++i) { free(P->bl[i].T); free(P->bl[i].W1); free(P->bl[i].W2); }
    free(P->bl); free(P->beam); free(P->rho); free(P->rhos); free(P->A); free(P->water);
    free(P->dens); free(P->beamraw); free(P);
}

int or_plan_n_beamlets(const void* h) { return ((const OPlan*)h)->B; }
double or_plan_step(const void* h) { return ((const OPlan*)h)->d; }

void or_plan_smoothed(const void* h, double* out)
{
    const OPlan* P = (const OPlan*)h;
    memcpy(out, P->rhos, sizeof(double) * P->V);
}

/* rec: n[3], ex[3], ey[3], theta, hit, L_in, L_out, K, src[3] (17 values). */
void or_plan_beamlet(const void* h, int i, double* rec)
{
    const OPlan* P = (const OPlan*)h;
    const OBeamlet* bl = &P->bl[i];
    for (int q = 0; q < 3; ++q) { rec[q] = bl->n[q]; rec[3 + q] = bl->ex[q]; rec[6 + q] = bl->ey[q]; }
    rec[9] = bl->theta; rec[10] = bl->hit; rec[11] = bl->L_in; rec[12] = bl->L_out; rec[13] = bl->K;
    for (int q = 0; q < 3; ++q) rec[14 + q] = P->beam[bl->beam].src[q];
}

int or_plan_table(const void* h, int i, double* T, double* W1, double* W2, int kmax)
{
    const OPlan* P = (const OPlan*)h;
    const OBeamlet* bl = &P->bl[i];
    for (int j = 0; j < bl->K && j < kmax; ++j) { T[j] = bl->T[j]; W1[j] = bl->W1[j]; W2[j] = bl->W2[j]; }
    return bl->K;
}

/* ------------------------------------------------------------------------ */
/* Lateral density sampling along the beam's axes (the "AXIS" form of the
 * step-11 correction; with lateral_mode = 0 the paper's rho(r), rho_hat(r) are
 * used instead).  For voxel r and beam b, 16 taps along each of the beam's
 * axes e_x', e_y', e_z' through r at s_j = (j + 1/2) d, j = -8..7; at each tap
 * the density is interpolated trilinearly (clamp-to-edge); per axis the taps
 * are averaged with Gaussian weights exp(-s_j^2 / 2 sigma^2) normalised to one.
 * eff = (mean of the three axis averages, x-axis average, y-axis average): the
 * densities at which f_omega, f_u2 along x and f_u2 along y are taken.
 * Optionally returns the 48 taps (axis-major) and the 48 nearest-voxel
 * densities at the same points. */
#define N_TAPS 16

static double rho_trilinear(const OPlan* P, const double* p)
{
    const OInputs* in = &P->in;
    const int dims[3] = {in->nx, in->ny, in->nz};
    const double del[3] = {in->dx, in->dy, in->dz}, org[3] = {in->ox, in->oy, in->oz};
    int i0[3], i1[3];
    double w[3];
    for (int a = 0; a < 3; ++a) {
        double u = (p[a] - org[a]) / del[a];
        if (u < 0) u = 0;
        if (u > dims[a] - 1) u = dims[a] - 1;
        int f = (int)floor(u);
        if (f > dims[a] - 2) f = dims[a] - 2;
        if (f < 0) f = 0;
        i0[a] = f;
        i1[a] = dims[a] > 1 ? f + 1 : f;
        w[a] = dims[a] > 1 ? u - f : 0.0;
    }
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
        int ix = (c & 1) ? i1[0] : i0[0], iy = (c & 2) ? i1[1] : i0[1], iz = (c & 4) ? i1[2] : i0[2];
        double wt = ((c & 1) ? w[0] : 1 - w[0]) * ((c & 2) ? w[1] : 1 - w[1]) * ((c & 4) ? w[2] : 1 - w[2]);
        s += wt * P->rho[((size_t)iz * in->ny + iy) * in->nx + ix];
    }
    return s;
}

static double rho_nearest(const OPlan* P, const double* p)
{
    const OInputs* in = &P->in;
    const int dims[3] = {in->nx, in->ny, in->nz};
    const double del[3] = {in->dx, in->dy, in->dz}, org[3] = {in->ox, in->oy, in->oz};
    int id[3];
    for (int a = 0; a < 3; ++a) id[a] = clampi((int)floor((p[a] - org[a]) / del[a] + 0.5), 0, dims[a] - 1);
    return P->rho[((size_t)id[2] * in->ny + id[1]) * in->nx + id[0]];
}

static void axis_densities(const OPlan* P, int64_t v, int beam, double* taps, double* nearest, double* eff)
{
    const OInputs* in = &P->in;
    const OBeam* bm = &P->beam[beam];
    int64_t ii = v % in->nx, jj = (v / in->nx) % in->ny, kk = v / ((int64_t)in->nx * in->ny);
    double r[3] = {in->ox + ii * in->dx, in->oy + jj * in->dy, in->oz + kk * in->dz};
    const double* axes[3] = {bm->ex, bm->ey, bm->ez};
    double avg[3];
    for (int a = 0; a < 3; ++a) {
        double sw = 0.0, s = 0.0;
        for (int j = -N_TAPS / 2; j < N_TAPS / 2; ++j) {
            double sj = (j + 0.5) * P->d;
            double p[3] = {r[0] + sj * axes[a][0], r[1] + sj * axes[a][1], r[2] + sj * axes[a][2]};
            double rv = rho_trilinear(P, p);
            double g = in->sigma > 0 ? exp(-sj * sj / (2.0 * in->sigma * in->sigma)) : 1.0;
            if (taps) taps[a * N_TAPS + j + N_TAPS / 2] = rv;
            if (nearest) nearest[a * N_TAPS + j + N_TAPS / 2] = rho_nearest(P, p);
            s += g * rv;
            sw += g;
        }
        avg[a] = s / sw;
    }
    eff[0] = (avg[0] + avg[1] + avg[2]) / 3.0;
    eff[1] = avg[0];
    eff[2] = avg[1];
}

/* Exposed for the tests: the stencil of (voxel v, beam b). */
void or_plan_axis_stencil(const void* h, int64_t v, int beam, double* taps48, double* nearest48, double* eff3)
{
    axis_densities((const OPlan*)h, v, beam, taps48, nearest48, eff3);
}

/* ------------------------------------------------------------------------ */
/* Steps 8-12 for one (voxel, beamlet) pair.  Returns 1 if the pair is in the
 * beamlet's ROI and depth range, 0 otherwise; *amb is set when either
 * decision lies within the rounding margin of its boundary.  *D is D_i(r) of
 * eq. (2) for unit fluence (also evaluated for ambiguous pairs outside).
 * out6 (optional): x, y, t, t_eq, |r_a|, |perp|^2. */
static int pair_dose(const OPlan* P, int64_t v, int i, double* D, int* amb, double* out6)
{
    const OInputs* in = &P->in;
    const OBeamlet* bl = &P->bl[i];
    const OBeam* bm = &P->beam[bl->beam];
    *D = 0.0; *amb = 0;
    if (!bl->hit) return 0;
    int64_t ii = v % in->nx, jj = (v / in->nx) % in->ny, kk = v / ((int64_t)in->nx * in->ny);
    double r[3] = {in->ox + ii * in->dx, in->oy + jj * in->dy, in->oz + kk * in->dz};
    double w[3] = {r[0] - bm->src[0], r[1] - bm->src[1], r[2] - bm->src[2]};
    double L = dot3(w, bl->n);                 /* |r_a| */
    double perp[3] = {w[0] - L * bl->n[0], w[1] - L * bl->n[1], w[2] - L * bl->n[2]};
    double q2 = dot3(perp, perp);
    double t = L - bl->L_in;
    double tout = bl->L_out - bl->L_in;
    double R2 = in->roi * in->roi;
    int inside = (q2 <= R2) && (t >= 0.0) && (t <= tout);
    int near = (fabs(q2 - R2) < EPS_Q) || (fabs(t) < EPS_T) || (fabs(t - tout) < EPS_T);
    int cand = (q2 <= R2 + EPS_Q) && (t >= -EPS_T) && (t <= tout + EPS_T);
    if (!inside && !(near && cand)) return 0;
    *amb = near && cand;
    if (t < 0.0) t = 0.0;
    if (t > tout) t = tout;

    /* x, y at the isocentre plane */
    double x = dot3(perp, bl->ex) * bm->sad / L;
    double y = dot3(perp, bl->ey) * bm->sad / L;
    double x0 = 0.5 * in->bx, y0 = 0.5 * in->by;

    /* step 5 table: radiological depth, step 6 table: omega_corr */
    double teq = lut_tab(bl->T, bl->K, P->d, t);
    double c1 = lut_tab(bl->W1, bl->K, P->d, t);
    double c2 = lut_tab(bl->W2, bl->K, P->d, t);
    /* step 9 */
    double Aval = lut_A(P, teq, bl->theta);
    /* step 10 */
    const double* wt = P->water;
    double u1w = or_lut1(wt + 0 * (size_t)in->w_n, in->w_n, 0.0, in->w_dt, t);
    double u2w = or_lut1(wt + 1 * (size_t)in->w_n, in->w_n, 0.0, in->w_dt, t);
    double w1w = or_lut1(wt + 2 * (size_t)in->w_n, in->w_n, 0.0, in->w_dt, t);
    double w2w = or_lut1(wt + 3 * (size_t)in->w_n, in->w_n, 0.0, in->w_dt, t);
    /* step 11 */
    double u1, u2x, u2y, w1, w2;
    if (in->density_correction) {
        const double* f = P->dens;
        size_t fn = (size_t)in->f_n;
        double rl = P->rho[v];
        double ru_x, ru_y, rw;   /* densities that set u_2 along x, along y, and omega */
        if (in->lateral_mode == 1) {
            double eff[3];
            axis_densities(P, v, bl->beam, NULL, NULL, eff);
            rw = eff[0]; ru_x = eff[1]; ru_y = eff[2];
        } else {
            ru_x = ru_y = rw = P->rhos[v];
        }
        u1 = or_lut1(f + 0 * fn, in->f_n, in->f_rho0, in->f_drho, rl) * u1w;
        u2x = or_lut1(f + 1 * fn, in->f_n, in->f_rho0, in->f_drho, ru_x) * u2w;
        u2y = or_lut1(f + 1 * fn, in->f_n, in->f_rho0, in->f_drho, ru_y) * u2w;
        w1 = or_lut1(f + 2 * fn, in->f_n, in->f_rho0, in->f_drho, rw) * (w1w + c1);
        w2 = or_lut1(f + 3 * fn, in->f_n, in->f_rho0, in->f_drho, rw) * (w2w + c2);
        if (w1 < 0) w1 = 0;
        if (w2 < 0) w2 = 0;
    } else {
        u1 = u1w; u2x = u2y = u2w; w1 = w1w; w2 = w2w;
    }
    /* step 12: eqs. (3) and (2) */
    double F = w1 * or_p(x, u1, x0) * or_p(y, u1, y0) + w2 * or_p(x, u2x, x0) * or_p(y, u2y, y0);
    double isq = (bm->sad / L) * (bm->sad / L);
    *D = F * Aval * isq;
    if (out6) { out6[0] = x; out6[1] = y; out6[2] = t; out6[3] = teq; out6[4] = L; out6[5] = q2; }
    return inside;
}

/* Eq. (1) for listed voxels (all voxels if vox == NULL, n = V).
 * amb (optional) receives, per voxel, the sum of |f_i D_i| over ambiguous pairs. */
void or_plan_dose_voxels(const void* h, const double* fluence, const int64_t* vox, int64_t n,
                         double* dose, double* amb, int nthreads)
{
    const OPlan* P = (const OPlan*)h;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t q = 0; q < n; ++q) {
        int64_t v = vox ? vox[q] : q;
        double s = 0.0, sa = 0.0;
        for (int i = 0; i < P->B; ++i) {       /* step 8 */
            double D;
            int a;
            int inside = pair_dose(P, v, i, &D, &a, NULL);
            if (inside) s += fluence[i] * D;
            if (a) sa += fabs(fluence[i] * D);
        }
        dose[q] = s;
        if (amb) amb[q] = sa;
    }
}

void or_plan_dose(const void* h, const double* fluence, double* dose, double* amb, int nthreads)
{
    const OPlan* P = (const OPlan*)h;
    or_plan_dose_voxels(h, fluence, NULL, P->V, dose, amb, nthreads);
}

/* Single pair: out[0] = D_i(r_v), out[1] = inside, out[2] = ambiguous,
 * out[3..8] = x, y, t, t_eq, |r_a|, |perp|^2. */
void or_plan_pair(const void* h, int64_t v, int i, double* out)
{
    int a;
    double D;
    out[3] = out[4] = out[5] = out[6] = out[7] = out[8] = 0.0;
    int inside = pair_dose((const OPlan*)h, v, i, &D, &a, out + 3);
    out[0] = D; out[1] = inside; out[2] = a;
}

/* Number of pairs (inside ROI and depth range) at listed voxels. */
void or_plan_pairs_voxels(const void* h, const int64_t* vox, int64_t n, int64_t* counts, int nthreads)
{
    const OPlan* P = (const OPlan*)h;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t q = 0; q < n; ++q) {
        int64_t c = 0;
        for (int i = 0; i < P->B; ++i) {
            double D;
            int a;
            c += pair_dose(P, vox[q], i, &D, &a, NULL);
        }
        counts[q] = c;
    }
}

/* Dose-deposition matrix M[v, i] = D_i(r_v) by voxel rows, columns ascending,
 * for the listed voxels (all voxels if vox == NULL, n = V).
 * Counting pass: per row, the number of candidate entries (inside or ambiguous). */
void or_plan_matrix_count(const void* h, const int64_t* vox, int64_t n, int64_t* counts, int nthreads)
{
    const OPlan* P = (const OPlan*)h;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t q = 0; q < n; ++q) {
        int64_t v = vox ? vox[q] : q;
        int64_t c = 0;
        for (int i = 0; i < P->B; ++i) {
            double D;
            int a;
            int inside = pair_dose(P, v, i, &D, &a, NULL);
            if (inside || a) ++c;
        }
        counts[q] = c;
    }
}

/* Fill pass: flags bit 0 = inside, bit 1 = ambiguous. */
void or_plan_matrix_fill(const void* h, const int64_t* vox, int64_t n, const int64_t* rowptr,
                         int32_t* cols, double* vals, uint8_t* flags, int nthreads)
{
    const OPlan* P = (const OPlan*)h;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int64_t q = 0; q < n; ++q) {
        int64_t v = vox ? vox[q] : q;
        int64_t o = rowptr[q];
        for (int i = 0; i < P->B; ++i) {
            double D;
            int a;
            int inside = pair_dose(P, v, i, &D, &a, NULL);
            if (inside || a) {
                cols[o] = i; vals[o] = D; flags[o] = (uint8_t)(inside | (a << 1)); ++o;
            }
        }
    }
}
