/*
 * FP64 CPU oracle: beamlet fluence from MLC leaf sequences (Gu et al.,
 * arXiv 1103.1164, Section 2.3: the plans' leaf sequences and monitor units
 * were converted into fluence maps on the 0.2 x 0.5 cm beamlet grid, 0.2 cm
 * along the leaf motion).
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: only the tests, the smoke check
 * and the CPU legs of the benchmark load it.  It shares no code with the CUDA
 * path.
 *
 * What it computes (the paper gives no formula; the reading is the plain
 * definition of delivered fluence):
 *   fluence_i = 1/(bx by) * sum over leaf pairs j, control-point intervals c of
 *       h_ij * [ (1 - tau) * |P_jc clipped to the beamlet's x-range|
 *                + tau * (x-range length) * (mu_c+1 - mu_c) ]
 * where the beamlet's rectangle is first clipped to the jaws, h_ij is the
 * length of its y-range inside leaf pair j, and P_jc is the region of the
 * (x, mu) plane that leaf pair j leaves open while the meterset runs from
 * mu_c to mu_c+1: the quadrilateral (l_c, mu_c), (r_c, mu_c), (r_c+1, mu_c+1),
 * (l_c+1, mu_c+1), leaf tips moving linearly in mu between control points.
 * A step-and-shoot segment is two control points with equal leaf positions;
 * the leaf moves between segments happen at a repeated meterset value (an
 * interval of zero length, which delivers nothing).  Fluence is in meterset
 * units (MU times the open fraction).
 *
 * The clipped area is computed as the definition reads: the quadrilateral is
 * clipped by the half-planes x >= xa and x <= xb (Sutherland-Hodgman) and its
 * area taken by the shoelace formula.
 */
#include <math.h>
#include <stdint.h>

/* Clips polygon (px, py)[n] against x >= c (side = +1) or x <= c (side = -1);
 * writes at most n + 1 vertices to (qx, qy) and returns their count. */
static int clip_x(const double* px, const double* py, int n, double c, int side, double* qx, double* qy)
{
    int m = 0;
    for (int k = 0; k < n; ++k) {
        const int k1 = (k + 1) % n;
        const double ax = px[k], ay = py[k], bx = px[k1], by = py[k1];
        const int ain = side > 0 ? ax >= c : ax <= c;
        const int bin = side > 0 ? bx >= c : bx <= c;
        if (ain) {
            qx[m] = ax;
            qy[m] = ay;
            ++m;
        }
        if (ain != bin) {
            /* the edge crosses x = c */
            const double s = (c - ax) / (bx - ax);
            qx[m] = c;
            qy[m] = ay + s * (by - ay);
            ++m;
        }
    }
    return m;
}

static double shoelace(const double* x, const double* y, int n)
{
    double a = 0.0;
    for (int k = 0; k < n; ++k) {
        const int k1 = (k + 1) % n;
        a += x[k] * y[k1] - x[k1] * y[k];
    }
    return 0.5 * fabs(a);
}

/* Area of the quadrilateral (l0, m0), (r0, m0), (r1, m1), (l1, m1) between
 * x = xa and x = xb. */
double or_open_area(double l0, double r0, double l1, double r1, double m0, double m1, double xa, double xb)
{
    double px[4] = {l0, r0, r1, l1}, py[4] = {m0, m0, m1, m1};
    double qx[5], qy[5], sx[6], sy[6];
    const int n1 = clip_x(px, py, 4, xa, +1, qx, qy);
    if (n1 < 3) return 0.0;
    const int n2 = clip_x(qx, qy, n1, xb, -1, sx, sy);
    if (n2 < 3) return 0.0;
    return shoelace(sx, sy, n2);
}

static double overlap(double a0, double a1, double b0, double b1)
{
    const double lo = a0 > b0 ? a0 : b0, hi = a1 < b1 ? a1 : b1;
    return hi > lo ? hi - lo : 0.0;
}

/*
 * Fluence of the M x N beamlets of one beam (beamlet (m, n) at out[n M + m],
 * its rectangle [-field_x/2 + m bx, ... + bx] x [-field_y/2 + n by, ... + by]
 * in the isocentre plane of the collimator frame).
 *   edges [n_leaves + 1]   leaf-pair boundaries along y (increasing)
 *   mu    [n_cp]           cumulative meterset (non-decreasing)
 *   left, right [n_cp][n_leaves]  leaf tip positions along x, left <= right
 *   jaws  [4]              x1, x2, y1, y2
 */
void or_leaf_fluence(int M, int N, double field_x, double field_y, double bx, double by,
                     int n_leaves, int n_cp, const double* edges, const double* mu,
                     const double* left, const double* right, const double* jaws, double tau,
                     double* out, int nthreads)
{
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t e = 0; e < (int64_t)M * N; ++e) {
        const int m = (int)(e % M), n = (int)(e / M);
        double xa = -0.5 * field_x + m * bx, xb = xa + bx;
        double ya = -0.5 * field_y + n * by, yb = ya + by;
        if (xa < jaws[0]) xa = jaws[0];
        if (xb > jaws[1]) xb = jaws[1];
        if (ya < jaws[2]) ya = jaws[2];
        if (yb > jaws[3]) yb = jaws[3];
        double total = 0.0;
        if (xb > xa && yb > ya) {
            for (int j = 0; j < n_leaves; ++j) {
                const double h = overlap(ya, yb, edges[j], edges[j + 1]);
                if (h <= 0.0) continue;
                for (int c = 0; c + 1 < n_cp; ++c) {
                    const double dmu = mu[c + 1] - mu[c];
                    if (!(dmu > 0.0)) continue;
                    const double open = or_open_area(left[(int64_t)c * n_leaves + j], right[(int64_t)c * n_leaves + j],
                                                     left[(int64_t)(c + 1) * n_leaves + j],
                                                     right[(int64_t)(c + 1) * n_leaves + j], mu[c], mu[c + 1], xa, xb);
                    total += h * ((1.0 - tau) * open + tau * (xb - xa) * dmu);
                }
            }
        }
        out[e] = total / (bx * by);
    }
}
