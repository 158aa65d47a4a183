// Per-plan pre-pass kernels of the DC-FSPB engine:
//   smoothing of the density (Algorithm A1 step 1 / A2 Kernel 1),
//   per-voxel density-correction factors (the rho-dependent part of step 11),
//   beamlet geometry, body entry/exit and depth tables (steps 2-6 / Kernels 2-4).
#include <math.h>

#include "dc_internal.cuh"

namespace dc {
namespace {

constexpr int kMaxSmoothRadius = 64;

struct SmoothArgs {
    const float* in;
    float* out;
    int nx, ny, nz, r;
    float w[2 * kMaxSmoothRadius + 1];
};

// One axis of the separable Gaussian (clamp-to-edge).  Threads run along x,
// so the y and z passes read coalesced rows and the x pass hits L1.
template <int AXIS>
__global__ void __launch_bounds__(256) k_smooth_axis(const SmoothArgs a)
{
    int64_t V = (int64_t)a.nx * a.ny * a.nz;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
         v += (int64_t)gridDim.x * blockDim.x) {
        // plan grids hold at most 2^31 voxels: 32-bit division
        const uint32_t u = (uint32_t)v, qx = u / (uint32_t)a.nx;
        int i = (int)(u - qx * (uint32_t)a.nx);
        int j = (int)(qx % (uint32_t)a.ny);
        int k = (int)(qx / (uint32_t)a.ny);
        float s = 0.f;
        for (int q = -a.r; q <= a.r; ++q) {
            int ii = i, jj = j, kk = k;
            if (AXIS == 0) ii = min(max(i + q, 0), a.nx - 1);
            if (AXIS == 1) jj = min(max(j + q, 0), a.ny - 1);
            if (AXIS == 2) kk = min(max(k + q, 0), a.nz - 1);
            s = fmaf(a.w[q + a.r], __ldg(a.in + ((int64_t)kk * a.ny + jj) * a.nx + ii), s);
        }
        a.out[v] = s;
    }
}

__device__ __forceinline__ float lut1(const float* f, int n, float x0, float inv_h, float x)
{
    float s = fminf(fmaxf((x - x0) * inv_h, 0.f), (float)(n - 1));
    int j = min((int)s, n - 2);
    float w = s - (float)j;
    float f0 = __ldg(f + j), f1 = __ldg(f + j + 1);
    return fmaf(w, f1 - f0, f0);
}

__global__ void __launch_bounds__(256) k_factors(const float* __restrict__ rho,
                                                 const float* __restrict__ rhos,
                                                 const float* __restrict__ dens, int f_n,
                                                 float f_rho0, float inv_drho, int dc, int64_t V,
                                                 float4* __restrict__ fac)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V;
         v += (int64_t)gridDim.x * blockDim.x) {
        float4 f = make_float4(1.f, 1.f, 1.f, 1.f);
        if (dc) {
            float r = __ldg(rho + v), rs = __ldg(rhos + v);
            f.x = lut1(dens + 0 * (size_t)f_n, f_n, f_rho0, inv_drho, r);
            f.y = lut1(dens + 1 * (size_t)f_n, f_n, f_rho0, inv_drho, rs);
            f.z = lut1(dens + 2 * (size_t)f_n, f_n, f_rho0, inv_drho, rs);
            f.w = lut1(dens + 3 * (size_t)f_n, f_n, f_rho0, inv_drho, rs);
        }
        fac[v] = f;
    }
}

// ---------------------------------------------------------------------------
// Beamlet geometry + FP64 Siddon ray trace + depth tables, one thread per beamlet.

struct BeamletArgs {
    const dc_beam* beams;
    const float* rho;
    const float* dens;
    int f_n;
    float f_rho0, inv_drho;
    int nx, ny, nz, B, n_beams, Kmax;
    double dx, dy, dz, ox, oy, oz, d;
    double idx, idy, idz;    // 1 / voxel size
    double inv_d;            // 1 / d
    double bx, by;
    float rho_surf;
    int a_nth;
    float inv_adth;
    BeamDev* out_beams;
    BeamletDev* out_bl;
    float* out_theta;
    double* ray;             // [B][8] FP64 axis source and direction (k_beamlets -> k_trace)
    float2* lio;             // [B] (L_in, L_out) for the binning bounds (k_trace)
    float4* tab;
    int first[kMaxBeams + 1];
    int M[kMaxBeams];
};

__device__ __forceinline__ void rot_z(double a, double* v)
{
    double c = cos(a), s = sin(a), x = v[0], y = v[1];
    v[0] = c * x - s * y;
    v[1] = s * x + c * y;
}
__device__ __forceinline__ void rot_y(double a, double* v)
{
    double c = cos(a), s = sin(a), x = v[0], z = v[2];
    v[0] = c * x + s * z;
    v[2] = -s * x + c * z;
}

// Incremental (Amanatides-Woo form of Siddon's) voxel walk of the ray s + a n,
// a in [amin, amax], calling visit(a0, a1, voxel) for every segment of positive
// length.  The crossing parameters are FP64.
struct Walk {
    int idx[3], step[3];
    double anext[3], adelta[3];
    double acur, amax;
};

// 1 / n[a] per axis (0 where the axis is parallel to the ray): the walk
// multiplies by these instead of dividing (FP64 division is a long sequence
// on this GPU, whose FP64 rate is a small fraction of its FP32 rate).
__device__ __forceinline__ void ray_inverse(const double* n, double* inv_n)
{
    for (int a = 0; a < 3; ++a) inv_n[a] = fabs(n[a]) < 1e-15 ? 0.0 : 1.0 / n[a];
}

__device__ bool walk_init(const BeamletArgs& A, const double* s, const double* n, const double* inv_n, Walk& w)
{
    const int dims[3] = {A.nx, A.ny, A.nz};
    const double del[3] = {A.dx, A.dy, A.dz};
    const double idel[3] = {A.idx, A.idy, A.idz};
    const double org[3] = {A.ox, A.oy, A.oz};
    double amin = 0.0, amax = 1e300;
    for (int a = 0; a < 3; ++a) {
        double p0 = org[a] - 0.5 * del[a], p1 = org[a] + (dims[a] - 0.5) * del[a];
        if (fabs(n[a]) < 1e-15) {
            if (s[a] <= p0 || s[a] >= p1) return false;
            continue;
        }
        double t0 = (p0 - s[a]) * inv_n[a], t1 = (p1 - s[a]) * inv_n[a];
        amin = fmax(amin, fmin(t0, t1));
        amax = fmin(amax, fmax(t0, t1));
    }
    if (!(amin < amax)) return false;
    for (int a = 0; a < 3; ++a) {
        double p0 = org[a] - 0.5 * del[a];
        double pos = s[a] + amin * n[a];
        double f = (pos - p0) * idel[a];
        int id = (int)floor(f);
        if (n[a] < 0 && f == floor(f)) id -= 1;
        id = min(max(id, 0), dims[a] - 1);
        w.idx[a] = id;
        if (fabs(n[a]) < 1e-15) {
            w.step[a] = 0;
            w.anext[a] = 1e300;
            w.adelta[a] = 1e300;
        } else if (n[a] > 0) {
            w.step[a] = 1;
            w.anext[a] = (p0 + (id + 1) * del[a] - s[a]) * inv_n[a];
            w.adelta[a] = del[a] * inv_n[a];
        } else {
            w.step[a] = -1;
            w.anext[a] = (p0 + id * del[a] - s[a]) * inv_n[a];
            w.adelta[a] = -del[a] * inv_n[a];
        }
    }
    w.acur = amin;
    w.amax = amax;
    return true;
}

// The walk state at a_start on the ray s + a n, to run up to a_end (both
// inside [amin, amax] of walk_init): the voxel holding the ray just past
// a_start and the next plane crossing along each axis.
__device__ void walk_from(const BeamletArgs& A, const double* s, const double* n, const double* inv_n,
                          double a_start, double a_end, Walk& w)
{
    const int dims[3] = {A.nx, A.ny, A.nz};
    const double del[3] = {A.dx, A.dy, A.dz};
    const double idel[3] = {A.idx, A.idy, A.idz};
    const double org[3] = {A.ox, A.oy, A.oz};
    for (int a = 0; a < 3; ++a) {
        const double p0 = org[a] - 0.5 * del[a];
        const double f = (s[a] + a_start * n[a] - p0) * idel[a];
        int id = (int)floor(f);
        if (n[a] < 0 && f == floor(f)) id -= 1;
        id = min(max(id, 0), dims[a] - 1);
        w.idx[a] = id;
        if (fabs(n[a]) < 1e-15) {
            w.step[a] = 0;
            w.anext[a] = 1e300;
            w.adelta[a] = 1e300;
        } else if (n[a] > 0) {
            w.step[a] = 1;
            w.anext[a] = (p0 + (id + 1) * del[a] - s[a]) * inv_n[a];
            w.adelta[a] = del[a] * inv_n[a];
        } else {
            w.step[a] = -1;
            w.anext[a] = (p0 + id * del[a] - s[a]) * inv_n[a];
            w.adelta[a] = -del[a] * inv_n[a];
        }
    }
    w.acur = a_start;
    w.amax = a_end;
}

template <typename F>
__device__ void walk_run(const BeamletArgs& A, Walk w, F&& visit)
{
    const int dims[3] = {A.nx, A.ny, A.nz};
    const int maxit = A.nx + A.ny + A.nz + 8;
    for (int it = 0; it < maxit; ++it) {
        int ax = 0;
        double an = w.anext[0];
        if (w.anext[1] < an) { an = w.anext[1]; ax = 1; }
        if (w.anext[2] < an) { an = w.anext[2]; ax = 2; }
        bool last = an >= w.amax;
        if (last) an = w.amax;
        if (an > w.acur)
            visit(w.acur, an, ((int64_t)w.idx[2] * A.ny + w.idx[1]) * A.nx + w.idx[0]);
        if (last) return;
        w.idx[ax] += w.step[ax];
        if (w.idx[ax] < 0 || w.idx[ax] >= dims[ax]) return;
        w.anext[ax] += w.adelta[ax];
        w.acur = an;
    }
}

__device__ __forceinline__ float lut_dens(const BeamletArgs& A, int q, float r)
{
    return lut1(A.dens + (size_t)q * A.f_n, A.f_n, A.f_rho0, A.inv_drho, r);
}

// Steps 4-6 in one FP64 walk of the beamlet's central axis.  The body entry
// L_in is the start of the first segment whose density exceeds the surface
// threshold and L_out the end of the last one.  From L_in on, the cumulative
// integrals of rho, b_1(rho), b_2(rho) are sampled at L_in + k d and stored as
// value + slope to the next sample:
//   tab[2k] = (T_k, T_k+1 - T_k, W1_k, W1_k+1 - W1_k), tab[2k+1] = (W2_k, W2_k+1 - W2_k, 0, 0)
// with zero slope at k = K - 1, K = ceil((L_out - L_in) / d) + 1 (at least 2,
// at most Kmax).  K is known only at the end of the walk, so samples are
// emitted up to the end of the ray (or Kmax) and the table is closed at K - 1
// afterwards.  Acc is float for rays up to 40 cm in the grid and double beyond.
template <typename Acc>
__device__ void trace_beamlet(const BeamletArgs& A, const Walk& w0, float4* __restrict__ tab, double& L_in,
                              double& L_out, int& K)
{
    Acc cT = 0, c1 = 0, c2 = 0;
    float pT = 0.f, p1 = 0.f, p2 = 0.f;
    int k = 0;
    const int kcap = A.Kmax;
    double first_a = -1, last_a = -1;
    auto emit = [&](float T, float a, float b) {
        if (k > 0) {
            tab[2 * (k - 1)] = make_float4(pT, T - pT, p1, a - p1);
            tab[2 * (k - 1) + 1] = make_float4(p2, b - p2, 0.f, 0.f);
        }
        pT = T; p1 = a; p2 = b;
        ++k;
    };
    const float surf = A.rho_surf;
    walk_run(A, w0, [&](double a0, double a1, int64_t vox) {
        const float r = __ldg(A.rho + vox);
        if (r > surf) {
            if (first_a < 0) first_a = a0;
            last_a = a1;
        }
        if (first_a < 0 || k >= kcap) return;
        const double lo = fmax(a0, first_a);
        Acc vr = (Acc)r, v1 = (Acc)lut_dens(A, 4, r), v2 = (Acc)lut_dens(A, 5, r);
        while (k < kcap) {
            double sk = first_a + k * A.d;
            if (sk > a1) break;
            Acc len = (Acc)(sk - lo);
            emit((float)(cT + vr * len), (float)(c1 + v1 * len), (float)(c2 + v2 * len));
        }
        Acc len = (Acc)(a1 - lo);
        cT += vr * len;
        c1 += v1 * len;
        c2 += v2 * len;
    });
    K = 0;
    if (first_a < 0) return;
    L_in = first_a;
    L_out = last_a;
    K = max(2, (int)ceil((L_out - L_in) / A.d) + 1);
    K = min(K, kcap);
    while (k < K) emit((float)cT, (float)c1, (float)c2);
    if (k == K) {
        // sample K - 1 is still pending
        tab[2 * (K - 1)] = make_float4(pT, 0.f, p1, 0.f);
        tab[2 * (K - 1) + 1] = make_float4(p2, 0.f, 0.f, 0.f);
    } else {
        // samples past K - 1 were emitted: only the slopes of K - 1 change
        tab[2 * (K - 1)].y = 0.f;
        tab[2 * (K - 1)].w = 0.f;
        tab[2 * (K - 1) + 1].y = 0.f;
    }
}

// Merged per-beamlet tables for plans whose water tables are sampled on the
// same depth grid as the beamlet tables (w_dt == d): the water values at
// sample k are the water table's knot k (clamped at its end, where its slope
// is zero), so interpolating their sum with omega_corr in t is exactly the sum
// of the two interpolations.
__global__ void __launch_bounds__(256) k_merge_tables(const float4* __restrict__ tab,
                                                      const float4* __restrict__ water, int w_n,
                                                      const BeamletDev* __restrict__ bl, int B, int Kmax,
                                                      float wscale, float4* __restrict__ tabm)
{
    const int64_t n = (int64_t)B * Kmax;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / Kmax), k = (int)(e % Kmax);
        if (k >= __ldg(&bl[i].meta.x)) continue;
        const float4 a = __ldg(tab + 2 * e), b = __ldg(tab + 2 * e + 1);
        const int j = min(k, w_n - 1);
        const float4 w0 = __ldg(water + 2 * j), w1 = __ldg(water + 2 * j + 1);
        const float dw = k < w_n - 1 ? 1.f : 0.f;   // slope of the clamped water tables
        // values and slopes of the pairs (O1, O2) and (u1w, u2w) side by side,
        // for packed FP32 interpolation
        tabm[3 * e] = make_float4(a.x, a.y, fmaf(wscale, a.z, w1.x), fmaf(wscale, b.x, w1.z));
        tabm[3 * e + 1] = make_float4(fmaf(wscale, a.w, dw * w1.y), fmaf(wscale, b.y, dw * w1.w), w0.x, w0.z);
        tabm[3 * e + 2] = make_float4(dw * w0.y, dw * w0.w, 0.f, 0.f);
    }
}

// A(t_eq, theta) interpolated at each beamlet's theta, one row per beamlet,
// stored as (value, slope to the next t_eq sample).
__global__ void __launch_bounds__(256) k_arows(const float* __restrict__ A, int a_nt,
                                               const BeamletDev* __restrict__ bl, int B,
                                               float2* __restrict__ arow)
{
    const int64_t n = (int64_t)B * a_nt;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / a_nt), j = (int)(e % a_nt);
        const int l = __ldg(&bl[i].meta.y);
        const float w = __ldg(&bl[i].exy_z.w);
        const float* r0 = A + (size_t)l * a_nt;
        const float* r1 = r0 + a_nt;
        const float v = fmaf(w, __ldg(r1 + j) - __ldg(r0 + j), __ldg(r0 + j));
        float dv = 0.f;
        if (j + 1 < a_nt) dv = fmaf(w, __ldg(r1 + j + 1) - __ldg(r0 + j + 1), __ldg(r0 + j + 1)) - v;
        arow[e] = make_float2(v, dv);
    }
}

// Steps 2-3: beam frame, beamlet axis and frame, theta; one thread per beamlet.
constexpr int kBeamletThreads = 64;
__global__ void __launch_bounds__(kBeamletThreads) k_beamlets(const BeamletArgs A)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.B) return;
    int b = 0;
    while (b + 1 < A.n_beams && A.first[b + 1] <= i) ++b;
    const dc_beam bm = A.beams[b];
    const double deg = M_PI / 180.0;

    // beam frame: gantry about +z, couch about +y, collimator about the axis
    double ex[3] = {1, 0, 0}, ey[3] = {0, 0, 1}, ez[3] = {0, 1, 0};
    rot_z(bm.gantry_deg * deg, ex); rot_z(bm.gantry_deg * deg, ey); rot_z(bm.gantry_deg * deg, ez);
    rot_y(bm.couch_deg * deg, ex); rot_y(bm.couch_deg * deg, ey); rot_y(bm.couch_deg * deg, ez);
    double cc = cos(bm.coll_deg * deg), sc = sin(bm.coll_deg * deg);
    double fx_[3], fy_[3];
    for (int q = 0; q < 3; ++q) {
        fx_[q] = cc * ex[q] + sc * ey[q];
        fy_[q] = -sc * ex[q] + cc * ey[q];
    }
    const double sad = bm.sad;
    double src[3], iso[3] = {bm.iso[0], bm.iso[1], bm.iso[2]};
    for (int q = 0; q < 3; ++q) src[q] = iso[q] - sad * ez[q];

    const int M = A.M[b];
    const int local = i - A.first[b];
    const int n = local / M, m = local % M;
    const double hfx = 0.5 * (double)bm.field_x, hfy = 0.5 * (double)bm.field_y;
    const double a = -hfx + (m + 0.5) * A.bx, c = -hfy + (n + 0.5) * A.by;

    double nv[3];
    for (int q = 0; q < 3; ++q) nv[q] = iso[q] + a * fx_[q] + c * fy_[q] - src[q];
    double nn = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    for (int q = 0; q < 3; ++q) nv[q] /= nn;
    const double theta = atan2(sqrt(a * a + c * c), sad);
    double exx[3], en = fx_[0] * nv[0] + fx_[1] * nv[1] + fx_[2] * nv[2];
    for (int q = 0; q < 3; ++q) exx[q] = fx_[q] - en * nv[q];
    double ne = sqrt(exx[0] * exx[0] + exx[1] * exx[1] + exx[2] * exx[2]);
    for (int q = 0; q < 3; ++q) exx[q] /= ne;
    double eyy[3] = {exx[1] * nv[2] - exx[2] * nv[1], exx[2] * nv[0] - exx[0] * nv[2],
                     exx[0] * nv[1] - exx[1] * nv[0]};

    if (local == 0) {
        BeamDev o;
        for (int q = 0; q < 3; ++q) {
            o.src[q] = (float)src[q];
            o.ez[q] = (float)ez[q];
            o.ex[q] = (float)fx_[q];
            o.ey[q] = (float)fy_[q];
        }
        o.sad = (float)sad;
        o.inv_cos_max = (float)(sqrt(sad * sad + hfx * hfx + hfy * hfy) / sad);
        o.half_fx = (float)hfx;
        o.half_fy = (float)hfy;
        o.M = M;
        o.N = (A.first[b + 1] - A.first[b]) / M;
        o.first = A.first[b];
        o.pad = 0;
        A.out_beams[b] = o;
    }

    // row of A(t_eq, theta) and the weight of the next row
    float rl = fminf(fmaxf((float)theta * A.inv_adth, 0.f), (float)(A.a_nth - 1));
    int l = min((int)rl, A.a_nth - 2);
    float wl = rl - (float)l;

    // the axis in FP64 for the trace (k_trace), which also fills in L_in,
    // L_out, K and hit
    double* ray = A.ray + 8 * (size_t)i;
    for (int q = 0; q < 3; ++q) {
        ray[q] = src[q];
        ray[4 + q] = nv[q];
    }
    ray[3] = ray[7] = 0.0;
    BeamletDev r;
    r.n_lin = make_float4((float)nv[0], (float)nv[1], (float)nv[2], 0.f);
    r.exy_xy = make_float4((float)exx[0], (float)eyy[0], (float)exx[1], (float)eyy[1]);
    r.exy_z = make_float4((float)exx[2], (float)eyy[2], -1.0f, wl);
    r.meta = make_int4(0, l, 0, b);
    A.out_bl[i] = r;
    A.out_theta[i] = (float)theta;
}

// ---------------------------------------------------------------------------
// Steps 4-6 with one warp per beamlet.  The ray [amin, amax] inside the grid
// is cut into 32 pieces of equal length and lane j walks piece j, keeping its
// segments (end, density) in shared memory.  FP64 only places each piece on
// the ray (its first voxel and first plane crossings); the walk itself runs
// in FP32 offsets from the piece's start, which stay below the piece length,
// so their rounding is far below that of the absolute FP64 walk's results
// once stored in FP32 (this GPU's FP64 pipe runs at a small fraction of its
// FP32 rate and would otherwise bound the kernel).  Ballots give the body
// entry L_in (start of the first segment denser than the surface threshold)
// and exit L_out (end of the last), an exclusive warp scan of the pieces'
// integrals of rho, b_1(rho), b_2(rho) from L_in gives each piece its starting
// values, and each lane then emits the depth samples L_in + k d of its piece.
// The sample indices are split between the lanes exactly (in FP64), so every
// sample is written once.  A ray with more segments in a piece than the buffer
// holds is traced by one lane with the single FP64 walk (trace_beamlet).
constexpr int kTraceWarps = 4;
constexpr int kSegCap = 24;     // segments per piece (rays of up to ~700 voxel crossings)

__device__ __forceinline__ float warp_exclusive_sum(float x, int lane)
{
    float incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    return incl - x;
}

// Walk state of one piece: plane crossings as FP32 offsets from its start.
struct PieceWalk {
    int idx[3], step[3];
    float next[3], delta[3];
    float len;
};

__device__ void piece_init(const BeamletArgs& A, const double* s, const double* n, const double* inv_n,
                           double a_start, double a_end, PieceWalk& w)
{
    Walk f;
    walk_from(A, s, n, inv_n, a_start, a_end, f);
    for (int a = 0; a < 3; ++a) {
        w.idx[a] = f.idx[a];
        w.step[a] = f.step[a];
        const bool par = f.step[a] == 0;
        w.next[a] = par ? 3.0e38f : (float)(f.anext[a] - a_start);
        w.delta[a] = par ? 0.f : (float)f.adelta[a];
    }
    w.len = (float)(a_end - a_start);
}

template <typename F>
__device__ void piece_run(const BeamletArgs& A, const PieceWalk& w, F&& visit)
{
    // the state in scalars (no dynamically indexed arrays: registers only)
    int i0 = w.idx[0], i1 = w.idx[1], i2 = w.idx[2];
    float n0 = w.next[0], n1 = w.next[1], n2 = w.next[2];
    const int maxit = A.nx + A.ny + A.nz + 8;
    float cur = 0.f;
    for (int it = 0; it < maxit; ++it) {
        float an = n0;
        int ax = 0;
        if (n1 < an) { an = n1; ax = 1; }
        if (n2 < an) { an = n2; ax = 2; }
        const bool last = an >= w.len;
        if (last) an = w.len;
        if (an > cur) visit(cur, an, ((int64_t)i2 * A.ny + i1) * A.nx + i0);
        if (last) return;
        if (ax == 0) {
            i0 += w.step[0];
            if (i0 < 0 || i0 >= A.nx) return;
            n0 += w.delta[0];
        } else if (ax == 1) {
            i1 += w.step[1];
            if (i1 < 0 || i1 >= A.ny) return;
            n1 += w.delta[1];
        } else {
            i2 += w.step[2];
            if (i2 < 0 || i2 >= A.nz) return;
            n2 += w.delta[2];
        }
        cur = an;
    }
}

// Returns false if a piece overflowed its segment buffer (nothing written).
__device__ bool trace_warp(const BeamletArgs& A, const double* s, const double* n, const double* inv_n,
                           const Walk& w0, int lane, float2* __restrict__ seg, float4* __restrict__ tab,
                           double& L_in, double& L_out, int& K)
{
    const double amin = w0.acur, amax = w0.amax;
    const double span = (amax - amin) / 32.0;
    // piece j starts at amin + j span; the end of piece j is the start of
    // piece j + 1 (the same expression, so the same value)
    const double a_start = amin + lane * span;
    const double a_end = lane == 31 ? amax : amin + (lane + 1) * span;
    const float surf = A.rho_surf;

    // 1. walk the piece
    int ns = 0;
    bool dense = false;
    float first_r = 0.f, last_r = 0.f;
    PieceWalk w;
    piece_init(A, s, n, inv_n, a_start, a_end, w);
    piece_run(A, w, [&](float a0, float a1, int64_t vox) {
        const float r = __ldg(A.rho + vox);
        if (ns < kSegCap) seg[ns] = make_float2(a1, r);
        ++ns;
        if (r > surf) {
            if (!dense) first_r = a0;
            dense = true;
            last_r = a1;
        }
    });
    if (__any_sync(0xffffffffu, ns > kSegCap)) return false;

    // 2. body entry and exit of the whole ray: the first dense segment of the
    // first lane that has one, the last dense segment of the last
    const unsigned dm = __ballot_sync(0xffffffffu, dense);
    K = 0;
    if (dm == 0) return true;   // the axis misses the body
    const int lf = __ffs(dm) - 1, ll = 31 - __clz(dm);
    const float fr = __shfl_sync(0xffffffffu, first_r, lf);
    const float lr = __shfl_sync(0xffffffffu, last_r, ll);
    L_in = (amin + lf * span) + (double)fr;
    L_out = (amin + ll * span) + (double)lr;
    const double d = A.d;
    K = max(2, (int)ceil((L_out - L_in) / d) + 1);
    K = min(K, A.Kmax);

    // 3. this piece's integrals from L_in, and the piece's starting values
    const float Lrel = (float)(L_in - a_start);
    float pT = 0.f, p1 = 0.f, p2 = 0.f;
    float a0 = 0.f;
    for (int q = 0; q < ns; ++q) {
        const float2 sg = seg[q];
        if (sg.x > Lrel) {
            const float len = sg.x - fmaxf(a0, Lrel);
            pT = fmaf(sg.y, len, pT);
            p1 = fmaf(lut_dens(A, 4, sg.y), len, p1);
            p2 = fmaf(lut_dens(A, 5, sg.y), len, p2);
        }
        a0 = sg.x;
    }
    float cT = warp_exclusive_sum(pT, lane), c1 = warp_exclusive_sum(p1, lane), c2 = warp_exclusive_sum(p2, lane);

    // 4. the samples of this piece: k in [k_lo, k_hi), k_lo the least k >= 0
    // with L_in + k d >= a_start, k_hi the next lane's k_lo (lane 31: K, the
    // samples past the end of the ray included); positions as FP32 offsets
    // from a_start
    int k_lo = 0;
    if (a_start > L_in) {
        k_lo = (int)ceil((a_start - L_in) * A.inv_d);
        while (k_lo > 0 && L_in + (k_lo - 1) * d >= a_start) --k_lo;
        while (L_in + k_lo * d < a_start) ++k_lo;
    }
    int k_hi = __shfl_down_sync(0xffffffffu, k_lo, 1);
    if (lane == 31) k_hi = K;
    k_hi = min(k_hi, K);
    const float base = (float)((L_in + k_lo * d) - a_start);
    const float df = (float)d;
    int k = k_lo;
    a0 = 0.f;
    for (int q = 0; q < ns && k < k_hi; ++q) {
        const float2 sg = seg[q];
        if (sg.x > Lrel) {
            const float lo = fmaxf(a0, Lrel);
            const float v1 = lut_dens(A, 4, sg.y), v2 = lut_dens(A, 5, sg.y);
            while (k < k_hi) {
                const float sk = fmaf((float)(k - k_lo), df, base);
                if (sk > sg.x) break;
                const float len = sk - lo;
                tab[2 * k] = make_float4(fmaf(sg.y, len, cT), 0.f, fmaf(v1, len, c1), 0.f);
                tab[2 * k + 1] = make_float4(fmaf(v2, len, c2), 0.f, 0.f, 0.f);
                ++k;
            }
            const float len = sg.x - lo;
            cT = fmaf(sg.y, len, cT);
            c1 = fmaf(v1, len, c1);
            c2 = fmaf(v2, len, c2);
        }
        a0 = sg.x;
    }
    // past the last segment: the samples beyond the end of the ray (lane 31),
    // or within rounding of the piece's end
    for (; k < k_hi; ++k) {
        tab[2 * k] = make_float4(cT, 0.f, c1, 0.f);
        tab[2 * k + 1] = make_float4(c2, 0.f, 0.f, 0.f);
    }
    __syncwarp();

    // 5. slopes to the next sample (zero at K - 1): read, then write
    for (int k0 = 0; k0 < K; k0 += 32) {
        const int kk = k0 + lane;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        float nT = 0.f, n1 = 0.f, n2 = 0.f;
        if (kk < K) {
            a = tab[2 * kk];
            b = tab[2 * kk + 1];
            nT = a.x;
            n1 = a.z;
            n2 = b.x;
            if (kk + 1 < K) {
                const float4 an = tab[2 * kk + 2], bn = tab[2 * kk + 3];
                nT = an.x;
                n1 = an.z;
                n2 = bn.x;
            }
        }
        __syncwarp();
        if (kk < K) {
            tab[2 * kk] = make_float4(a.x, nT - a.x, a.z, n1 - a.z);
            tab[2 * kk + 1] = make_float4(b.x, n2 - b.x, 0.f, 0.f);
        }
        __syncwarp();
    }
    return true;
}

__global__ void __launch_bounds__(32 * kTraceWarps) k_trace(const BeamletArgs A)
{
    __shared__ float2 s_seg[kTraceWarps][32][kSegCap];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kTraceWarps + warp;
    if (i >= A.B) return;   // whole warps
    const double* ray = A.ray + 8 * (size_t)i;
    const double s[3] = {ray[0], ray[1], ray[2]}, n[3] = {ray[4], ray[5], ray[6]};
    double inv_n[3];
    ray_inverse(n, inv_n);
    Walk w;
    int K = 0;
    double L_in = 0, L_out = 0;
    if (walk_init(A, s, n, inv_n, w)) {
        float4* tb = A.tab + 2 * (size_t)i * A.Kmax;
        const bool ok = trace_warp(A, s, n, inv_n, w, lane, s_seg[warp][lane], tb, L_in, L_out, K);
        if (!ok && lane == 0) {
            if (w.amax - w.acur > 40.0)
                trace_beamlet<double>(A, w, tb, L_in, L_out, K);
            else
                trace_beamlet<float>(A, w, tb, L_in, L_out, K);
        }
        if (!ok) {
            K = __shfl_sync(0xffffffffu, K, 0);
            L_in = __shfl_sync(0xffffffffu, L_in, 0);
            L_out = __shfl_sync(0xffffffffu, L_out, 0);
        }
    }
    if (lane == 0) {
        BeamletDev& r = A.out_bl[i];
        const int hit = K > 0 ? 1 : 0;
        r.n_lin.w = (float)L_in;
        r.exy_z.z = hit ? (float)L_out : -1.0f;
        r.meta.x = K;
        r.meta.z = hit;
        A.lio[i] = make_float2((float)L_in, hit ? (float)L_out : -1.0f);
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (int)(g > 152 * 64 ? 152 * 64 : (g < 1 ? 1 : g));
}

void gauss_weights(double sigma, double delta, int* r, float* w)
{
    int rr = sigma > 0 ? (int)ceil(3.0 * sigma / delta) : 0;
    double tmp[2 * kMaxSmoothRadius + 1], s = 0.0;
    for (int j = -rr; j <= rr; ++j) {
        tmp[j + rr] = sigma > 0 ? exp(-(j * delta) * (j * delta) / (2.0 * sigma * sigma)) : 1.0;
        s += tmp[j + rr];
    }
    for (int j = 0; j < 2 * rr + 1; ++j) w[j] = (float)(tmp[j] / s);
    *r = rr;
}

}  // namespace

int smooth_radius(double sigma, double delta)
{
    return sigma > 0 ? (int)ceil(3.0 * sigma / delta) : 0;
}

cudaError_t launch_smooth(const dc_plan* p, float sigma)
{
    const dc_grid& g = p->grid;
    SmoothArgs a;
    a.nx = g.nx; a.ny = g.ny; a.nz = g.nz;
    int gsz = grid_for(p->V, 256);
    // x pass: rho -> rhos, y pass: rhos -> tmp, z pass: tmp -> rhos
    gauss_weights(sigma, g.dx, &a.r, a.w);
    a.in = p->d_rho; a.out = p->d_rhos;
    k_smooth_axis<0><<<gsz, 256, 0, p->stream>>>(a);
    gauss_weights(sigma, g.dy, &a.r, a.w);
    a.in = p->d_rhos; a.out = p->d_tmp;
    k_smooth_axis<1><<<gsz, 256, 0, p->stream>>>(a);
    gauss_weights(sigma, g.dz, &a.r, a.w);
    a.in = p->d_tmp; a.out = p->d_rhos;
    k_smooth_axis<2><<<gsz, 256, 0, p->stream>>>(a);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_factors(const dc_plan* p)
{
    const dc_kernel_coeffs& c = p->coeffs;
    k_factors<<<grid_for(p->V, 256), 256, 0, p->stream>>>(
        p->d_rho, p->d_rhos, p->d_dens, c.f_n, c.f_rho0, 1.0f / c.f_drho, c.density_correction,
        p->V, p->d_fac);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_beamlets(const dc_plan* p)
{
    if (p->n_beams > kMaxBeams) return cudaErrorInvalidValue;
    BeamletArgs A;
    const dc_grid& g = p->grid;
    const dc_kernel_coeffs& c = p->coeffs;
    A.beams = p->d_beamin;
    A.rho = p->d_rho;
    A.dens = p->d_dens;
    A.f_n = c.f_n;
    A.f_rho0 = c.f_rho0;
    A.inv_drho = 1.0f / c.f_drho;
    A.nx = g.nx; A.ny = g.ny; A.nz = g.nz;
    A.B = p->B;
    A.n_beams = p->n_beams;
    A.Kmax = p->Kmax;
    A.dx = g.dx; A.dy = g.dy; A.dz = g.dz;
    A.idx = 1.0 / (double)g.dx; A.idy = 1.0 / (double)g.dy; A.idz = 1.0 / (double)g.dz;
    A.ox = g.ox; A.oy = g.oy; A.oz = g.oz;
    A.d = 0.5 * fmin((double)g.dx, fmin((double)g.dy, (double)g.dz));
    A.inv_d = 1.0 / A.d;
    A.bx = p->bx;
    A.by = p->by;
    A.rho_surf = c.rho_surface;
    A.a_nth = c.a_ntheta;
    A.inv_adth = 1.0f / c.a_dtheta;
    A.out_beams = p->d_beams;
    A.out_bl = p->d_bl;
    A.out_theta = p->d_theta;
    A.tab = p->d_tab;
    A.ray = p->d_ray;
    A.lio = p->d_lio;
    for (int b = 0; b < p->n_beams; ++b) {
        A.first[b] = p->first[b];
        A.M[b] = p->M[b];
    }
    A.first[p->n_beams] = p->B;
    k_beamlets<<<(p->B + kBeamletThreads - 1) / kBeamletThreads, kBeamletThreads, 0, p->stream>>>(A);
    k_trace<<<(p->B + kTraceWarps - 1) / kTraceWarps, 32 * kTraceWarps, 0, p->stream>>>(A);
    count_launches(2);
    k_arows<<<grid_for((int64_t)p->B * p->coeffs.a_nt, 256), 256, 0, p->stream>>>(
        p->d_A, p->coeffs.a_nt, p->d_bl, p->B, p->d_arow);
    count_launches(1);
    if (p->merged) {
        k_merge_tables<<<grid_for((int64_t)p->B * p->Kmax, 256), 256, 0, p->stream>>>(
            p->d_tab, p->d_water, p->coeffs.w_n, p->d_bl, p->B, p->Kmax,
            p->coeffs.density_correction ? 1.0f : 0.0f, p->d_tabm);
        count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace dc
