// Dose kernel of the DC-FSPB engine (Algorithm A1 steps 7-14 / A2 Kernel 5):
// the per-(voxel, beamlet) evaluation of eq. (2) with the lateral kernel of
// eqs. (3)-(4), and the fluence-weighted sum of eq. (1).
//
// Work decomposition (gather, no global atomics): each warp owns a 4x4x2
// brick of voxels, one voxel per lane, and accumulates its dose in registers.
// For each beam the warp projects its voxels into the isocentre plane and
// walks, row by row, the union of the lanes' ROI discs over the beamlet grid;
// each lane applies the exact ROI and depth-range test of its own pair.  The
// same traversal, with the evaluation replaced by a counter or by a CSR
// store, gives the dose-deposition matrix.
#include <math.h>

#include "dc_internal.cuh"

namespace dc {
namespace {

constexpr int kWarps = 8;           // warps per CTA
constexpr int kThreads = 32 * kWarps;
constexpr float kLog2e = 1.4426950408889634f;

enum Mode { kDose = 0, kCount = 1, kFill = 2 };

struct DoseArgs {
    PlanView P;
    const float* fluence;   // [nf][ldf]
    int nf, ldf;
    float* dose;            // [nf][ldd]
    int64_t ldd;
    int32_t* counts;        // kCount
    const int64_t* rowptr;  // kFill
    int32_t* cols;
    void* vals;
    int value_dtype;
    int bricks_x, bricks_y, bricks_z;
};

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Eq. (4) with k = u log2(e): inside |x| <= x0 it is 1 - (e1 + e2)/2,
// outside (e1 - e2)/2, with e1 = exp(-u ||x| - x0|), e2 = exp(-u (|x| + x0)).
__device__ __forceinline__ float penumbra(float x, float k, float x0)
{
    float ax = fabsf(x);
    float e1 = ex2(-k * fabsf(ax - x0));
    float e2 = ex2(-k * (ax + x0));
    return ax <= x0 ? fmaf(-0.5f, e1 + e2, 1.0f) : 0.5f * (e1 - e2);
}

struct Lane {
    float vx, vy, vz;     // r - source
    float4 fac;           // density-correction factors of the voxel
    bool valid;
};

// Decides whether the lane's voxel is in beamlet i's ROI and depth range and,
// if EVAL, returns D_i(r) of eq. (2) for unit fluence.
template <bool EVAL>
__device__ __forceinline__ bool pair(const PlanView& P, const Lane& ln, int i, float sad,
                                     const float4* __restrict__ sW, const float* __restrict__ sA,
                                     float& D)
{
    const BeamletDev* bl = P.bl + i;
    const float4 q0 = __ldg(&bl->n_lin);
    const float4 q1 = __ldg(&bl->ex_tout);
    const float4 q2 = __ldg(&bl->ey_wth);
    const int4 q3 = __ldg(&bl->meta);
    float L = fmaf(ln.vx, q0.x, fmaf(ln.vy, q0.y, ln.vz * q0.z));
    float xp = fmaf(ln.vx, q1.x, fmaf(ln.vy, q1.y, ln.vz * q1.z));
    float yp = fmaf(ln.vx, q2.x, fmaf(ln.vy, q2.y, ln.vz * q2.z));
    float t = L - q0.w;
    bool in = ln.valid && q3.z && fmaf(xp, xp, yp * yp) <= P.R2 && t >= 0.f && t <= q1.w;
    if (!EVAL || !in) return in;

    const float s = sad * __frcp_rn(L);          // SAD / |r_a|
    const float x = xp * s, y = yp * s;          // isocentre-plane coordinates

    // radiological depth and omega_corr tables (steps 5-6), linear in t
    const float kf = t * P.inv_d;
    const int k = min((int)kf, q3.x - 2);
    const float fr = kf - (float)k;
    const float4* tb = P.tab + (size_t)i * P.Kmax + k;
    const float4 e0 = __ldg(tb), e1 = __ldg(tb + 1);
    const float teq = fmaf(fr, e1.x - e0.x, e0.x);
    const float c1 = fmaf(fr, e1.y - e0.y, e0.y);
    const float c2 = fmaf(fr, e1.z - e0.z, e0.z);

    // water parameters u_i^w(t), omega_i^w(t) (step 10)
    const float sw = fminf(t * P.inv_wdt, (float)(P.w_n - 1));
    const int jw = min((int)sw, P.w_n - 2);
    const float fw = sw - (float)jw;
    const float4 w0 = sW[jw], w1 = sW[jw + 1];
    const float u1w = fmaf(fw, w1.x - w0.x, w0.x);
    const float u2w = fmaf(fw, w1.y - w0.y, w0.y);
    const float o1w = fmaf(fw, w1.z - w0.z, w0.z);
    const float o2w = fmaf(fw, w1.w - w0.w, w0.w);

    // A(t_eq, theta), bilinear (step 9)
    const float sa = fminf(fmaxf(teq * P.inv_adt, 0.f), (float)(P.a_nt - 1));
    const int j = min((int)sa, P.a_nt - 2);
    const float wt = sa - (float)j;
    const float* Ar = sA + q3.y * P.a_nt + j;
    const float a0 = fmaf(wt, Ar[1] - Ar[0], Ar[0]);
    const float a1 = fmaf(wt, Ar[P.a_nt + 1] - Ar[P.a_nt], Ar[P.a_nt]);
    const float Av = fmaf(q2.w, a1 - a0, a0);

    // density correction (step 11)
    const float k1 = ln.fac.x * u1w * kLog2e;
    const float k2 = ln.fac.y * u2w * kLog2e;
    const float om1 = fmaxf(ln.fac.z * fmaf(P.wscale, c1, o1w), 0.f);
    const float om2 = fmaxf(ln.fac.w * fmaf(P.wscale, c2, o2w), 0.f);

    // eqs. (3) and (2)
    const float F = fmaf(om1 * penumbra(x, k1, P.x0), penumbra(y, k1, P.y0),
                         om2 * penumbra(x, k2, P.x0) * penumbra(y, k2, P.y0));
    D = F * Av * (s * s);
    return true;
}

template <int MODE, int NF>
__global__ void __launch_bounds__(kThreads) k_dose(const DoseArgs a)
{
    extern __shared__ float4 smem[];
    const PlanView& P = a.P;
    float4* sW = smem;
    float* sA = reinterpret_cast<float*>(smem + P.w_n);
    if (MODE != kCount) {
        for (int q = threadIdx.x; q < P.w_n; q += blockDim.x) sW[q] = __ldg(P.water + q);
        for (int q = threadIdx.x; q < P.a_nt * P.a_nth; q += blockDim.x) sA[q] = __ldg(P.A + q);
        __syncthreads();
    }

    // brick of this CTA: 8 x 8 x 4 voxels, warp tiles of 4 x 4 x 2
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int bid = blockIdx.x;
    const int bxi = bid % a.bricks_x;
    bid /= a.bricks_x;
    const int byi = bid % a.bricks_y;
    const int bzi = bid / a.bricks_y;
    const int ix = bxi * 8 + (warp & 1) * 4 + (lane & 3);
    const int iy = byi * 8 + ((warp >> 1) & 1) * 4 + ((lane >> 2) & 3);
    const int iz = bzi * 4 + (warp >> 2) * 2 + (lane >> 4);

    Lane ln;
    ln.valid = ix < P.nx && iy < P.ny && iz < P.nz;
    const int64_t v = ((int64_t)min(iz, P.nz - 1) * P.ny + min(iy, P.ny - 1)) * P.nx + min(ix, P.nx - 1);
    // explicit fma: the count and fill passes must round these identically
    const float rx = fmaf((float)ix, P.dx, P.ox), ry = fmaf((float)iy, P.dy, P.oy),
                rz = fmaf((float)iz, P.dz, P.oz);
    ln.fac = MODE == kCount ? make_float4(1, 1, 1, 1) : __ldg(P.fac + v);

    float acc[NF];
#pragma unroll
    for (int q = 0; q < NF; ++q) acc[q] = 0.f;
    int32_t cnt = 0;
    int64_t pos = (MODE == kFill && ln.valid) ? a.rowptr[v] : 0;
    // a fill never writes past its own row, whatever the rounding
    const int64_t pend = (MODE == kFill && ln.valid) ? a.rowptr[v + 1] : 0;

    for (int b = 0; b < P.n_beams; ++b) {
        const BeamDev& bm = P.beams[b];
        const float sx = __ldg(&bm.src[0]), sy = __ldg(&bm.src[1]), sz = __ldg(&bm.src[2]);
        const float sad = __ldg(&bm.sad);
        ln.vx = rx - sx; ln.vy = ry - sy; ln.vz = rz - sz;
        const float zz = ln.vx * __ldg(&bm.ez[0]) + ln.vy * __ldg(&bm.ez[1]) + ln.vz * __ldg(&bm.ez[2]);
        const float pa = ln.vx * __ldg(&bm.ex[0]) + ln.vy * __ldg(&bm.ex[1]) + ln.vz * __ldg(&bm.ex[2]);
        const float pc = ln.vx * __ldg(&bm.ey[0]) + ln.vy * __ldg(&bm.ey[1]) + ln.vz * __ldg(&bm.ey[2]);
        const int M = __ldg(&bm.M), N = __ldg(&bm.N), first = __ldg(&bm.first);
        const float hfx = __ldg(&bm.half_fx), hfy = __ldg(&bm.half_fy);
        const bool live = ln.valid && zz > 1e-3f;
        // isocentre-plane projection of the voxel and a conservative radius of
        // the set of beamlet axes whose ROI cylinder can hold it
        const float sz_ = sad / zz;
        const float ca = pa * sz_, cc = pc * sz_;
        const float rw = live ? (P.roi * sz_ * __ldg(&bm.inv_cos_max)) * 1.0005f + 1e-3f : 0.f;

        int nlo = INT_MAX, nhi = INT_MIN;
        if (live) {
            nlo = max(0, (int)ceilf((cc - rw + hfy) / P.by - 0.5f));
            nhi = min(N - 1, (int)floorf((cc + rw + hfy) / P.by - 0.5f));
        }
        const int wnlo = __reduce_min_sync(0xffffffffu, nlo);
        const int wnhi = __reduce_max_sync(0xffffffffu, nhi);
        for (int n = wnlo; n <= wnhi; ++n) {
            const float dc_ = cc - (-hfy + (n + 0.5f) * P.by);
            const float h2 = rw * rw - dc_ * dc_;
            int mlo = INT_MAX, mhi = INT_MIN;
            if (live && h2 >= 0.f) {
                const float hx = sqrtf(h2);
                mlo = max(0, (int)ceilf((ca - hx + hfx) / P.bx - 0.5f));
                mhi = min(M - 1, (int)floorf((ca + hx + hfx) / P.bx - 0.5f));
            }
            const int wmlo = __reduce_min_sync(0xffffffffu, mlo);
            const int wmhi = __reduce_max_sync(0xffffffffu, mhi);
            const int row = first + n * M;
            for (int m = wmlo; m <= wmhi; ++m) {
                const int i = row + m;
                if (MODE == kDose) {
                    float f[NF];
                    bool any = false;
#pragma unroll
                    for (int q = 0; q < NF; ++q) {
                        f[q] = q < a.nf ? __ldg(a.fluence + (size_t)q * a.ldf + i) : 0.f;
                        any |= f[q] != 0.f;
                    }
                    if (!any) continue;
                    float D;
                    if (pair<true>(P, ln, i, sad, sW, sA, D)) {
#pragma unroll
                        for (int q = 0; q < NF; ++q) acc[q] = fmaf(f[q], D, acc[q]);
                    }
                } else if (MODE == kCount) {
                    float D;
                    cnt += pair<false>(P, ln, i, sad, sW, sA, D) ? 1 : 0;
                } else {
                    float D;
                    if (pair<true>(P, ln, i, sad, sW, sA, D) && pos < pend) {
                        a.cols[pos] = i;
                        if (a.value_dtype == DC_BF16)
                            reinterpret_cast<__nv_bfloat16*>(a.vals)[pos] = __float2bfloat16_rn(D);
                        else
                            reinterpret_cast<float*>(a.vals)[pos] = D;
                        ++pos;
                    }
                }
            }
        }
    }
    if (!ln.valid) return;
    if (MODE == kDose) {
#pragma unroll
        for (int q = 0; q < NF; ++q)
            if (q < a.nf) a.dose[(size_t)q * a.ldd + v] = acc[q];
    } else if (MODE == kCount) {
        a.counts[v] = cnt;
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of per-voxel counts (int32) into CSR row pointers (int64).
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanChunk = kScanThreads * kScanPer;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t* s_warp, int64_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    int64_t r = incl - x + s_warp[warp];
    *total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const int32_t* __restrict__ c, int64_t n,
                                                            int64_t* __restrict__ sums)
{
    __shared__ int64_t sw[33];
    int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    int64_t s = 0;
    for (int q = 0; q < kScanPer; ++q)
        if (base + q < n) s += c[base + q];
    int64_t tot;
    block_exclusive_scan(s, sw, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int64_t* __restrict__ sums, int nb,
                                                           int64_t* __restrict__ total)
{
    __shared__ int64_t sw[33];
    int64_t carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        int q = base + threadIdx.x;
        int64_t x = q < nb ? sums[q] : 0;
        int64_t tot;
        int64_t e = block_exclusive_scan(x, sw, &tot);
        if (q < nb) sums[q] = e + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int32_t* __restrict__ c, int64_t n,
                                                             const int64_t* __restrict__ offs,
                                                             int64_t* __restrict__ rowptr,
                                                             const int64_t* __restrict__ total)
{
    __shared__ int64_t sw[33];
    int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    int32_t x[kScanPer];
    int64_t s = 0;
    for (int q = 0; q < kScanPer; ++q) {
        x[q] = base + q < n ? c[base + q] : 0;
        s += x[q];
    }
    int64_t tot;
    int64_t e = block_exclusive_scan(s, sw, &tot) + offs[blockIdx.x];
    for (int q = 0; q < kScanPer; ++q) {
        if (base + q < n) rowptr[base + q] = e;
        e += x[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rowptr[n] = *total;
}

DoseArgs make_args(const dc_plan* p)
{
    DoseArgs a{};
    a.P = p->view();
    a.bricks_x = (p->grid.nx + 7) / 8;
    a.bricks_y = (p->grid.ny + 7) / 8;
    a.bricks_z = (p->grid.nz + 3) / 4;
    return a;
}

size_t smem_bytes(const dc_plan* p)
{
    return sizeof(float4) * p->coeffs.w_n + sizeof(float) * (size_t)p->coeffs.a_nt * p->coeffs.a_ntheta;
}

template <int MODE, int NF>
cudaError_t run(const dc_plan* p, const DoseArgs& a)
{
    size_t sm = MODE == kCount ? 0 : smem_bytes(p);
    cudaError_t e = cudaFuncSetAttribute(k_dose<MODE, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    int nb = a.bricks_x * a.bricks_y * a.bricks_z;
    k_dose<MODE, NF><<<nb, kThreads, sm, p->stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dose(const dc_plan* p, const float* fluence, int nf, int ldf, float* dose,
                        int64_t ldd)
{
    DoseArgs a = make_args(p);
    a.ldf = ldf;
    a.ldd = ldd;
    for (int q0 = 0; q0 < nf; q0 += 16) {
        a.fluence = fluence + (size_t)q0 * ldf;
        a.dose = dose + (size_t)q0 * ldd;
        a.nf = nf - q0 < 16 ? nf - q0 : 16;
        cudaError_t e = a.nf == 1 ? run<kDose, 1>(p, a) : run<kDose, 16>(p, a);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_count(const dc_plan* p, int32_t* counts)
{
    DoseArgs a = make_args(p);
    a.counts = counts;
    return run<kCount, 1>(p, a);
}

cudaError_t launch_fill(const dc_plan* p, const int64_t* rowptr, int32_t* cols, void* vals,
                        int value_dtype)
{
    DoseArgs a = make_args(p);
    a.rowptr = rowptr;
    a.cols = cols;
    a.vals = vals;
    a.value_dtype = value_dtype;
    return run<kFill, 1>(p, a);
}

cudaError_t launch_scan_counts(const dc_plan* p, const int32_t* counts, int64_t* rowptr,
                               int64_t* total_dev)
{
    int64_t n = p->V;
    int nb = (int)((n + kScanChunk - 1) / kScanChunk);
    int64_t* sums = reinterpret_cast<int64_t*>(p->d_scan_tmp);
    k_scan_sums<<<nb, kScanThreads, 0, p->stream>>>(counts, n, sums);
    k_scan_top<<<1, kScanThreads, 0, p->stream>>>(sums, nb, total_dev);
    k_scan_apply<<<nb, kScanThreads, 0, p->stream>>>(counts, n, sums, rowptr, total_dev);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace dc
