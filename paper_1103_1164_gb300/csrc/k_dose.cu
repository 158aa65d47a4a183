// Dose kernel of the DC-FSPB engine (Algorithm A1 steps 7-14 / A2 Kernel 5):
// the per-(voxel, beamlet) evaluation of eq. (2) with the lateral kernel of
// eqs. (3)-(4), and the fluence-weighted sum of eq. (1).
//
// Work decomposition (gather, no global atomics): a warp takes 32 voxels of
// one beam's list (voxels binned by their beam's-eye-view cell, k_bin.cu), one
// voxel per lane, and accumulates that beam's dose in registers.  It projects
// its voxels into the isocentre plane and walks, row by row, the union of the
// lanes' ROI discs over the beamlet grid; each lane applies the exact ROI and
// depth-range test of its own pair.  Per-beam partial doses are summed in
// beam order afterwards.  The same traversal, with the evaluation replaced by
// a counter or by a CSR store, gives the dose-deposition matrix.
//
// Hot-loop choices: table indices come from a magic-constant rounding (no
// float->int conversion, which would share the quarter-rate pipe with the
// exponentials); every table stores value + slope so an interpolation is one
// load and one fma; eq. (4) is evaluated without branches.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "dc_internal.cuh"

namespace dc {
namespace {

constexpr int kWarps = 8;           // warps per CTA
constexpr int kThreads = 32 * kWarps;
constexpr float kLog2e = 1.4426950408889634f;
// CSR entries staged per lane: a ring in which the entry at position g of the
// column array sits in slot g mod kRing, so a run of pending entries never
// needs moving when only its head is written out
constexpr int kRing = 16;
constexpr int kRingLd = kRing + 1;
// beamlet records of a row window staged per warp at a time: fewer in the
// fill, whose CSR staging shares the CTA's shared memory, and with more than
// 32 fluence vectors, whose staging does
constexpr int row_max(int mode, int nf = 1) { return mode == 2 || nf > 32 ? 16 : 32; }

enum Mode { kDose = 0, kCount = 1, kFill = 2, kGrad = 3 };
// fluence vectors per pass of the dose kernel: 1, or 16, 32 or 64 staged
// beside each beamlet record (as NF / 4 float4, whose order the staging
// rotates by the lane's low two bits)
constexpr bool valid_nf(int nf) { return nf == 1 || nf == 16 || nf == 32 || nf == 64; }

// PREC 2, the tensor-core form of the multi-fluence dose (64 vectors): per
// warp and chunk of 16 beamlets, Y[32 voxels][64] += D[32][16] F[16][64] as
// mma.m16n8k16 with BF16 operands (D and F rounded to nearest even) and FP32
// accumulators in registers.  D is staged as BF16 pairs of neighbouring
// beamlets per voxel row (words [tile of 16 rows][beamlet pair][row]), F as
// BF16 pairs of neighbouring beamlets per vector (words [beamlet pair][vector]);
// the padded strides keep the per-beamlet stores and the fragment loads free of
// bank conflicts (the second 16-row tile starts on the other 16 banks).
constexpr int kTcRowD = 24;
constexpr int kTcTileD = 8 * kTcRowD + 16;
constexpr int kTcRowF = 72;
constexpr int kTcOffF = kTcTileD + 8 * kTcRowD;
constexpr int kTcWords = kTcOffF + 8 * kTcRowF;   // per warp

__device__ __forceinline__ void mma_bf16(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x to about one ulp (MUFU.RCP alone: no Newton step, no special-case path;
// L is a positive, normal distance here).
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Table coordinates without a conversion instruction (conversions share the
// quarter-rate pipe with the exponentials).  For 0 <= x < 2^22, adding
// 1.5 * 2^23 with rounding toward -infinity leaves floor(x) in the low
// mantissa bits: the result's bits are kGridBits + floor(x), and table
// offsets subtract kGridBits in 32-bit arithmetic, which folds into one
// multiply-add.  frac = x - floor(x).
constexpr uint32_t kGridBits = 0x4B400000u;
__device__ __forceinline__ uint32_t grid_bits(float x, float& frac)
{
    const float f = __fadd_rd(x, 12582912.0f);
    frac = __fadd_rn(x, -__fadd_rn(f, -12582912.0f));
    return __float_as_uint(f);
}

// The same for x = a b without rounding the product: floor(a b) and
// frac = a b - floor(a b) from two multiply-adds of the exact product.
__device__ __forceinline__ uint32_t grid_bits_mul(float a, float b, float& frac)
{
    const float f = __fmaf_rd(a, b, 12582912.0f);
    frac = __fmaf_rn(a, b, -__fadd_rn(f, -12582912.0f));
    return __float_as_uint(f);
}

// Eq. (4) with k = u log2(e): with e1 = exp(-u ||x| - x0|) and
// e2 = exp(-u (|x| + x0)) it is (e1 - e2)/2 outside |x| <= x0 and
// 1 - (e1 + e2)/2 inside.
// Evaluated for the x and y profiles of one component at once, in packed FP32
// pairs (one instruction for both axes wherever the two run the same
// operation): ax = (|x|, |y|), nk = -k per axis, x0 = (x0, y0).  With
// d = |x| - x0 and c = copysign(1 - e1, d), eq. (4) is 1/2 - (c + e2)/2 on
// both sides of |x| = x0 (c = -(1 - e1) inside, 1 - e1 outside).
// 2^a.x and 2^a.y from one special-function instruction on a packed BF16
// pair: the arguments are rounded to BF16 (8 significant bits), the results
// come back as BF16 and are widened exactly to FP32.
__device__ __forceinline__ float2 ex2_bf16x2(float2 a)
{
    uint32_t in, out;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(in) : "f"(a.y), "f"(a.x));   // high half a.y, low half a.x
    asm("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(out) : "r"(in));
    return make_float2(__uint_as_float(out << 16), __uint_as_float(out & 0xffff0000u));
}

// PREC 0: four FP32 exponentials; PREC 1 (the reduced-precision form): the
// x and y exponentials of each kind in one packed BF16 instruction, the rest
// in FP32.
template <int PREC>
__device__ __forceinline__ float2 penumbra2(float2 ax, float2 nk, float2 x0, float2 nx0)
{
    const float2 d = __fadd2_rn(ax, nx0);
    const float2 t1 = __fmul2_rn(nk, make_float2(fabsf(d.x), fabsf(d.y)));
    const float2 t2 = __ffma2_rn(nk, ax, __fmul2_rn(nk, x0));
    const float2 e1 = PREC ? ex2_bf16x2(t1) : make_float2(ex2(t1.x), ex2(t1.y));
    const float2 e2 = PREC ? ex2_bf16x2(t2) : make_float2(ex2(t2.x), ex2(t2.y));
    const float2 c = __ffma2_rn(e1, make_float2(-1.f, -1.f), make_float2(1.f, 1.f));
    const float2 q = __fadd2_rn(make_float2(copysignf(c.x, d.x), copysignf(c.y, d.y)), e2);
    return __ffma2_rn(make_float2(-0.5f, -0.5f), q, make_float2(0.5f, 0.5f));
}

// Lateral correction of step 11: the paper's rho(r), rho_hat(r) per voxel
// (kIso), or per-(voxel, beam) factors precomputed for every entry of the
// beam's voxel list by the axis-stencil pass or by the trained network
// (k_lateral.cu), loaded once per work unit (kItem).
enum Lateral { kIso = 0, kItem = 1 };

struct Lane {
    float vx, vy, vz;     // r - source
    // correction factors of the voxel for the current beam:
    // log2(e) f_u1(rho), log2(e) f_u2 along x and along y, f_w1, f_w2
    float cu1, cu2x, cu2y, cw1, cw2;
    bool valid;
};

// The pair test of beamlet i for the lane's voxel: in the ROI and between
// body entry and exit.  Padding lanes carry NaN coordinates, so every test
// fails for them.  Record and table offsets are 32-bit (the plan checks
// B * 3 Kmax < 2^31).
struct PairTest {
    float L;       // |r_a| along the beamlet axis
    float2 pq;     // (x', y')
    float L_in;
    bool in;
};

// q0 = (n, L_in), q1 = (e_x''.x, e_y''.x, e_x''.y, e_y''.y),
// q2 = (e_x''.z, e_y''.z, L_out, theta weight): the beamlet's record.
__device__ __forceinline__ PairTest pair_test(const PlanView& P, const Lane& ln, const float4 q0, const float4 q1,
                                              const float4 q2)
{
    PairTest r;
    r.L = fmaf(ln.vx, q0.x, fmaf(ln.vy, q0.y, ln.vz * q0.z));
    // (x', y') in one packed chain, each component rounded as the scalar fma chain
    float2 pq = __fmul2_rn(make_float2(ln.vz, ln.vz), make_float2(q2.x, q2.y));
    pq = __ffma2_rn(make_float2(ln.vy, ln.vy), make_float2(q1.z, q1.w), pq);
    r.pq = __ffma2_rn(make_float2(ln.vx, ln.vx), make_float2(q1.x, q1.y), pq);
    r.L_in = q0.w;
    r.in = fmaf(r.pq.x, r.pq.x, r.pq.y * r.pq.y) <= P.R2 && r.L >= q0.w && r.L <= q2.z;
    return r;
}

// D_i(r) of eq. (2) for unit fluence (called only where the pair is in).
template <bool MERGED, int LAT, int PREC>
__device__ __forceinline__ float pair_eval(const PlanView& P, const Lane& ln, const uint32_t i, const float sad,
                                           const float4* __restrict__ sW, const PairTest& pt)
{
    const float L = pt.L;
    const float2 pq = pt.pq;
    const float t = L - pt.L_in;                 // depth below the surface
    const float s = sad * rcp_approx(L);         // SAD / |r_a|
    const float2 xy = __fmul2_rn(pq, make_float2(s, s));   // isocentre-plane coordinates
    const float x = xy.x, y = xy.y;

    // radiological depth and omega_corr tables (steps 5-6) and the water
    // parameters u_i^w(t), omega_i^w(t) (step 10), linear in t
    float fr;
    const uint32_t kb = grid_bits_mul(t, P.inv_d, fr);
    float teq, O1, O2, u1w, u2w;
    if (MERGED) {
        const float4* tb = P.tabm + (i * (3u * (uint32_t)P.Kmax) + 3u * DC_GUARD(P, kb - kGridBits, P.Kmax, 1));
        const float4 e0 = __ldg(tb), e1 = __ldg(tb + 1), e2 = __ldg(tb + 2);
        teq = fmaf(fr, e0.y, e0.x);
        const float2 frr = make_float2(fr, fr);
        const float2 O = __ffma2_rn(frr, make_float2(e1.x, e1.y), make_float2(e0.z, e0.w));
        const float2 U = __ffma2_rn(frr, make_float2(e2.x, e2.y), make_float2(e1.z, e1.w));
        O1 = O.x;
        O2 = O.y;
        u1w = U.x;
        u2w = U.y;
    } else {
        const float4* tb = P.tab + (i * (2u * (uint32_t)P.Kmax) + 2u * DC_GUARD(P, kb - kGridBits, P.Kmax, 1));
        const float4 e0 = __ldg(tb), e1 = __ldg(tb + 1);
        teq = fmaf(fr, e0.y, e0.x);
        const float c1 = fmaf(fr, e0.w, e0.z);
        const float c2 = fmaf(fr, e1.y, e1.x);
        float fw;
        const uint32_t jw = DC_GUARD(P, grid_bits(fminf(t * P.inv_wdt, P.w_hi), fw) - kGridBits, P.w_n, 3);
        const float4 w0 = sW[2 * jw], w1 = sW[2 * jw + 1];
        u1w = fmaf(fw, w0.y, w0.x);
        u2w = fmaf(fw, w0.w, w0.z);
        O1 = fmaf(P.wscale, c1, fmaf(fw, w1.y, w1.x));
        O2 = fmaf(P.wscale, c2, fmaf(fw, w1.w, w1.z));
    }

    // A(t_eq, theta) (step 9): the beamlet's theta-interpolated row, linear in t_eq
    float fa;
    // t_eq >= 0 (an integral of rho >= 0, interpolated with non-negative
    // slopes), so only the upper end of the A row needs a clamp
    const uint32_t jb = grid_bits(fminf(teq * P.inv_adt, P.a_hi), fa);
    const float2 ar = __ldg(P.arow + (i * (uint32_t)P.a_nt + DC_GUARD(P, jb - kGridBits, P.a_nt, 2)));
    const float Av = fmaf(fa, ar.y, ar.x);

    // density correction (step 11), in pairs: -(k1, k2) with k = log2(e) f_u u^w,
    // and (omega_1, omega_2)
    const float2 nk = __fmul2_rn(make_float2(-ln.cu1, -ln.cu2x), make_float2(u1w, u2w));
    const float nk2y = LAT == kIso ? nk.y : -ln.cu2y * u2w;
    const float2 om = __fmul2_rn(make_float2(ln.cw1, ln.cw2), make_float2(O1, O2));
    const float om1 = fmaxf(om.x, 0.f), om2 = fmaxf(om.y, 0.f);

    // eqs. (3) and (2): the x and y profiles of each component together
    const float2 axy = make_float2(fabsf(x), fabsf(y));
    const float2 x0 = make_float2(P.x0, P.y0), nx0 = make_float2(-P.x0, -P.y0);
    const float2 p1 = penumbra2<PREC>(axy, make_float2(nk.x, nk.x), x0, nx0);
    const float2 p2 = penumbra2<PREC>(axy, make_float2(nk.y, nk2y), x0, nx0);
    const float F = fmaf(om1 * p1.x, p1.y, om2 * p2.x * p2.y);
    return F * Av * (s * s);
}

// Eq. (4) and its derivative with respect to the width u (natural units):
// with e1 = exp(-u ||x| - x0|), e2 = exp(-u (|x| + x0)),
// dp/du = ((x0 - |x|) e1 + (|x| + x0) e2) / 2 on both sides of |x| = x0.
__device__ __forceinline__ void penumbra_du(float ax, float u, float x0, float& p, float& dp)
{
    const float dd = ax - x0;
    const float e1 = ex2(-kLog2e * u * fabsf(dd));
    const float e2 = ex2(-kLog2e * u * (ax + x0));
    p = dd > 0.f ? 0.5f * (e1 - e2) : 1.f - 0.5f * (e1 + e2);
    dp = 0.5f * (fmaf(-dd, e1, 0.f) + (ax + x0) * e2);
}

// Backward pass of one pair (commissioning fit, Section 2.1): with
// c = w_v f_i, accumulates c dD_i(r)/d(entry) into the shared bins of the
// water tables u_1^w, u_2^w, omega_1^w, omega_2^w (the two samples around t);
// into the lane's per-voxel sums the derivatives with respect to the values
// f_u1(rho), f_u2(rho_hat), f_omega1(rho_hat), f_omega2(rho_hat) (scattered to
// the density-function bins once per work unit); and into gc the derivatives
// with respect to a common scale of b_1 and b_2 (omega_i^corr scales with it).
// Paper's lateral form, general (unmerged) tables, density correction on.
__device__ __forceinline__ void pair_grad(const PlanView& P, const float4 facv, const uint32_t i, const float sad,
                                          const float4* __restrict__ sW, const PairTest& pt, const float c,
                                          float* sgw, float gl[4], float gc[2])
{
    const float L = pt.L;
    const float t = L - pt.L_in;
    const float s = sad * rcp_approx(L);
    const float x = pt.pq.x * s, y = pt.pq.y * s;
    float fr;
    const uint32_t kb = grid_bits_mul(t, P.inv_d, fr);
    const float4* tb = P.tab + (i * (2u * (uint32_t)P.Kmax) + 2u * DC_GUARD(P, kb - kGridBits, P.Kmax, 1));
    const float4 e0 = __ldg(tb), e1 = __ldg(tb + 1);
    const float teq = fmaf(fr, e0.y, e0.x);
    const float c1 = fmaf(fr, e0.w, e0.z);
    const float c2 = fmaf(fr, e1.y, e1.x);
    float fw;
    const int jw = (int)DC_GUARD(P, grid_bits(fminf(t * P.inv_wdt, P.w_hi), fw) - kGridBits, P.w_n, 3);
    const float4 w0 = sW[2 * jw], w1 = sW[2 * jw + 1];
    const float u1w = fmaf(fw, w0.y, w0.x), u2w = fmaf(fw, w0.w, w0.z);
    const float o1w = fmaf(fw, w1.y, w1.x), o2w = fmaf(fw, w1.w, w1.z);
    float fa;
    const uint32_t jb = grid_bits(fminf(teq * P.inv_adt, P.a_hi), fa);
    const float2 ar = __ldg(P.arow + (i * (uint32_t)P.a_nt + DC_GUARD(P, jb - kGridBits, P.a_nt, 2)));
    const float Av = fmaf(fa, ar.y, ar.x);

    const float u1 = facv.x * u1w, u2 = facv.y * u2w;
    const float O1 = facv.z * (o1w + c1), O2 = facv.w * (o2w + c2);
    const float om1 = fmaxf(O1, 0.f), om2 = fmaxf(O2, 0.f);
    float p1x, d1x, p1y, d1y, p2x, d2x, p2y, d2y;
    penumbra_du(fabsf(x), u1, P.x0, p1x, d1x);
    penumbra_du(fabsf(y), u1, P.y0, p1y, d1y);
    penumbra_du(fabsf(x), u2, P.x0, p2x, d2x);
    penumbra_du(fabsf(y), u2, P.y0, p2y, d2y);
    const float K = c * Av * (s * s);
    const float g_om1 = O1 > 0.f ? K * p1x * p1y : 0.f;     // dD/d omega_1 (zero where the clamp holds)
    const float g_om2 = O2 > 0.f ? K * p2x * p2y : 0.f;
    const float g_u1 = K * om1 * fmaf(d1x, p1y, p1x * d1y);  // dD/d u_1
    const float g_u2 = K * om2 * fmaf(d2x, p2y, p2x * d2y);
    // water tables: val = w[jw] + fw (w[jw + 1] - w[jw])
    const int wn = P.w_n;
    const float a0 = 1.f - fw;
    atomicAdd(sgw + 0 * wn + jw, a0 * g_u1 * facv.x);
    atomicAdd(sgw + 1 * wn + jw, a0 * g_u2 * facv.y);
    atomicAdd(sgw + 2 * wn + jw, a0 * g_om1 * facv.z);
    atomicAdd(sgw + 3 * wn + jw, a0 * g_om2 * facv.w);
    if (jw + 1 < wn && fw != 0.f) {
        atomicAdd(sgw + 0 * wn + jw + 1, fw * g_u1 * facv.x);
        atomicAdd(sgw + 1 * wn + jw + 1, fw * g_u2 * facv.y);
        atomicAdd(sgw + 2 * wn + jw + 1, fw * g_om1 * facv.z);
        atomicAdd(sgw + 3 * wn + jw + 1, fw * g_om2 * facv.w);
    }
    gl[0] = fmaf(g_u1, u1w, gl[0]);
    gl[1] = fmaf(g_u2, u2w, gl[1]);
    gl[2] = fmaf(g_om1, o1w + c1, gl[2]);
    gl[3] = fmaf(g_om2, o2w + c2, gl[3]);
    gc[0] = fmaf(g_om1 * facv.z, c1, gc[0]);
    gc[1] = fmaf(g_om2 * facv.w, c2, gc[1]);
}

// The interpolation of a density-function table at density r (clamped to
// its domain), as k_factors reads it: entry j with weight 1 - w, j + 1 with w.
__device__ __forceinline__ void dens_bins(const PlanView& P, float r, int& j, float& w)
{
    const float sx = fminf(fmaxf((r - P.f_rho0) * P.inv_drho, 0.f), (float)(P.f_n - 1));
    j = min((int)sx, P.f_n - 2);
    w = sx - (float)j;
}

// Writes nw staged CSR entries of every lane (nw <= kRing).  A quarter-warp
// takes one lane's run at a time, 8 entries (one 32-byte sector of the column
// array once the run is aligned) per pass: first the leading 8 entries of all
// 32 runs, then entries 8..15 of the runs that are longer, four runs per pass.
// Plain write-back stores: with evict-first (streaming) stores the thorax9
// fill took 4.58 ms, with these 4.40 ms, for the same matrix.  Each staged
// entry is (column, value bits).
template <typename VT>
__device__ __forceinline__ void store_entry(int32_t* cols, VT* vals, int64_t g, int2 e)
{
    cols[g] = e.x;
    if (sizeof(VT) == 2)
        reinterpret_cast<__nv_bfloat16*>(vals)[g] = __float2bfloat16_rn(__int_as_float(e.y));
    else
        reinterpret_cast<float*>(vals)[g] = __int_as_float(e.y);
}

template <typename VT>
__device__ __forceinline__ void flush_runs(int32_t* cols, VT* vals, const int2* st, int lane, int nw, int64_t pos)
{
    // (a lane's run never passes the end of its row segment: flush_stage cuts
    // nw at pend - pos, and the DC_BOUNDS_CHECK build verifies it there)
    const int q = lane >> 3, j = lane & 7;
#pragma unroll 2
    for (int o4 = 0; o4 < 32; o4 += 4) {
        const int owner = o4 + q;
        const int c = __shfl_sync(0xffffffffu, nw, owner);
        const int64_t base = __shfl_sync(0xffffffffu, pos, owner);
        if (j < c)
            store_entry(cols, vals, base + j,
                        st[owner * kRingLd + (int)(((uint32_t)base + (uint32_t)j) & (kRing - 1))]);
    }
    uint32_t longer = __ballot_sync(0xffffffffu, nw > 8);
    while (longer) {
        uint32_t mq = longer;   // quarter q takes the q-th lowest set bit
#pragma unroll
        for (int t = 0; t < 3; ++t)
            if (t < q) mq &= mq - 1u;
        const int src = mq ? __ffs((int)mq) - 1 : 0;
        int c = __shfl_sync(0xffffffffu, nw, src);
        const int64_t base = __shfl_sync(0xffffffffu, pos, src);
        if (!mq) c = 0;
        if (j + 8 < c)
            store_entry(cols, vals, base + 8 + j,
                        st[src * kRingLd + (int)(((uint32_t)base + 8u + (uint32_t)j) & (kRing - 1))]);
#pragma unroll
        for (int t = 0; t < 4; ++t) longer &= longer - 1u;
    }
}

// Writes out the lanes' pending entries.  Except at the end of a work unit
// (`last`), a lane stops at the last 32-byte boundary of the column array
// inside its run and keeps the rest staged, so that DRAM sees whole sectors
// (a partly written sector evicted from L2 costs a read-modify-write); mis is
// the column array's offset from a 32-byte boundary, in entries.  A lane never
// writes past the end of its (voxel, beam) segment of the row.
__device__ __forceinline__ void flush_stage(const DoseArgs& a, const int2* st, int lane, int& cnt, int64_t& pos,
                                            int64_t pend, int mis, bool last)
{
    int nw = cnt;
    if (!last) {
        const int64_t end = ((pos + cnt + mis) & ~(int64_t)7) - mis;
        nw = end > pos ? (int)(end - pos) : 0;
    }
    nw = (int)min((int64_t)nw, pend - pos);
#if DC_BOUNDS_CHECK
    if (nw > 0 && (pos < a.rowptr[0] || pos + nw > a.rowptr[(int64_t)a.P.nx * a.P.ny * a.P.nz]))
        atomicCAS(a.P.chk, 0, 6);
#endif
    __syncwarp();
    if (a.value_dtype == DC_BF16)
        flush_runs(a.cols, reinterpret_cast<__nv_bfloat16*>(a.vals), st, lane, nw, pos);
    else
        flush_runs(a.cols, reinterpret_cast<float*>(a.vals), st, lane, nw, pos);
    __syncwarp();
    pos += nw;
    cnt -= nw;
}

// Evaluates one warp work unit: the 32 list entries starting at e0 of beam b
// (one voxel per lane) against the beamlets of the warp's union window.
template <int MODE, int NF, bool MERGED, int LAT, int PREC = 0>
__device__ __forceinline__ void process_unit(const DoseArgs& a, const int32_t vi, const int64_t e0, const int b,
                                             const float4* __restrict__ sW, int2* sst, float4* srow,
                                             const int lane, float4* sflu = nullptr, uint32_t* stc = nullptr)
{
    // the tensor-core form of 64 fluence vectors; its pair values in FP32
    // exponentials like the plain form
    constexpr bool TC = MODE == kDose && PREC == 2;
    constexpr int EP = PREC == 1 ? 1 : 0;
    static_assert(!TC || NF == 64, "the tensor-core form takes 64 fluence vectors");
    const PlanView& P = a.P;
    const int64_t V = (int64_t)P.nx * P.ny * P.nz;
    Lane ln;
    ln.valid = vi >= 0;
    const int64_t v = ln.valid ? vi : 0;
    const int ix = (int)(v % P.nx), iy = (int)((v / P.nx) % P.ny), iz = (int)(v / ((int64_t)P.nx * P.ny));
    // explicit fma: the count and fill passes must round these identically
    const float rx = fmaf((float)ix, P.dx, P.ox), ry = fmaf((float)iy, P.dy, P.oy),
                rz = fmaf((float)iz, P.dz, P.oz);
    const BeamDev& bm = P.beams[b];
    float4 facv = make_float4(0.f, 0.f, 0.f, 0.f);
    float gl[4] = {0.f, 0.f, 0.f, 0.f}, gc[2] = {0.f, 0.f};
    const float wgt = MODE == kGrad && ln.valid ? __ldg(a.wv + v) : 0.f;   // voxel weight of the backward pass
    if (MODE != kCount) {
        const float4 fac = __ldg(P.fac + v);   // f_u1(rho), f_u2(rho_hat), f_w1(rho_hat), f_w2(rho_hat)
        facv = fac;
        ln.cu1 = kLog2e * fac.x;
        ln.cu2x = ln.cu2y = kLog2e * fac.y;
        ln.cw1 = fac.z;
        ln.cw2 = fac.w;
        if (LAT == kItem) {
            // (log2(e) f_u2 along x, along y, f_w1, f_w2) of this (voxel, beam)
            const float4 lf = __ldg(P.lfac + e0 + lane);   // e0 + lane: guarded with the list entry (code 4)
            ln.cu2x = lf.x;
            ln.cu2y = lf.y;
            ln.cw1 = lf.z;
            ln.cw2 = lf.w;
        }
    }
    float acc[NF > 0 ? NF : 1];
#pragma unroll
    for (int q = 0; q < (NF > 0 ? NF : 1); ++q) acc[q] = 0.f;
    int32_t cnt = 0;
    int64_t pos = 0, pend = 0;
    const int mis = MODE == kFill ? (int)((reinterpret_cast<uintptr_t>(a.cols) >> 2) & 7) : 0;
    if (MODE == kFill && ln.valid) {
        pos = a.rowptr[v];
        for (int bb = 0; bb < b; ++bb) pos += a.bcount[(size_t)bb * V + v];
        pend = pos + a.bcount[(size_t)b * V + v];   // this beam's segment of the row
    }

    const float sx = __ldg(&bm.src[0]), sy = __ldg(&bm.src[1]), sz = __ldg(&bm.src[2]);
    const float sad = __ldg(&bm.sad);
    ln.vx = rx - sx; ln.vy = ry - sy; ln.vz = rz - sz;
    if (!ln.valid) ln.vx = __int_as_float(0x7fffffff);   // NaN: no pair test passes
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
        const uint32_t row = (uint32_t)(first + n * M);
        // the records of the row's window go to shared memory with one
        // coalesced load per lane, so the traversal reads them without a
        // global-memory round trip per beamlet
        for (int m0 = wmlo; m0 <= wmhi; m0 += row_max(MODE, NF)) {
        const int m1 = min(wmhi, m0 + row_max(MODE, NF) - 1);
        __syncwarp();
        if (m0 + lane <= m1) {
            const uint32_t ib = DC_GUARD(P, row + (uint32_t)(m0 + lane), P.B, 5);
            const float4* src = reinterpret_cast<const float4*>(P.bl) + 4u * ib;
            srow[3 * lane] = __ldg(src);
            srow[3 * lane + 1] = __ldg(src + 1);
            float4 q2 = __ldg(src + 2);
            // one fluence vector: the staged record carries f_i in place of the
            // theta weight (which only the table set-up uses)
            if (MODE != kCount && NF == 1) q2.w = __ldg(a.fluence + ib);
            srow[3 * lane + 2] = q2;
            if (MODE == kDose && NF > 1 && !TC) {
                // the beamlet's NF fluences beside its record (zero past a.nf),
                // as NF / 4 float4 whose order is rotated by the lane (fewer
                // bank conflicts among the lanes' stores)
                float4* f4 = sflu + (NF / 4) * lane;
#pragma unroll
                for (int j = 0; j < NF / 4; ++j) {
                    float f[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h)
                        f[h] = 4 * j + h < a.nf ? __ldg(a.fluence + ((4 * j + h) * (uint32_t)a.ldf + ib)) : 0.f;
                    f4[j ^ (lane & 3)] = make_float4(f[0], f[1], f[2], f[3]);
                }
            }
        }
        if (TC) {
            // the chunk's 64 BF16 fluences of beamlets m0 + 2j and m0 + 2j + 1
            // as pairs (lane: pair j, vectors nb .. nb + 15); zero past m1
            const int j = lane >> 2, nb = (lane & 3) * 16;
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
            uint4 f0 = z, f1 = z, g0 = z, g1 = z;
            if (m0 + 2 * j <= m1) {
                const uint4* src = a.fpack + (size_t)DC_GUARD(P, row + (uint32_t)(m0 + 2 * j), P.B, 5) * 8 + nb / 8;
                f0 = __ldg(src);
                f1 = __ldg(src + 1);
            }
            if (m0 + 2 * j + 1 <= m1) {
                const uint4* src = a.fpack + (size_t)DC_GUARD(P, row + (uint32_t)(m0 + 2 * j + 1), P.B, 5) * 8 + nb / 8;
                g0 = __ldg(src);
                g1 = __ldg(src + 1);
            }
            uint4* dst = reinterpret_cast<uint4*>(stc + kTcOffF + j * kTcRowF + nb);
            dst[0] = make_uint4(__byte_perm(f0.x, g0.x, 0x5410), __byte_perm(f0.x, g0.x, 0x7632),
                                __byte_perm(f0.y, g0.y, 0x5410), __byte_perm(f0.y, g0.y, 0x7632));
            dst[1] = make_uint4(__byte_perm(f0.z, g0.z, 0x5410), __byte_perm(f0.z, g0.z, 0x7632),
                                __byte_perm(f0.w, g0.w, 0x5410), __byte_perm(f0.w, g0.w, 0x7632));
            dst[2] = make_uint4(__byte_perm(f1.x, g1.x, 0x5410), __byte_perm(f1.x, g1.x, 0x7632),
                                __byte_perm(f1.y, g1.y, 0x5410), __byte_perm(f1.y, g1.y, 0x7632));
            dst[3] = make_uint4(__byte_perm(f1.z, g1.z, 0x5410), __byte_perm(f1.z, g1.z, 0x7632),
                                __byte_perm(f1.w, g1.w, 0x5410), __byte_perm(f1.w, g1.w, 0x7632));
        }
        __syncwarp();
        // two beamlets per trip: their independent loads and arithmetic
        // interleave (measured: 3.10 -> 2.90 ms on thorax9; 3 and 4 were slower)
#pragma unroll 2
        for (int m = m0; m <= m1; ++m) {
            const uint32_t i = row + (uint32_t)m;
            const float4* rq = srow + 3 * (m - m0);
            const PairTest pt = pair_test(P, ln, rq[0], rq[1], rq[2]);
            if (MODE == kCount) {
                cnt += pt.in ? 1 : 0;
                continue;
            }
            if (MODE == kGrad) {
                if (pt.in && wgt != 0.f)
                    pair_grad(P, facv, i, sad, sW, pt, wgt * rq[2].w,
                              reinterpret_cast<float*>(sst), gl, gc);
                continue;
            }
            if (TC) {
                // D (zero outside the pair) into the lane's row of the chunk's tile
                float D = 0.f;
                if (pt.in) D = pair_eval<MERGED, LAT, 0>(P, ln, i, sad, sW, pt);
                const int c = m - m0;
                reinterpret_cast<__nv_bfloat16*>(stc)[2 * ((lane >> 4) * kTcTileD + (c >> 1) * kTcRowD + (lane & 15)) +
                                                      (c & 1)] = __float2bfloat16_rn(D);
                continue;
            }
            if (MODE == kDose) {
                if (NF == 1) cnt += pt.in ? 1 : 0;
                if (pt.in) {
                    const float D = pair_eval<MERGED, LAT, EP>(P, ln, i, sad, sW, pt);
                    if (NF == 1) {
                        acc[0] = fmaf(rq[2].w, D, acc[0]);
                    } else {
                        const float4* f4 = sflu + (NF / 4) * (m - m0);
#pragma unroll
                        for (int q4 = 0; q4 < NF / 4; ++q4) {
                            const float4 f = f4[q4 ^ ((m - m0) & 3)];
                            acc[4 * q4] = fmaf(f.x, D, acc[4 * q4]);
                            acc[4 * q4 + 1] = fmaf(f.y, D, acc[4 * q4 + 1]);
                            acc[4 * q4 + 2] = fmaf(f.z, D, acc[4 * q4 + 2]);
                            acc[4 * q4 + 3] = fmaf(f.w, D, acc[4 * q4 + 3]);
                        }
                    }
                }
            } else {
                if (pt.in) {
                    const float D = pair_eval<MERGED, LAT, 0>(P, ln, i, sad, sW, pt);
                    sst[lane * kRingLd + (int)(((uint32_t)pos + (uint32_t)cnt) & (kRing - 1))] =
                        make_int2((int)i, __float_as_int(D));
                    ++cnt;
                    if (NF == 1) acc[0] = fmaf(rq[2].w, D, acc[0]);   // eq. (1) from the same evaluation
                }
                if (__any_sync(0xffffffffu, cnt >= kRing)) flush_stage(a, sst, lane, cnt, pos, pend, mis, false);
            }
        }
        if (TC) {
            // Y[32][64] += D[32][16] F[16][64]: two 16-row tiles, eight 8-vector tiles
            __syncwarp();
            const int g = lane >> 2, t4 = lane & 3;
            uint32_t fa[2][4];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const uint32_t* d0 = stc + t * kTcTileD;
                fa[t][0] = d0[t4 * kTcRowD + g];
                fa[t][1] = d0[t4 * kTcRowD + g + 8];
                fa[t][2] = d0[(t4 + 4) * kTcRowD + g];
                fa[t][3] = d0[(t4 + 4) * kTcRowD + g + 8];
            }
            const uint32_t* sf = stc + kTcOffF;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t b0 = sf[t4 * kTcRowF + 8 * u + g], b1 = sf[(t4 + 4) * kTcRowF + 8 * u + g];
#pragma unroll
                for (int t = 0; t < 2; ++t) mma_bf16(acc + (t * 8 + u) * 4, fa[t][0], fa[t][1], fa[t][2], fa[t][3], b0, b1);
            }
        }
        }
    }
    if (MODE == kGrad) {
        if (ln.valid && wgt != 0.f) {
            // the per-voxel derivatives go to the bins of rho (f_u1) and rho_hat (the others)
            float* sgd = reinterpret_cast<float*>(sst) + 4 * P.w_n;
            int j;
            float w;
            dens_bins(P, __ldg(P.rho + v), j, w);
            atomicAdd(sgd + j, (1.f - w) * gl[0]);
            atomicAdd(sgd + j + 1, w * gl[0]);
            dens_bins(P, __ldg(P.rhos + v), j, w);
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                atomicAdd(sgd + q * P.f_n + j, (1.f - w) * gl[q]);
                atomicAdd(sgd + q * P.f_n + j + 1, w * gl[q]);
            }
            atomicAdd(sgd + 4 * P.f_n, gc[0]);
            atomicAdd(sgd + 4 * P.f_n + 1, gc[1]);
        }
    } else if (TC) {
        // accumulator (tile t, vectors 8u .. 8u + 7, element 2h + e) is row
        // 16t + 8h + g (that lane's voxel), vector 8u + 2 t4 + e
        const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int vr = __shfl_sync(0xffffffffu, vi, 16 * t + 8 * h + g);
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int n = 8 * u + 2 * t4 + e;
                        if (vr >= 0 && n < a.nf) a.part[((size_t)b * NF + n) * V + vr] = acc[(t * 8 + u) * 4 + 2 * h + e];
                    }
            }
    } else if (MODE == kFill) {
        flush_stage(a, sst, lane, cnt, pos, pend, mis, true);
        if (NF == 1 && ln.valid) a.part[(size_t)b * V + v] = acc[0];
    } else if (ln.valid) {
        if (MODE == kDose) {
#pragma unroll
            for (int q = 0; q < NF; ++q)
                if (q < a.nf) a.part[((size_t)b * NF + q) * V + v] = acc[q];
            if (NF == 1 && a.count_out) a.count_out[(size_t)b * V + v] = cnt;
        } else {
            a.bcount[(size_t)b * V + v] = cnt;
        }
    }
}

// One warp work unit = 32 consecutive entries of one beam's voxel list (voxels
// of one or two neighbouring beam's-eye-view cells; -1 entries are padding).
// Persistent CTAs take units from a global counter.
// Register budgets: 48 per thread for the single-fluence dose (5 CTAs per
// SM), 64 for the pair count and the CSR fill (4 CTAs; the fill's extra state
// would otherwise be recomputed in the hot loop), 80 for 16 fluence vectors,
// 128 for 32 or 64 (their accumulators).
template <int MODE, int NF>
constexpr int min_ctas()
{
    return MODE == kCount || MODE == kFill || MODE == kGrad ? 4 : (NF == 1 ? 5 : (NF == 16 ? 3 : 2));
}

template <int MODE, int NF, bool MERGED, int LAT, int PREC>
__global__ void __launch_bounds__(kThreads, min_ctas<MODE, NF>()) k_pairs(const DoseArgs a)
{
    extern __shared__ float4 smem[];
    __shared__ int64_t s_base[kMaxBeams + 1];
    const PlanView& P = a.P;
    float4* sW = smem;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4* sstage = smem + (MERGED ? 0 : 2 * P.w_n);
    int2* sst = reinterpret_cast<int2*>(sstage) + warp * (32 * kRingLd);
    // backward pass: the CTA's gradient bins (4 water tables, 4 density
    // functions, 2 scales of b) instead of the CSR staging
    float* sgrad = reinterpret_cast<float*>(sstage);
    const int ngrad = 4 * P.w_n + 4 * P.f_n + 2;
    if (MODE == kGrad) {
        sst = reinterpret_cast<int2*>(sgrad);
        for (int q = threadIdx.x; q < ngrad; q += blockDim.x) sgrad[q] = 0.f;
    }
    static_assert(valid_nf(NF) || MODE != kDose, "16, 32 or 64 fluence vectors per pass");
    constexpr bool TC = MODE == kDose && PREC == 2;
    __shared__ float4 s_row[kWarps][3 * row_max(MODE, NF)];
    // several fluence vectors: each staged beamlet's fluences (NF per record),
    // or the tensor-core form's operand tiles
    __shared__ float4 s_flu[NF > 1 && !TC ? kWarps : 1][NF > 1 && !TC ? row_max(MODE, NF) * NF / 4 : 1];
    __shared__ __align__(16) uint32_t s_tc[TC ? kWarps : 1][TC ? kTcWords : 4];
    if (TC) {
        // columns past a partial chunk keep earlier (finite) pair values, which
        // meet zero fluences; nothing may be left uninitialised
        for (int q = threadIdx.x & 31; q < kTcOffF; q += 32) s_tc[threadIdx.x >> 5][q] = 0u;
    }
    // the water tables are read from shared memory unless merged into the depth tables
    if (MODE != kCount && !MERGED)
        for (int q = threadIdx.x; q < 2 * P.w_n; q += blockDim.x) sW[q] = __ldg(P.water + q);
    for (int q = threadIdx.x; q <= P.n_beams; q += blockDim.x) s_base[q] = a.base[q];
    __syncthreads();
    const int total = a.work[0];

    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(a.work + 1, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= total) break;
        const int64_t e0 = (int64_t)DC_GUARD(P, w, (s_base[P.n_beams] + 31) / 32, 4) * 32;
        int b = 0;
        while (b + 1 < P.n_beams && s_base[b + 1] <= e0) ++b;
        const int32_t vi = __ldg(a.items + e0 + lane);
        process_unit<MODE, NF, MERGED, LAT, PREC>(a, vi, e0, b, sW, sst, s_row[warp], lane,
                                                  NF > 1 && !TC ? s_flu[NF > 1 && !TC ? warp : 0] : nullptr,
                                                  TC ? s_tc[TC ? warp : 0] : nullptr);
    }
    if (MODE == kGrad) {
        __syncthreads();
        for (int q = threadIdx.x; q < ngrad; q += blockDim.x) {
            const float g = sgrad[q];
            if (g == 0.f) continue;
            if (q < 4 * P.w_n) atomicAdd(a.g_water + q, g);
            else if (q < 4 * P.w_n + 4 * P.f_n) atomicAdd(a.g_dens + (q - 4 * P.w_n), g);
            else atomicAdd(a.g_corr + (q - 4 * P.w_n - 4 * P.f_n), g);
        }
    }
}

// ---------------------------------------------------------------------------
// Pair counts of the matrix pattern, several voxels per lane: a warp takes NV
// consecutive work units of one beam (lane l holds entry l of each) and walks
// the union of their windows; each staged beamlet record is tested against
// all of the lane's voxels, so the record reads and the loop's bookkeeping
// are shared by 32 NV pair tests instead of 32.  The voxels, the windows and
// pair_test are computed as process_unit computes them, so the counts are
// exactly the fill's entries per (voxel, beam).  A group of units that
// straddles two beams is taken one unit at a time.
struct CountVoxel {
    Lane ln;
    bool live;
    float ca, cc, rw;
    int64_t v;
};

__device__ __forceinline__ CountVoxel count_voxel(const PlanView& P, const BeamDev& bm, int32_t vi, float sad)
{
    CountVoxel c;
    c.ln.valid = vi >= 0;
    c.v = c.ln.valid ? vi : 0;
    const int ix = (int)(c.v % P.nx), iy = (int)((c.v / P.nx) % P.ny), iz = (int)(c.v / ((int64_t)P.nx * P.ny));
    const float rx = fmaf((float)ix, P.dx, P.ox), ry = fmaf((float)iy, P.dy, P.oy), rz = fmaf((float)iz, P.dz, P.oz);
    const float sx = __ldg(&bm.src[0]), sy = __ldg(&bm.src[1]), sz = __ldg(&bm.src[2]);
    c.ln.vx = rx - sx;
    c.ln.vy = ry - sy;
    c.ln.vz = rz - sz;
    if (!c.ln.valid) c.ln.vx = __int_as_float(0x7fffffff);   // NaN: no pair test passes
    const float zz = c.ln.vx * __ldg(&bm.ez[0]) + c.ln.vy * __ldg(&bm.ez[1]) + c.ln.vz * __ldg(&bm.ez[2]);
    const float pa = c.ln.vx * __ldg(&bm.ex[0]) + c.ln.vy * __ldg(&bm.ex[1]) + c.ln.vz * __ldg(&bm.ex[2]);
    const float pc = c.ln.vx * __ldg(&bm.ey[0]) + c.ln.vy * __ldg(&bm.ey[1]) + c.ln.vz * __ldg(&bm.ey[2]);
    c.live = c.ln.valid && zz > 1e-3f;
    const float sz_ = sad / zz;
    c.ca = pa * sz_;
    c.cc = pc * sz_;
    c.rw = c.live ? (P.roi * sz_ * __ldg(&bm.inv_cos_max)) * 1.0005f + 1e-3f : 0.f;
    return c;
}

// The voxel's range of beamlet rows, and of columns in row n (empty: lo > hi).
__device__ __forceinline__ void count_rows(const PlanView& P, const CountVoxel& c, int N, float hfy, int& lo, int& hi)
{
    lo = INT_MAX;
    hi = INT_MIN;
    if (c.live) {
        lo = max(0, (int)ceilf((c.cc - c.rw + hfy) / P.by - 0.5f));
        hi = min(N - 1, (int)floorf((c.cc + c.rw + hfy) / P.by - 0.5f));
    }
}

__device__ __forceinline__ void count_cols(const PlanView& P, const CountVoxel& c, int n, int M, float hfx, float hfy,
                                           int& lo, int& hi)
{
    const float dc_ = c.cc - (-hfy + (n + 0.5f) * P.by);
    const float h2 = c.rw * c.rw - dc_ * dc_;
    lo = INT_MAX;
    hi = INT_MIN;
    if (c.live && h2 >= 0.f) {
        const float hx = sqrtf(h2);
        lo = max(0, (int)ceilf((c.ca - hx + hfx) / P.bx - 0.5f));
        hi = min(M - 1, (int)floorf((c.ca + hx + hfx) / P.bx - 0.5f));
    }
}

template <int NV>
__device__ __forceinline__ void count_units(const DoseArgs& a, const int64_t e0, const int b, float4* srow, int lane)
{
    const PlanView& P = a.P;
    const int64_t V = (int64_t)P.nx * P.ny * P.nz;
    const BeamDev& bm = P.beams[b];
    const float sad = __ldg(&bm.sad);
    const int M = __ldg(&bm.M), N = __ldg(&bm.N), first = __ldg(&bm.first);
    const float hfx = __ldg(&bm.half_fx), hfy = __ldg(&bm.half_fy);
    CountVoxel c[NV];
    int nlo = INT_MAX, nhi = INT_MIN;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        c[k] = count_voxel(P, bm, __ldg(a.items + e0 + 32 * k + lane), sad);
        int lo, hi;
        count_rows(P, c[k], N, hfy, lo, hi);
        nlo = min(nlo, lo);
        nhi = max(nhi, hi);
    }
    int cnt[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) cnt[k] = 0;
    const int wnlo = __reduce_min_sync(0xffffffffu, nlo);
    const int wnhi = __reduce_max_sync(0xffffffffu, nhi);
    for (int n = wnlo; n <= wnhi; ++n) {
        int mlo = INT_MAX, mhi = INT_MIN;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            int lo, hi;
            count_cols(P, c[k], n, M, hfx, hfy, lo, hi);
            mlo = min(mlo, lo);
            mhi = max(mhi, hi);
        }
        const int wmlo = __reduce_min_sync(0xffffffffu, mlo);
        const int wmhi = __reduce_max_sync(0xffffffffu, mhi);
        const uint32_t row = (uint32_t)(first + n * M);
        for (int m0 = wmlo; m0 <= wmhi; m0 += 32) {
            const int m1 = min(wmhi, m0 + 31);
            __syncwarp();
            if (m0 + lane <= m1) {
                const uint32_t ib = DC_GUARD(P, row + (uint32_t)(m0 + lane), P.B, 5);
                const float4* src = reinterpret_cast<const float4*>(P.bl) + 4u * ib;
                srow[3 * lane] = __ldg(src);
                srow[3 * lane + 1] = __ldg(src + 1);
                srow[3 * lane + 2] = __ldg(src + 2);
            }
            __syncwarp();
#pragma unroll 2
            for (int m = m0; m <= m1; ++m) {
                const float4* rq = srow + 3 * (m - m0);
                const float4 q0 = rq[0], q1 = rq[1], q2 = rq[2];
#pragma unroll
                for (int k = 0; k < NV; ++k) cnt[k] += pair_test(P, c[k].ln, q0, q1, q2).in ? 1 : 0;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k)
        if (c[k].ln.valid) a.bcount[(size_t)b * V + c[k].v] = cnt[k];
}

template <int NV>
__global__ void __launch_bounds__(kThreads, NV <= 2 ? 4 : (NV == 3 ? 3 : 2)) k_count_units(const DoseArgs a)
{
    __shared__ int64_t s_base[kMaxBeams + 1];
    __shared__ float4 s_row[kWarps][3 * 32];
    const PlanView& P = a.P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q <= P.n_beams; q += blockDim.x) s_base[q] = a.base[q];
    __syncthreads();
    const int units = a.work[0];
    const int groups = (units + NV - 1) / NV;
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(a.work + 1, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= groups) break;
        const int u0 = NV * w;
        const int64_t e0 = (int64_t)DC_GUARD(P, u0, (s_base[P.n_beams] + 31) / 32, 4) * 32;
        int b = 0;
        while (b + 1 < P.n_beams && s_base[b + 1] <= e0) ++b;
        // all NV units in this beam: together; else one at a time
        if (u0 + NV <= units && e0 + 32 * NV <= s_base[b + 1]) {
            count_units<NV>(a, e0, b, s_row[warp], lane);
        } else {
            for (int k = 0; k < NV && u0 + k < units; ++k) {
                const int64_t ek = e0 + 32 * k;
                int bk = b;
                while (bk + 1 < P.n_beams && s_base[bk + 1] <= ek) ++bk;
                count_units<1>(a, ek, bk, s_row[warp], lane);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The SpMM's block-sparse BF16 matrix straight from the pair evaluation, with
// no CSR in between.  A warp's work unit (32 consecutive entries of a beam's
// voxel list) lies inside one row-block of 128 entries.  Mark pass: the unit's
// pair tests, as the count pass makes them, and the bit of every 4 x 4 beamlet
// patch holding one of its pairs in the row-block's bitmap.  Fill pass: the
// unit walks its window patch by patch (bands of four beamlet rows, patches
// left to right), evaluates the patch's 16 beamlets, and writes each lane's
// 16 BF16 values as two 16-byte pieces of the patch's tile: a warp's store
// fills four 128-byte cores.

__device__ __forceinline__ int unit_row_block(const PatchTiles& t, const DoseArgs& a, int64_t e0, int b, int& row0)
{
    const int64_t off = e0 - __ldg(a.base + b);
    row0 = (int)(off & 127);
    return __ldg(t.rb_first + b) + (int)(off >> 7);
}

// NV consecutive units of one row-block at once, as count_units takes them:
// lane l holds entry l of each, and every staged beamlet record is tested
// against all of the lane's voxels.
template <int NV>
__device__ __forceinline__ void mark_units(const DoseArgs& a, const PatchTiles& t, const int64_t e0, const int b,
                                           float4* srow, const int lane)
{
    const PlanView& P = a.P;
    const BeamDev& bm = P.beams[b];
    const float sad = __ldg(&bm.sad);
    const int M = __ldg(&bm.M), N = __ldg(&bm.N), first = __ldg(&bm.first);
    const float hfx = __ldg(&bm.half_fx), hfy = __ldg(&bm.half_fy);
    CountVoxel c[NV];
    int nlo = INT_MAX, nhi = INT_MIN;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        c[k] = count_voxel(P, bm, __ldg(a.items + e0 + 32 * k + lane), sad);
        int lo, hi;
        count_rows(P, c[k], N, hfy, lo, hi);
        nlo = min(nlo, lo);
        nhi = max(nhi, hi);
    }
    const int wnlo = __reduce_min_sync(0xffffffffu, nlo);
    const int wnhi = __reduce_max_sync(0xffffffffu, nhi);
    int row0;
    const int rb = unit_row_block(t, a, e0, b, row0);
    uint32_t* mk = t.marks + (size_t)rb * t.words;
    const int MB = (M + 3) >> 2;
    int last = -1;
    for (int n = wnlo; n <= wnhi; ++n) {
        int mlo = INT_MAX, mhi = INT_MIN;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            int lo, hi;
            count_cols(P, c[k], n, M, hfx, hfy, lo, hi);
            mlo = min(mlo, lo);
            mhi = max(mhi, hi);
        }
        const int wmlo = __reduce_min_sync(0xffffffffu, mlo);
        const int wmhi = __reduce_max_sync(0xffffffffu, mhi);
        const uint32_t row = (uint32_t)(first + n * M);
        for (int m0 = wmlo; m0 <= wmhi; m0 += 32) {
            const int m1 = min(wmhi, m0 + 31);
            __syncwarp();
            if (m0 + lane <= m1) {
                const uint32_t ib = DC_GUARD(P, row + (uint32_t)(m0 + lane), P.B, 5);
                const float4* src = reinterpret_cast<const float4*>(P.bl) + 4u * ib;
                srow[3 * lane] = __ldg(src);
                srow[3 * lane + 1] = __ldg(src + 1);
                srow[3 * lane + 2] = __ldg(src + 2);
            }
            __syncwarp();
            for (int m = m0; m <= m1; ++m) {
                const float4* rq = srow + 3 * (m - m0);
                const float4 q0 = rq[0], q1 = rq[1], q2 = rq[2];
                bool in = false;
#pragma unroll
                for (int k = 0; k < NV; ++k) in = in || pair_test(P, c[k].ln, q0, q1, q2).in;
                if (__any_sync(0xffffffffu, in)) {
                    const int patch = (n >> 2) * MB + (m >> 2);
                    if (patch != last) {
                        if (lane == 0) atomicOr(mk + DC_GUARD(P, patch >> 5, t.words, 7), 1u << (patch & 31));
                        last = patch;
                    }
                }
            }
        }
    }
}

// two units per warp where they share a beam and a row-block (one at a time otherwise)
__global__ void __launch_bounds__(kThreads, 4) k_mark_patches(const DoseArgs a, const PatchTiles t)
{
    __shared__ int64_t s_base[kMaxBeams + 1];
    __shared__ float4 s_row[kWarps][3 * 32];
    const PlanView& P = a.P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q <= P.n_beams; q += blockDim.x) s_base[q] = a.base[q];
    __syncthreads();
    const int units = a.work[0];
    const int groups = (units + 1) / 2;
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(a.work + 1, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= groups) break;
        const int u0 = 2 * w;
        const int64_t e0 = (int64_t)DC_GUARD(P, u0, (s_base[P.n_beams] + 31) / 32, 4) * 32;
        int b = 0;
        while (b + 1 < P.n_beams && s_base[b + 1] <= e0) ++b;
        if (u0 + 1 < units && e0 + 64 <= s_base[b + 1] && ((e0 - s_base[b]) >> 7) == ((e0 + 32 - s_base[b]) >> 7)) {
            mark_units<2>(a, t, e0, b, s_row[warp], lane);
        } else {
            mark_units<1>(a, t, e0, b, s_row[warp], lane);
            if (u0 + 1 < units) {
                const int64_t e1 = e0 + 32;
                int b1 = b;
                while (b1 + 1 < P.n_beams && s_base[b1 + 1] <= e1) ++b1;
                mark_units<1>(a, t, e1, b1, s_row[warp], lane);
            }
        }
    }
}

template <bool MERGED, int LAT>
__device__ __forceinline__ void tile_unit(const DoseArgs& a, const PatchTiles& t, const int32_t vi, const int64_t e0,
                                          const int b, const float4* __restrict__ sW, float4* srow,
                                          uint32_t* sval, const int lane)
{
    const PlanView& P = a.P;
    Lane ln;
    ln.valid = vi >= 0;
    const int64_t v = ln.valid ? vi : 0;
    const int ix = (int)(v % P.nx), iy = (int)((v / P.nx) % P.ny), iz = (int)(v / ((int64_t)P.nx * P.ny));
    // the same roundings as the mark pass's count_voxel
    const float rx = fmaf((float)ix, P.dx, P.ox), ry = fmaf((float)iy, P.dy, P.oy),
                rz = fmaf((float)iz, P.dz, P.oz);
    const BeamDev& bm = P.beams[b];
    const float4 fac = __ldg(P.fac + v);
    ln.cu1 = kLog2e * fac.x;
    ln.cu2x = ln.cu2y = kLog2e * fac.y;
    ln.cw1 = fac.z;
    ln.cw2 = fac.w;
    if (LAT == kItem) {
        const float4 lf = __ldg(P.lfac + e0 + lane);
        ln.cu2x = lf.x;
        ln.cu2y = lf.y;
        ln.cw1 = lf.z;
        ln.cw2 = lf.w;
    }
    const float sx = __ldg(&bm.src[0]), sy = __ldg(&bm.src[1]), sz = __ldg(&bm.src[2]);
    const float sad = __ldg(&bm.sad);
    ln.vx = rx - sx;
    ln.vy = ry - sy;
    ln.vz = rz - sz;
    if (!ln.valid) ln.vx = __int_as_float(0x7fffffff);   // NaN: no pair test passes
    const float zz = ln.vx * __ldg(&bm.ez[0]) + ln.vy * __ldg(&bm.ez[1]) + ln.vz * __ldg(&bm.ez[2]);
    const float pa = ln.vx * __ldg(&bm.ex[0]) + ln.vy * __ldg(&bm.ex[1]) + ln.vz * __ldg(&bm.ex[2]);
    const float pc = ln.vx * __ldg(&bm.ey[0]) + ln.vy * __ldg(&bm.ey[1]) + ln.vz * __ldg(&bm.ey[2]);
    const int M = __ldg(&bm.M), N = __ldg(&bm.N), first = __ldg(&bm.first);
    const float hfx = __ldg(&bm.half_fx), hfy = __ldg(&bm.half_fy);
    const bool live = ln.valid && zz > 1e-3f;
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
    int row0;
    const int rb = unit_row_block(t, a, e0, b, row0);
    const int row = row0 + lane;
    const int MB = (M + 3) >> 2;
    const uint32_t* mk = t.marks + (size_t)rb * t.words;
    const uint16_t* wp = t.wprefix + (size_t)rb * t.words;
    if (wnlo > wnhi) return;
    for (int pb = wnlo >> 2; pb <= (wnhi >> 2); ++pb) {
        // the band's beamlet columns: the union over its rows of the lanes' ROI chords
        int mlo = INT_MAX, mhi = INT_MIN;
        for (int r = 0; r < 4; ++r) {
            const int n = 4 * pb + r;
            if (!live || n < nlo || n > nhi) continue;
            const float dc_ = cc - (-hfy + (n + 0.5f) * P.by);
            const float h2 = rw * rw - dc_ * dc_;
            if (h2 < 0.f) continue;
            const float hx = sqrtf(h2);
            mlo = min(mlo, max(0, (int)ceilf((ca - hx + hfx) / P.bx - 0.5f)));
            mhi = max(mhi, min(M - 1, (int)floorf((ca + hx + hfx) / P.bx - 0.5f)));
        }
        const int wmlo = __reduce_min_sync(0xffffffffu, mlo);
        const int wmhi = __reduce_max_sync(0xffffffffu, mhi);
        if (wmlo > wmhi) continue;
        for (int X = wmlo >> 2; X <= (wmhi >> 2); ++X) {
            // the patch's 16 beamlet records (beamlets past the grid's edge get
            // an entry depth no pair reaches)
            __syncwarp();
            if (lane < 16) {
                const int n = 4 * pb + (lane >> 2), m = 4 * X + (lane & 3);
                float4 q0 = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000)), q1 = make_float4(0.f, 0.f, 0.f, 0.f),
                       q2 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (n < N && m < M) {
                    const uint32_t ib = DC_GUARD(P, (uint32_t)(first + n * M + m), P.B, 5);
                    const float4* src = reinterpret_cast<const float4*>(P.bl) + 4u * ib;
                    q0 = __ldg(src);
                    q1 = __ldg(src + 1);
                    q2 = __ldg(src + 2);
                }
                srow[3 * lane] = q0;
                srow[3 * lane + 1] = q1;
                srow[3 * lane + 2] = q2;
            }
            __syncwarp();
            // the lane's 16 values, two BF16 per word (word j: columns 2j, 2j + 1)
            bool any = false;
#pragma unroll 1
            for (int j = 0; j < 8; ++j) {
                uint32_t word = 0u;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = 2 * j + h;
                    const float4* rq = srow + 3 * k;
                    const PairTest pt = pair_test(P, ln, rq[0], rq[1], rq[2]);
                    if (pt.in) {
                        const uint32_t i = (uint32_t)(first + (4 * pb + (k >> 2)) * M + 4 * X + (k & 3));
                        const float D = pair_eval<MERGED, LAT, 0>(P, ln, i, sad, sW, pt);
                        word |= (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(D)) << (16 * h);
                        any = true;
                    }
                }
                sval[9 * lane + j] = word;
            }
            if (__any_sync(0xffffffffu, any)) {
                // the patch's chunk: the row-block's chunks before it
                const int patch = pb * MB + X;
                const int wi = DC_GUARD(P, patch >> 5, t.words, 7);
                const int ch = __ldg(wp + wi) + __popc(__ldg(mk + wi) & ((1u << (patch & 31)) - 1u));
                uint4* tile = reinterpret_cast<uint4*>(t.tiles + (size_t)(__ldg(t.chunk_off + rb) + ch) * (128 * 16));
                // k-block h of the chunk is core (row / 8) * 2 + h; the row's 8 values of it are 16 contiguous bytes
                const uint32_t* w = sval + 9 * lane;
                tile[((row >> 3) * 2) * 8 + (row & 7)] = make_uint4(w[0], w[1], w[2], w[3]);
                tile[((row >> 3) * 2 + 1) * 8 + (row & 7)] = make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
    }
}

template <bool MERGED, int LAT>
__global__ void __launch_bounds__(kThreads, 4) k_tile_fill(const DoseArgs a, const PatchTiles t)
{
    extern __shared__ float4 smem[];
    __shared__ int64_t s_base[kMaxBeams + 1];
    __shared__ float4 s_row[kWarps][3 * 16];
    __shared__ uint32_t s_val[kWarps][32 * 9];   // per lane 8 words, one of padding (no bank conflicts)
    const PlanView& P = a.P;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4* sW = smem;
    if (!MERGED)
        for (int q = threadIdx.x; q < 2 * P.w_n; q += blockDim.x) sW[q] = __ldg(P.water + q);
    for (int q = threadIdx.x; q <= P.n_beams; q += blockDim.x) s_base[q] = a.base[q];
    __syncthreads();
    const int total = a.work[0];
    for (;;) {
        int w = 0;
        if (lane == 0) w = atomicAdd(a.work + 1, 1);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= total) break;
        const int64_t e0 = (int64_t)DC_GUARD(P, w, (s_base[P.n_beams] + 31) / 32, 4) * 32;
        int b = 0;
        while (b + 1 < P.n_beams && s_base[b + 1] <= e0) ++b;
        const int32_t vi = __ldg(a.items + e0 + lane);
        tile_unit<MERGED, LAT>(a, t, vi, e0, b, sW, s_row[warp], s_val[warp], lane);
    }
}

// voxels per lane in the pair-count pass (measured on thorax9: 2 -> 0.722 ms,
// 3 -> 0.725 ms, 4 -> 0.796 ms; one voxel per lane, the pair kernel's count
// mode, took 0.847 ms)
constexpr int kCountVoxels = 2;

// ---------------------------------------------------------------------------
// Several plans in one persistent launch.  The plans are grouped by lateral
// form (per-voxel or per-item factors); a group runs on the merged depth tables
// when all its plans have them, else on the general tables (which every plan
// keeps).  The work units of a group's plans (one fluence vector each) form
// one range, and
// a warp takes the next unit from the group's counter, finds its plan and
// beam, and runs the same per-unit body as k_pairs, specialised for the group
// (no run-time choice of variant in the hot loop).  The plans' arguments travel
// as one grid-constant kernel parameter, so the hot loop reads them from the
// constant bank as k_pairs does.  When every plan uses the same water tables
// (one commissioned beam model), they are staged in shared memory once per
// CTA; otherwise each plan's are read through L1.
constexpr int kMaxBatch = 64;
constexpr int kBatchGroups = 4;   // (per-voxel or per-item lateral factors) x (FP32 or BF16 exponentials)

struct BatchParams {
    DoseArgs a[kMaxBatch];
};
static_assert(sizeof(BatchParams) + 64 + 72 <= 32764, "kernel parameter space");

// The plans of one group: indices into BatchParams::a.
struct BatchGroup {
    int8_t j[kMaxBatch];
    int n;
};

// prefix[q] = units of the group's plans 0..q-1 (the unit counts were written
// by each plan's binning on the device); resets the group's work counter.
__global__ void k_batch_prefix(const DoseArgs* __restrict__ args, const BatchGroup g, int64_t* __restrict__ prefix,
                               unsigned int* __restrict__ counter)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t s = 0;
    for (int q = 0; q < g.n; ++q) {
        prefix[q] = s;
        s += *args[g.j[q]].work;
    }
    prefix[g.n] = s;
    *counter = 0u;
}

// MINB: CTAs per SM the register budget is set for (4: 64 registers; 5: 48).
// SHARED_W: all plans share the water tables of plan 0.
template <int MINB, bool SHARED_W, bool MERGED, int LAT, int PREC>
__global__ void __launch_bounds__(kThreads, MINB) k_pairs_batch(const __grid_constant__ BatchParams bp,
                                                                const __grid_constant__ BatchGroup g,
                                                                const int64_t* __restrict__ prefix,
                                                                unsigned int* __restrict__ counter)
{
    extern __shared__ float4 smem[];
    __shared__ int64_t s_pre[kMaxBatch + 1];
    __shared__ float4 s_row[kWarps][3 * row_max(kDose)];
    const int n = g.n;
    for (int q = threadIdx.x; q <= n; q += blockDim.x) s_pre[q] = prefix[q];
    if (SHARED_W && !MERGED)
        for (int q = threadIdx.x; q < 2 * bp.a[0].P.w_n; q += blockDim.x) smem[q] = __ldg(bp.a[0].P.water + q);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t total = s_pre[n];
    for (;;) {
        unsigned int w = 0;
        if (lane == 0) w = atomicAdd(counter, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if ((int64_t)w >= total) break;
        int q = 0;
        while (q + 1 < n && s_pre[q + 1] <= (int64_t)w) ++q;
        const DoseArgs& a = bp.a[g.j[q]];
        const int64_t e0 = ((int64_t)w - s_pre[q]) * 32;   // w < s_pre[n]: inside plan q's units
        const int nb = a.P.n_beams;
        int b = 0;
        while (b + 1 < nb && __ldg(a.base + b + 1) <= e0) ++b;
        const int32_t vi = __ldg(a.items + e0 + lane);
        const float4* wt = SHARED_W ? smem : a.P.water;
        process_unit<kDose, 1, MERGED, LAT, PREC>(a, vi, e0, b, wt, nullptr, s_row[threadIdx.x >> 5], lane);
    }
}

template <int MINB, bool SHARED_W, bool MERGED, int LAT, int PREC>
cudaError_t batch_kernel(cudaStream_t s, const BatchParams& bp, const BatchGroup& g, const int64_t* d_prefix,
                         unsigned int* d_counter, int device, int w_n)
{
    auto kern = k_pairs_batch<MINB, SHARED_W, MERGED, LAT, PREC>;
    const size_t sm = (SHARED_W && !MERGED) ? 2 * sizeof(float4) * (size_t)w_n : 0;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, sm);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    kern<<<sms * (per_sm > 0 ? per_sm : 1), kThreads, sm, s>>>(bp, g, d_prefix, d_counter);
    return cudaGetLastError();
}

template <bool MERGED, int LAT, int PREC>
cudaError_t batch_group(cudaStream_t s, const BatchParams& bp, const BatchGroup& g, const int64_t* d_prefix,
                        unsigned int* d_counter, int device, int w_n, int variant, bool shared_water)
{
    if (variant == 0)
        return shared_water ? batch_kernel<4, true, MERGED, LAT, PREC>(s, bp, g, d_prefix, d_counter, device, w_n)
                            : batch_kernel<4, false, MERGED, LAT, PREC>(s, bp, g, d_prefix, d_counter, device, w_n);
    return shared_water ? batch_kernel<5, true, MERGED, LAT, PREC>(s, bp, g, d_prefix, d_counter, device, w_n)
                        : batch_kernel<5, false, MERGED, LAT, PREC>(s, bp, g, d_prefix, d_counter, device, w_n);
}

template <int LAT, int PREC>
cudaError_t batch_group_tables(bool merged, cudaStream_t s, const BatchParams& bp, const BatchGroup& g,
                               const int64_t* d_prefix, unsigned int* d_counter, int device, int w_n, int variant,
                               bool shared_water)
{
    return merged ? batch_group<true, LAT, PREC>(s, bp, g, d_prefix, d_counter, device, w_n, variant, shared_water)
                  : batch_group<false, LAT, PREC>(s, bp, g, d_prefix, d_counter, device, w_n, variant, shared_water);
}

// dose_j[v] = sum over plan j's beams of its partial doses (fixed beam order)
// for every voxel of every plan; vpre[j] = voxels of plans 0..j-1.
__global__ void __launch_bounds__(256) k_sum_batch(const DoseArgs* __restrict__ args, int n,
                                                   const int64_t* __restrict__ vpre)
{
    __shared__ int64_t s_v[kMaxBatch + 1];
    for (int q = threadIdx.x; q <= n; q += blockDim.x) s_v[q] = vpre[q];
    __syncthreads();
    const int64_t total = s_v[n];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n - 1;   // last j with s_v[j] <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_v[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        const DoseArgs& a = args[lo];
        const int64_t V = s_v[lo + 1] - s_v[lo];
        const int64_t v = e - s_v[lo];
        float sum = 0.f;
        for (int b = 0; b < a.P.n_beams; ++b) sum += __ldg(a.part + (size_t)b * V + v);
        a.dose[v] = sum;
    }
}

// dose[q][v] = sum over beams of the partial doses (fixed beam order).
__global__ void __launch_bounds__(256) k_sum_beams(const float* __restrict__ part, int n_beams, int nfs,
                                                   int nf, int64_t V, float* __restrict__ dose, int64_t ldd)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)nf * V;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / V);
        const int64_t v = e % V;
        float s = 0.f;
        for (int b = 0; b < n_beams; ++b) s += __ldg(part + ((size_t)b * nfs + q) * V + v);
        dose[(size_t)q * ldd + v] = s;
    }
}

// rowcount[v] = number of pairs of voxel v over all beams.
__global__ void __launch_bounds__(256) k_rowsum(const int32_t* __restrict__ bcount, int n_beams, int64_t V,
                                                int32_t* __restrict__ rowcount)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = 0;
        for (int b = 0; b < n_beams; ++b) s += __ldg(bcount + (size_t)b * V + v);
        rowcount[v] = s;
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
    a.items = p->d_items;
    a.base = p->d_base;
    a.work = p->d_work;
    a.bcount = p->d_bcount;
    return a;
}

size_t smem_bytes(const dc_plan* p, int mode)
{
    if (mode == kCount) return 0;
    if (mode == kGrad)   // water tables + gradient bins (always the general tables)
        return 2 * sizeof(float4) * p->coeffs.w_n + sizeof(float) * (4 * (size_t)p->coeffs.w_n + 4 * p->coeffs.f_n + 2);
    size_t s = p->merged ? 0 : 2 * sizeof(float4) * p->coeffs.w_n;
    if (mode == kFill) s += sizeof(int2) * kWarps * 32 * kRingLd;
    return s;
}

int grid_for(int64_t n)
{
    int64_t g = (n + 255) / 256;
    return (int)(g > 152 * 32 ? 152 * 32 : (g < 1 ? 1 : g));
}

// Persistent launch: as many CTAs as fit on the device at once.
template <int MODE, int NF, bool MERGED, int LAT, int PREC = 0>
cudaError_t run_variant(const dc_plan* p, const DoseArgs& a)
{
    const size_t sm = smem_bytes(p, MODE);
    auto kern = k_pairs<MODE, NF, MERGED, LAT, PREC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, sm);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p->d_work + 1, 0, sizeof(int32_t), p->stream);
    if (e != cudaSuccess) return e;
    kern<<<sms * (per_sm > 0 ? per_sm : 1), kThreads, sm, p->stream>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

// The tensor-core form of 64 fluence vectors (PREC 2) for the plan's lateral
// form and tables.
cudaError_t run_tc(const dc_plan* p, const DoseArgs& a)
{
    const bool item = p->coeffs.density_correction && p->lateral_mode != DC_LATERAL_ISO;
    if (p->merged)
        return item ? run_variant<kDose, 64, true, kItem, 2>(p, a) : run_variant<kDose, 64, true, kIso, 2>(p, a);
    return item ? run_variant<kDose, 64, false, kItem, 2>(p, a) : run_variant<kDose, 64, false, kIso, 2>(p, a);
}

// The fluences of the tensor-core form: fpack[i][n] = BF16(F[n][i]) (round to
// nearest even), zero for n >= nf.
__global__ void __launch_bounds__(256) k_pack_fluence_bf16(const float* __restrict__ F, int nf, int ldf, int B,
                                                           __nv_bfloat16* __restrict__ fpack)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * 64;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(e / B), i = (int)(e % B);
        fpack[(size_t)i * 64 + n] = __float2bfloat16_rn(n < nf ? __ldg(F + (size_t)n * ldf + i) : 0.f);
    }
}

template <int MODE, int NF>
cudaError_t run(const dc_plan* p, const DoseArgs& a)
{
    if (MODE == kCount) return run_variant<kCount, 1, false, kIso>(p, a);
    // per-item factors exist for the axis and network forms with the density correction on
    const bool item = p->coeffs.density_correction && p->lateral_mode != DC_LATERAL_ISO;
    if (MODE == kDose && NF == 1 && p->precision == DC_PRECISION_BF16) {
        if (p->merged)
            return item ? run_variant<kDose, 1, true, kItem, 1>(p, a) : run_variant<kDose, 1, true, kIso, 1>(p, a);
        return item ? run_variant<kDose, 1, false, kItem, 1>(p, a) : run_variant<kDose, 1, false, kIso, 1>(p, a);
    }
    if (p->merged) return item ? run_variant<MODE, NF, true, kItem>(p, a) : run_variant<MODE, NF, true, kIso>(p, a);
    return item ? run_variant<MODE, NF, false, kItem>(p, a) : run_variant<MODE, NF, false, kIso>(p, a);
}

}  // namespace

DoseArgs dose_args(const dc_plan* p, const float* fluence, float* dose)
{
    DoseArgs a = make_args(p);
    a.fluence = fluence;
    a.nf = 1;
    a.ldf = p->B;
    a.dose = dose;
    a.ldd = p->V;
    a.part = p->d_part;
    return a;
}

int batch_max_plans() { return kMaxBatch; }
int batch_groups() { return kBatchGroups; }

cudaError_t launch_batch(cudaStream_t s, const DoseArgs* h_args, const DoseArgs* d_args, int n,
                         const int64_t* d_vpre, int64_t v_total, int64_t* d_prefix, unsigned int* d_counter,
                         int device, int variant, bool shared_water)
{
    if (n < 1 || n > kMaxBatch || variant < 0 || variant >= kBatchVariants) return cudaErrorInvalidValue;
    static BatchParams bp;   // 24 KiB: kept off the stack; the launch copies it
    static std::mutex bp_mu;
    std::lock_guard<std::mutex> lock(bp_mu);
    memset(&bp, 0, sizeof(bp));
    memcpy(bp.a, h_args, sizeof(DoseArgs) * n);
    const int w_n = h_args[0].P.w_n;
    for (int gi = 0; gi < kBatchGroups; ++gi) {
        const bool item = (gi & 1) != 0;
        const int prec = gi >> 1;
        BatchGroup g{};
        bool merged = true;
        for (int j = 0; j < n; ++j)
            if ((h_args[j].P.item_rt != 0) == item && h_args[j].P.prec_rt == prec) {
                g.j[g.n++] = (int8_t)j;
                merged = merged && h_args[j].P.merged_rt != 0;
            }
        if (g.n == 0) continue;
        int64_t* pre = d_prefix + (size_t)gi * (n + 1);
        unsigned int* cnt = d_counter + gi;
        k_batch_prefix<<<1, 32, 0, s>>>(d_args, g, pre, cnt);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (prec == 0)
            e = item ? batch_group_tables<kItem, 0>(merged, s, bp, g, pre, cnt, device, w_n, variant, shared_water)
                     : batch_group_tables<kIso, 0>(merged, s, bp, g, pre, cnt, device, w_n, variant, shared_water);
        else
            e = item ? batch_group_tables<kItem, 1>(merged, s, bp, g, pre, cnt, device, w_n, variant, shared_water)
                     : batch_group_tables<kIso, 1>(merged, s, bp, g, pre, cnt, device, w_n, variant, shared_water);
        if (e != cudaSuccess) return e;
        count_launches(2);
    }
    k_sum_batch<<<grid_for(v_total), 256, 0, s>>>(d_args, n, d_vpre);
    count_launches(1);
    return cudaGetLastError();
}

// One pass evaluates each pair once for all of its fluence vectors: on the
// 16 head-and-neck plans' largest grid, 64 vectors took 145 ms as four passes
// of 16 and 80 ms as one pass of 64 (the same doses bit for bit).
int dose_pass_width(int nf)
{
    return nf <= 1 ? 1 : (nf <= 16 ? 16 : (nf <= 32 ? 32 : 64));
}

cudaError_t launch_dose(const dc_plan* p, const float* fluence, int nf, int ldf, float* dose,
                        int64_t ldd, bool record_counts)
{
    DoseArgs a = make_args(p);
    a.ldf = ldf;
    a.part = p->d_part;
    if (nf > 1 && p->precision == DC_PRECISION_BF16) {
        // the reduced-precision form of several vectors: the pair values and
        // fluences rounded to BF16 and applied on the tensor cores, one pass
        if (nf > 64 || p->part_cap < (size_t)p->n_beams * 64 * p->V || p->sp_fp_cap < (size_t)p->B * 64)
            return cudaErrorInvalidValue;
        k_pack_fluence_bf16<<<grid_for((int64_t)p->B * 64), 256, 0, p->stream>>>(
            fluence, nf, ldf, p->B, static_cast<__nv_bfloat16*>(p->d_sp_fp));
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        a.fluence = fluence;
        a.nf = nf;
        a.fpack = static_cast<const uint4*>(p->d_sp_fp);
        e = cudaMemsetAsync(p->d_part, 0, sizeof(float) * (size_t)p->n_beams * 64 * p->V, p->stream);
        if (e != cudaSuccess) return e;
        e = run_tc(p, a);
        if (e != cudaSuccess) return e;
        k_sum_beams<<<grid_for((int64_t)nf * p->V), 256, 0, p->stream>>>(p->d_part, p->n_beams, 64, nf, p->V, dose,
                                                                        ldd);
        count_launches(1);
        return cudaGetLastError();
    }
    if (record_counts && nf == 1) {
        cudaError_t e = cudaMemsetAsync(p->d_bcount, 0, sizeof(int32_t) * (size_t)p->n_beams * p->V, p->stream);
        if (e != cudaSuccess) return e;
        a.count_out = p->d_bcount;
    }
    const int width = dose_pass_width(nf);
    for (int q0 = 0; q0 < nf; q0 += width) {
        a.fluence = fluence + (size_t)q0 * ldf;
        a.nf = nf - q0 < width ? nf - q0 : width;
        const int nfs = a.nf == 1 ? 1 : width;
        if (p->part_cap < (size_t)p->n_beams * nfs * p->V) return cudaErrorInvalidValue;
        cudaError_t e = cudaMemsetAsync(p->d_part, 0, sizeof(float) * (size_t)p->n_beams * nfs * p->V, p->stream);
        if (e != cudaSuccess) return e;
        e = nfs == 1 ? run<kDose, 1>(p, a)
                     : (nfs == 16 ? run<kDose, 16>(p, a) : (nfs == 32 ? run<kDose, 32>(p, a) : run<kDose, 64>(p, a)));
        if (e != cudaSuccess) return e;
        k_sum_beams<<<grid_for((int64_t)a.nf * p->V), 256, 0, p->stream>>>(p->d_part, p->n_beams, nfs, a.nf, p->V,
                                                                          dose + (size_t)q0 * ldd, ldd);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_count(const dc_plan* p, int32_t* counts)
{
    DoseArgs a = make_args(p);
    cudaError_t e = cudaMemsetAsync(p->d_bcount, 0, sizeof(int32_t) * (size_t)p->n_beams * p->V, p->stream);
    if (e != cudaSuccess) return e;
    {
        auto kern = k_count_units<kCountVoxels>;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
        if (e == cudaSuccess) e = cudaMemsetAsync(p->d_work + 1, 0, sizeof(int32_t), p->stream);
        if (e != cudaSuccess) return e;
        kern<<<sms * (per_sm > 0 ? per_sm : 1), kThreads, 0, p->stream>>>(a);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    k_rowsum<<<grid_for(p->V), 256, 0, p->stream>>>(p->d_bcount, p->n_beams, p->V, counts);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rowsum(const dc_plan* p, int32_t* counts)
{
    k_rowsum<<<grid_for(p->V), 256, 0, p->stream>>>(p->d_bcount, p->n_beams, p->V, counts);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fill(const dc_plan* p, const int64_t* rowptr, int32_t* cols, void* vals,
                        int value_dtype, const float* fluence, float* dose)
{
    DoseArgs a = make_args(p);
    a.rowptr = rowptr;
    a.cols = cols;
    a.vals = vals;
    a.value_dtype = value_dtype;
    if (!fluence) return run<kFill, 0>(p, a);
    // the matrix and eq. (1) from one evaluation of each pair: per-beam
    // partial doses as in launch_dose, summed in beam order
    if (p->part_cap < (size_t)p->n_beams * p->V) return cudaErrorInvalidValue;
    a.fluence = fluence;
    a.nf = 1;
    a.ldf = p->B;
    a.part = p->d_part;
    cudaError_t e = cudaMemsetAsync(p->d_part, 0, sizeof(float) * (size_t)p->n_beams * p->V, p->stream);
    if (e != cudaSuccess) return e;
    e = run<kFill, 1>(p, a);
    if (e != cudaSuccess) return e;
    k_sum_beams<<<grid_for((int64_t)p->V), 256, 0, p->stream>>>(p->d_part, p->n_beams, 1, 1, p->V, dose, p->V);
    count_launches(1);
    return cudaGetLastError();
}

template <typename K>
static cudaError_t launch_persistent(const dc_plan* p, K kern, size_t sm, const DoseArgs& a, const PatchTiles& t)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, sm);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p->d_work + 1, 0, sizeof(int32_t), p->stream);
    if (e != cudaSuccess) return e;
    kern<<<sms * (per_sm > 0 ? per_sm : 1), kThreads, sm, p->stream>>>(a, t);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mark_patches(const dc_plan* p, const PatchTiles& t)
{
    return launch_persistent(p, k_mark_patches, 0, make_args(p), t);
}

cudaError_t launch_tile_fill(const dc_plan* p, const PatchTiles& t)
{
    const DoseArgs a = make_args(p);
    const bool item = p->coeffs.density_correction && p->lateral_mode != DC_LATERAL_ISO;
    const size_t sm = p->merged ? 0 : 2 * sizeof(float4) * p->coeffs.w_n;
    if (p->merged)
        return item ? launch_persistent(p, k_tile_fill<true, kItem>, sm, a, t)
                    : launch_persistent(p, k_tile_fill<true, kIso>, sm, a, t);
    return item ? launch_persistent(p, k_tile_fill<false, kItem>, sm, a, t)
                : launch_persistent(p, k_tile_fill<false, kIso>, sm, a, t);
}

cudaError_t launch_dose_vjp(const dc_plan* p, const float* fluence, const float* wv, float* g_water, float* g_dens,
                            float* g_corr)
{
    if (smem_bytes(p, kGrad) > 200 * 1024) return cudaErrorInvalidValue;
    DoseArgs a = make_args(p);
    a.fluence = fluence;
    a.nf = 1;
    a.ldf = p->B;
    a.wv = wv;
    a.g_water = g_water;
    a.g_dens = g_dens;
    a.g_corr = g_corr;
    cudaError_t e = cudaMemsetAsync(g_water, 0, sizeof(float) * 4 * (size_t)p->coeffs.w_n, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_dens, 0, sizeof(float) * 4 * (size_t)p->coeffs.f_n, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g_corr, 0, sizeof(float) * 2, p->stream);
    if (e != cudaSuccess) return e;
    return run_variant<kGrad, 1, false, kIso>(p, a);
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
