// Device-side records and the kernel-side view of a plan: the structures the
// pair kernels read.  Host-only plan state lives in dc_internal.cuh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dc {

// Per-beam record written by the geometry kernel (FP32 copy of FP64 values).
struct BeamDev {
    float src[3];
    float sad;
    float ez[3];          // beam central axis (source -> isocentre)
    float inv_cos_max;    // 1 / cos(largest beamlet angle of the field)
    float ex[3];          // field axis e_x'
    float half_fx;
    float ey[3];          // field axis e_y'
    float half_fy;
    int M, N, first, pad;
};

// Per-beamlet record (64 bytes, four 16-byte vectors).
struct BeamletDev {
    float4 n_lin;     // unit direction n, L_in (source to body entry along the axis)
    float4 exy_xy;    // (e_x''.x, e_y''.x, e_x''.y, e_y''.y): the lateral axes interleaved, so that
                      // (x', y') = v . (e_x'', e_y'') runs as packed FP32 pairs
    float4 exy_z;     // (e_x''.z, e_y''.z, L_out (-1 if the axis misses the body),
                      //  weight of the theta row l+1 in A)
    int4 meta;        // K (table samples), l (theta row of A), hit (0/1), beam
};

// Beam's-eye-view binning grid of one beam (see k_bin.cu): tiles of `tile` cm
// in the isocentre plane starting at (a0, c0), depth slabs of `slab` cm
// starting at zz0; cell = (tc * nta + ta) * nzs + slab index.
struct BinGeom {
    float a0, c0, tile, zz0, slab, rw_max;
    int nta, ntc, nzs, cells;
};

constexpr int kMaxBeams = 64;

// Kernel-side view of a plan.
//
// Table layouts (value + slope to the next sample, so one load and one fma
// give a linear interpolation, and a sample index never needs a clamp):
//   tab   [B][Kmax][2] float4: (t_eq, dt_eq, W1, dW1), (W2, dW2, 0, 0) at t = k d
//   arow  [B][a_nt]    float2: (A_i, dA_i) at t_eq = j a_dt, where A_i is A
//                      already interpolated at the beamlet's theta (the bilinear
//                      lookup of A factors into theta then t_eq)
//   water [w_n][2]     float4: (u1w, du1w, u2w, du2w), (w1w, dw1w, w2w, dw2w)
struct PlanView {
    int nx, ny, nz, n_beams, B, Kmax;
    float dx, dy, dz, ox, oy, oz;
    float d, inv_d;
    float R2, roi;
    float x0, y0, bx, by;
    float wscale;                 // 1 with the density correction, 0 without
    int a_nt; float inv_adt;
    const float2* arow;
    const float4* water; int w_n; float inv_wdt;
    // per-voxel factors f_u1(rho), f_u2(rho_hat), f_w1(rho_hat), f_w2(rho_hat)
    const float4* fac;
    const BeamDev* beams;
    const BeamletDev* bl;
    const float4* tab;
    // when the water tables' step equals d: [B][Kmax][3] float4
    //   (t_eq, dt_eq, O1, O2), (dO1, dO2, u1w, u2w), (du1w, du2w, 0, 0)
    // with O_i = omega_i^w + omega_i^corr (times 0 without density correction)
    const float4* tabm;
    // per-(voxel, beam) lateral factors for every voxel-list entry (axis and
    // network forms): (log2 e f_u2 along x, along y, f_w1, f_w2)
    const float4* lfac;
    // density and density-function tables for the lateral stencils
    const float* rho;
    const float* rhos;            // smoothed density (backward pass)
    const float* dens;
    int f_n;
    float f_rho0, inv_drho;
    float idx, idy, idz;          // 1 / voxel size
    float gw[16];                 // normalised Gaussian weights of the 16 stencil taps
    int merged_rt;                // tabm is in use (runtime copy of the plan's choice)
    int item_rt;                  // lfac is in use
    int prec_rt;                  // direct-dose arithmetic (DC_PRECISION_*)
    float a_hi, w_hi;             // a_nt - 1, w_n - 1 as floats (clamps of the table coordinates)
    int32_t* chk;                 // status word of the DC_BOUNDS_CHECK build (first violated guard)
};

// DC_BOUNDS_CHECK builds: every index the pair kernels use to read a table,
// a beamlet record, a voxel list or the fluence is checked against its
// extent; a violation records the guard's code in the plan's status word
// (first one wins) and reads element 0 instead.  Other builds: no check.
#if DC_BOUNDS_CHECK
__device__ __forceinline__ uint32_t dc_guard(int32_t* chk, uint32_t idx, uint32_t n, int code)
{
    if (idx < n) return idx;
    atomicCAS(chk, 0, code);
    return 0u;
}
#define DC_GUARD(P, idx, n, code) dc::dc_guard((P).chk, (uint32_t)(idx), (uint32_t)(n), (code))
#else
#define DC_GUARD(P, idx, n, code) (idx)
#endif

// Arguments of the pair kernels (k_dose.cu) for one plan.
struct DoseArgs {
    PlanView P;
    const float* fluence;   // [nf][ldf]
    int nf, ldf;
    float* dose;            // [nf][ldd]
    int64_t ldd;
    float* part;            // dose: per-beam partial dose [n_beams][NF][V]
    const uint4* fpack;     // dose, tensor-core form: the fluences as BF16 [B][64] (zero past nf)
    int32_t* bcount;        // count: per-beam pair counts [n_beams][V]; fill reads them
    int32_t* count_out;     // dose with one fluence vector: where to record the same counts (or null)
    const int64_t* rowptr;  // fill
    int32_t* cols;
    void* vals;
    int value_dtype;
    const int32_t* items;   // beam voxel lists (k_bin.cu)
    const int64_t* base;    // [n_beams + 1]
    int32_t* work;          // [0] work units, [1] counter
    // backward pass with respect to the commissioning tables: voxel weights
    // [V] and the gradients [4][w_n], [4][f_n], [2]
    const float* wv;
    float* g_water;
    float* g_dens;
    float* g_corr;
};

}  // namespace dc
