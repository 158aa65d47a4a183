// Internal declarations shared by the CUDA translation units of the DC-FSPB
// engine (not part of the ABI; see include/dc_fspb.h for the public calls).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dc_fspb.h"

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
    //   (t_eq, dt_eq, O1, dO1), (O2, dO2, u1w, du1w), (u2w, du2w, 0, 0)
    // with O_i = omega_i^w + omega_i^corr (times 0 without density correction)
    const float4* tabm;
    // per-(voxel, beam) lateral factors for every voxel-list entry (axis and
    // network forms): (log2 e f_u2 along x, along y, f_w1, f_w2)
    const float4* lfac;
    // density and density-function tables for the lateral stencils
    const float* rho;
    const float* dens;
    int f_n;
    float f_rho0, inv_drho;
    float idx, idy, idz;          // 1 / voxel size
    float gw[16];                 // normalised Gaussian weights of the 16 stencil taps
    int merged_rt;                // tabm is in use (runtime copy of the plan's choice)
    int item_rt;                  // lfac is in use
    float a_hi, w_hi;             // a_nt - 1, w_n - 1 as floats (clamps of the table coordinates)
};

// Arguments of the pair kernels (k_dose.cu) for one plan.
struct DoseArgs {
    PlanView P;
    const float* fluence;   // [nf][ldf]
    int nf, ldf;
    float* dose;            // [nf][ldd]
    int64_t ldd;
    float* part;            // dose: per-beam partial dose [n_beams][NF][V]
    int32_t* bcount;        // count: per-beam pair counts [n_beams][V]; fill reads them
    int32_t* count_out;     // dose with one fluence vector: where to record the same counts (or null)
    const int64_t* rowptr;  // fill
    int32_t* cols;
    void* vals;
    int value_dtype;
    const int32_t* items;   // beam voxel lists (k_bin.cu)
    const int64_t* base;    // [n_beams + 1]
    int32_t* work;          // [0] work units, [1] counter
};

}  // namespace dc

struct dc_plan {
    int device = 0;
    cudaStream_t stream = nullptr;
    dc_grid grid{};
    int64_t V = 0;
    int B = 0, n_beams = 0, Kmax = 0;
    float bx = 0, by = 0, d = 0;
    dc_kernel_coeffs coeffs{};
    std::vector<dc_beam> beams;
    std::vector<int> M, N, first;

    // device memory owned by the plan
    float* d_rho = nullptr;
    float* d_rhos = nullptr;
    float* d_tmp = nullptr;
    float4* d_fac = nullptr;
    dc::BeamDev* d_beams = nullptr;
    dc::BeamletDev* d_bl = nullptr;
    float* d_theta = nullptr;
    double* d_ray = nullptr;         // [B][8]: FP64 source (3) and direction (3) of each beamlet axis
    float2* d_lio = nullptr;         // [B]: (L_in, L_out) of each axis, L_out < 0 if it misses the body
    float4* d_tab = nullptr;
    float2* d_arow = nullptr;
    float4* d_tabm = nullptr;        // merged depth + water tables (only when w_dt == d)
    bool merged = false;
    // lateral form of step 11 (DC_LATERAL_*) and its per-entry factors
    int lateral_mode = 0;
    float4* d_lfac = nullptr;        // [n_beams][V + 32]
    uint2* d_mlp_frag = nullptr;     // BF16 B fragments of the surrogate network
    float* d_mlp_bias = nullptr;
    float mlp_lo = 0.f, mlp_hi = 0.f;
    bool mlp_ready = false;
    int32_t* d_nfall = nullptr;      // entries that fell back to the plain stencil
    float gw[16] = {0};
    float* d_A = nullptr;
    float4* d_water = nullptr;
    float* d_dens = nullptr;
    dc_beam* d_beamin = nullptr;
    // staging for calls with host pointers
    float* d_fluence = nullptr;
    size_t fluence_cap = 0;
    float* d_dose = nullptr;
    size_t dose_cap = 0;
    // beam's-eye-view binning: per beam a list of voxels grouped by cell
    std::vector<dc::BinGeom> bin_host;
    dc::BinGeom* d_bin = nullptr;
    int tiles_max = 0, cells_max = 0;   // of the current binning
    int tiles_cap = 0, cells_cap = 0;   // allocated for
    float bin_tile = 0.f, bin_slab = 0.f;
    float2* d_bounds = nullptr;      // [n_beams][tiles_max] (min L_in, max L_out)
    int32_t* d_cellof = nullptr;     // [n_beams][V]
    int32_t* d_hist = nullptr;       // [n_beams][cells_max]
    int32_t* d_nitems = nullptr;     // [n_beams]
    int32_t* d_bstart = nullptr;     // [n_beams + 1] start of each beam's cells in the device-wide cell scan
    int32_t* d_bscan = nullptr;      // chunk sums of that scan
    int64_t* d_base = nullptr;       // [n_beams + 1] start of each beam's list (whole warps)
    int32_t* d_work = nullptr;       // [0] warp work units, [1] work counter
    int32_t* d_items = nullptr;      // [n_beams][V + 32]
    float* d_part = nullptr;         // per-beam partial dose [n_beams][nf][V]
    size_t part_cap = 0;
    int32_t* d_bcount = nullptr;     // per-beam pair counts [n_beams][V]
    int persist_ctas[4] = {0, 0, 0, 0};
    // bumped whenever a buffer or a launch parameter that a captured batch
    // graph holds changes (binning geometry, partial-dose buffer, lateral form)
    uint64_t layout_gen = 0;
    // block-sparse BF16 dose-deposition matrix for the tensor-core SpMM (k_spmm.cu)
    bool sp_ready = false;
    int sp_n_rb = 0;
    int64_t sp_chunks = 0, sp_items_total = 0;
    int32_t* d_sp_rbfirst = nullptr;
    int4* d_sp_first = nullptr;      // per beam (first beamlet, M, N, first tile column), [n_beams + 1]
    int sp_cols = 0;                 // tile columns of all beams (4 x 4 beamlet patches)
    int32_t* d_sp_nchunk = nullptr;
    int64_t* d_sp_off = nullptr;
    int32_t* d_sp_kb = nullptr;
    void* d_sp_tiles = nullptr;
    int32_t* d_sp_inv = nullptr;
    int32_t* d_sp_zero = nullptr;    // one-beam plans: voxels in no list (their output rows are zero)
    int64_t sp_n_zero = 0;
    void* d_sp_fp = nullptr;
    size_t sp_fp_cap = 0;
    float* d_sp_p = nullptr;
    size_t sp_p_cap = 0;
    int32_t* d_err = nullptr;        // device status word of bounded waits
    void spmm_free()
    {
        void* bufs[] = {d_sp_rbfirst, d_sp_first, d_sp_nchunk, d_sp_off, d_sp_kb, d_sp_tiles, d_sp_inv, d_sp_zero};
        for (void* b : bufs)
            if (b) cudaFree(b);
        d_sp_rbfirst = d_sp_nchunk = nullptr;
        d_sp_first = nullptr;
        sp_cols = 0;
        d_sp_off = nullptr;
        d_sp_kb = nullptr;
        d_sp_tiles = nullptr;
        d_sp_inv = nullptr;
        d_sp_zero = nullptr;
        sp_n_zero = 0;
        sp_ready = false;
        sp_n_rb = 0;
        sp_chunks = 0;
    }
    // dose-deposition matrix pattern
    int32_t* d_rowcount = nullptr;
    int64_t* d_rowptr = nullptr;
    int64_t pairs = -1;
    bool counts_fresh = false;       // d_bcount holds the pair counts of the current voxel lists
    void* d_scan_tmp = nullptr;
    // device staging of the matrix for calls with host buffers
    int32_t* d_mcols = nullptr;
    void* d_mvals = nullptr;
    size_t mstage_bytes = 0;
    size_t scan_tmp_bytes = 0;

    dc::PlanView view() const;
};

namespace dc {

// number of kernels launched by the library (dc_fspb_launch_count)
void count_launches(int n);

// error plumbing -------------------------------------------------------------
void set_error(const std::string& msg);
dc_status cuda_fail(cudaError_t e, const char* what);

#define DC_CUDA(call)                                                       \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return dc::cuda_fail(e_, #call);             \
    } while (0)

// kernel launchers (defined in the kernel translation units) ------------------
cudaError_t launch_smooth(const dc_plan* p, float sigma);
cudaError_t launch_factors(const dc_plan* p);
cudaError_t launch_beamlets(const dc_plan* p);   // also builds the theta-blended A rows
cudaError_t launch_binning(const dc_plan* p);
// record_counts (one fluence vector only): the pass also writes the per-beam
// pair counts that launch_count would (the matrix pattern then needs no
// second traversal; see launch_rowsum)
cudaError_t launch_dose(const dc_plan* p, const float* fluence, int nf, int ldf, float* dose,
                        int64_t ldd, bool record_counts = false);
cudaError_t launch_count(const dc_plan* p, int32_t* counts);
// rowcount[v] = sum over beams of the per-beam pair counts already in d_bcount
cudaError_t launch_rowsum(const dc_plan* p, int32_t* counts);
cudaError_t launch_fill(const dc_plan* p, const int64_t* rowptr, int32_t* cols, void* vals,
                        int value_dtype);
cudaError_t launch_scan_counts(const dc_plan* p, const int32_t* counts, int64_t* rowptr,
                               int64_t* total_dev);
// lateral factors, stencil samples and the surrogate network (k_lateral.cu)
cudaError_t launch_lateral(const dc_plan* p);
cudaError_t launch_stencils(const dc_plan* p, const int32_t* vox, const int32_t* beam, int n, float* X, float* T);
cudaError_t launch_mlp_predict_bf16(cudaStream_t s, const float* X, int n, const uint2* wfrag, const float* bias,
                                    float* Y);
cudaError_t launch_mlp_grad(cudaStream_t s, int nctas, const float* theta, const float* X, const float* T, int n,
                            float* partial, float* loss_part);
cudaError_t launch_mlp_adam(cudaStream_t s, const float* partial, int nparts, float* theta, float* m1, float* m2,
                            float* grad, float lr, float b1, float b2, float eps, int step);
constexpr int kMlpParams = 7491;
constexpr int kMlpFragU2 = (3 * 8 + 4 * 8 + 4) * 32;
constexpr int kMlpBias = 64 + 64 + 3;
void mlp_pack(const float* theta, std::vector<uint2>& frag, std::vector<float>& bias);
// multi-plan batch (k_dose.cu)
// arguments of one plan for one fluence vector (partials in the plan's d_part)
DoseArgs dose_args(const dc_plan* p, const float* fluence, float* dose);
int batch_max_plans();
constexpr int kBatchVariants = 2;   // register budgets of the batch pair kernel (4 or 5 CTAs per SM)
// The plans are grouped by lateral form (at most batch_groups() groups); per
// group, the prefix of its plans' unit counts and one persistent pair kernel
// over all their units (one launch in all when the plans share the lateral
// form, the usual case); then the per-plan beam sums.  Arguments
// h_args by value, d_args the same records on the device; d_prefix holds
// batch_groups() x (n + 1) entries and d_counter batch_groups(); the partials
// must be zero beforehand.
int batch_groups();
cudaError_t launch_batch(cudaStream_t s, const DoseArgs* h_args, const DoseArgs* d_args, int n,
                         const int64_t* d_vpre, int64_t v_total, int64_t* d_prefix, unsigned int* d_counter,
                         int device, int variant, bool shared_water);
// block-sparse tensor-core SpMM (k_spmm.cu)
dc_status spmm_prepare(dc_plan* p, const int64_t* rowptr, const int32_t* cols, const uint16_t* vals);
cudaError_t spmm_run(dc_plan* p, const float* F, int k, float* Y);
cudaError_t spmm_run_static(dc_plan* p, const float* F, int k, float* Y);   // scratch in static device memory

}  // namespace dc
