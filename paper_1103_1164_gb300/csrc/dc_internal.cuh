// Internal declarations shared by the CUDA translation units of the DC-FSPB
// engine (not part of the ABI; see include/dc_fspb.h for the public calls).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dc_fspb.h"
#include "dc_views.cuh"

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
    int precision = DC_PRECISION_FP32;   // arithmetic of the direct dose (dc_fspb_set_precision)
    float4* d_lfac = nullptr;        // [n_beams][V + 32]
    float* d_leaf = nullptr;         // leaf sequences of dc_fluence_from_leaves (packed)
    size_t leaf_cap = 0;             // floats allocated at d_leaf
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
    uint32_t* d_sp_marks = nullptr;  // preparation: the occupied patches of each row-block (bitmaps)
    uint16_t* d_sp_wpre = nullptr;   // preparation: chunks before each bitmap word
    int64_t sp_n_zero = 0;
    void* d_sp_fp = nullptr;
    size_t sp_fp_cap = 0;
    float* d_sp_p = nullptr;
    size_t sp_p_cap = 0;
    int32_t* d_err = nullptr;        // device status word of bounded waits
    int32_t* d_chk = nullptr;        // status word of the DC_BOUNDS_CHECK build
    float* d_grad = nullptr;         // dc_fspb_dose_vjp with host buffers: the gradients on the device
    // bytes held by each block-sparse buffer: a new preparation reuses a
    // buffer that is large enough (re-allocating tens of GB per density costs
    // more than building the tiles)
    size_t sp_cap[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    // The tiles no longer describe the plan (new voxel lists, lateral form or
    // tables): dc_fspb_spmm needs a new dc_fspb_spmm_prepare.  The buffers stay.
    void spmm_invalidate()
    {
        sp_ready = false;
        sp_n_rb = 0;
        sp_chunks = 0;
        sp_n_zero = 0;
    }
    // Frees the block-sparse buffers.
    void spmm_free()
    {
        void* bufs[] = {d_sp_rbfirst, d_sp_first, d_sp_nchunk, d_sp_off, d_sp_kb, d_sp_tiles, d_sp_inv, d_sp_zero,
                        d_sp_marks, d_sp_wpre};
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
        d_sp_marks = nullptr;
        d_sp_wpre = nullptr;
        for (size_t& c : sp_cap) c = 0;
        spmm_invalidate();
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

// An NVTX range around each C-ABI call, named after the call: a profiler's
// timeline then groups the kernels by the call that launched them (NVTX costs
// a pointer test when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define DC_NVTX(name) dc::NvtxRange dc_nvtx_range_(name)

// Every device allocation of the library goes through dev_malloc.  Test hook
// of the out-of-memory paths: with DC_FSPB_FAIL_ALLOC_AT=N in the environment,
// the N-th allocation counted since the variable last changed value fails
// with cudaErrorMemoryAllocation (nothing is allocated).
cudaError_t dev_malloc_bytes(void** p, size_t bytes);
template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes)
{
    return dev_malloc_bytes(reinterpret_cast<void**>(p), bytes);
}

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
// fluence vectors that one pass of launch_dose takes for nf vectors (1, 16,
// 32 or 64); the per-beam partial doses hold n_beams * width * V floats
int dose_pass_width(int nf);
cudaError_t launch_count(const dc_plan* p, int32_t* counts);
// rowcount[v] = sum over beams of the per-beam pair counts already in d_bcount
cudaError_t launch_rowsum(const dc_plan* p, int32_t* counts);
// with a fluence (device), the same pass also accumulates eq. (1) into dose [V]
cudaError_t launch_fill(const dc_plan* p, const int64_t* rowptr, int32_t* cols, void* vals,
                        int value_dtype, const float* fluence = nullptr, float* dose = nullptr);
cudaError_t launch_scan_counts(const dc_plan* p, const int32_t* counts, int64_t* rowptr,
                               int64_t* total_dev);
// The SpMM's block-sparse BF16 matrix straight from the pair evaluation
// (k_dose.cu; the layout is k_spmm.cu's).  Row-block r of beam b holds its
// list entries 128 r .. 128 r + 127; its chunks are the 4 x 4 beamlet patches
// (16 tile columns) in which any of its pairs lies, in patch order.
struct PatchTiles {
    uint32_t* marks;            // [n_rb][words] patch bitmaps of each row-block
    const uint16_t* wprefix;    // [n_rb][words] chunks of the row-block before each bitmap word
    const int32_t* rb_first;    // [n_beams + 1] first row-block of each beam
    const int64_t* chunk_off;   // [n_rb + 1] first chunk of each row-block
    uint16_t* tiles;            // [chunks][128 x 16] BF16, zero where no pair
    int words;
};
// sets the bit of every patch that holds a pair of the row-block (marks zeroed by the caller)
cudaError_t launch_mark_patches(const dc_plan* p, const PatchTiles& t);
// writes every pair's BF16 value into its tile (tiles zeroed by the caller)
cudaError_t launch_tile_fill(const dc_plan* p, const PatchTiles& t);
// backward pass of eq. (1) with respect to the commissioning tables (device
// buffers; the gradients are cleared first)
cudaError_t launch_dose_vjp(const dc_plan* p, const float* fluence, const float* wv, float* g_water, float* g_dens,
                            float* g_corr);
// lateral factors, stencil samples and the surrogate network (k_lateral.cu)
cudaError_t launch_lateral(const dc_plan* p);
cudaError_t launch_stencils(const dc_plan* p, const int32_t* vox, const int32_t* beam, int n, float* X, float* T);
cudaError_t launch_mlp_predict_bf16(cudaStream_t s, const float* X, int n, const uint2* wfrag, const float* bias,
                                    float* Y);
cudaError_t launch_mlp_grad(cudaStream_t s, int nctas, const float* theta, const float* X, const float* T, int n,
                            float* partial, float* loss_part);
// the same gradient with BF16 tensor-core products (k_mlp_bf16.cu)
cudaError_t launch_mlp_grad_bf16(cudaStream_t s, int nctas, const float* theta, const float* X, const float* T, int n,
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
constexpr int kBatchPerPlan = 2;    // batch variant: the plans' own dose launches, one after another
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
dc_status spmm_prepare(dc_plan* p);
cudaError_t spmm_run(dc_plan* p, const float* F, int k, float* Y);
cudaError_t spmm_run_static(dc_plan* p, const float* F, int k, float* Y);   // scratch in static device memory

}  // namespace dc
