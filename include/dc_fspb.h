/*
 * dc_fspb.h - C ABI of the GB300 DC-FSPB dose engine.
 *
 * The engine computes the density-corrected finite-size pencil-beam dose of
 * Gu, Jelen, Li, Jia and Jiang, "GPU-based finite-size pencil beam algorithm
 * with 3D-density correction for radiotherapy dose calculation"
 * (arXiv 1103.1164):
 *
 *   D(r)   = sum_i D_i(r) f_i                                         (eq. 1)
 *   D_i(r) = F(x, y, omega, u_x, u_y, x0, y0) A(t_eq, theta) (SAD/|r_a|)^2 (eq. 2)
 *   F      = sum_{i=1,2} omega_i p(x, u_ix, x0) p(y, u_iy, y0)          (eq. 3)
 *   p      = the piecewise sinh/cosh/exp penumbra profile               (eq. 4)
 *
 * with the lateral density correction of Section 2.1 (u_1 = f_u1(rho) u_1^w,
 * u_2 = f_u2(rho_hat) u_2^w, omega_i = f_omega_i(rho_hat)(omega_i^w +
 * omega_i^corr)) and the per-beamlet radiological-depth and omega_corr tables
 * of Algorithm A1 steps 5-6 / Algorithm A2 Kernel 4.  All compute runs in the
 * library's own CUDA kernels for sm_103a on one GPU.
 *
 * Conventions (all entry points):
 *  - lengths in cm, angles in degrees at the ABI (radians inside);
 *  - volumes are float32 [nz][ny][nx], x fastest; voxel (i, j, k) has its
 *    centre at (ox + i dx, oy + j dy, oz + k dz); voxel v = (k ny + j) nx + i;
 *  - beam frame: at gantry 0 the beam travels +y with field axes e_x' = +x,
 *    e_y' = +z; the gantry turns it about +z, the couch about +y, the
 *    collimator turns e_x', e_y' about the beam axis; source = iso - SAD e_z';
 *  - beamlets are numbered beam-major, then row (e_y' index n), then column
 *    (e_x' index m): i = first(b) + n M_b + m, M_b = field_x / beamlet_x;
 *  - unless a function says otherwise, pointer arguments are host memory; with
 *    DC_DEVICE_PTRS in `flags` they are device memory of the plan's device;
 *  - the caller owns every buffer it passes; the library owns the plan and
 *    everything the plan allocates (released by dc_fspb_destroy);
 *  - no exception crosses the ABI: each call returns a dc_status, and
 *    dc_last_error() gives a message for the calling thread's last failure;
 *  - calls on one plan are not thread-safe; work is ordered on the plan's
 *    CUDA stream.  Calls given host pointers return after the result is in
 *    host memory; calls given device pointers return once the work is queued.
 */
#ifndef DC_FSPB_H
#define DC_FSPB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DC_OK = 0,
    DC_EINVAL = 1,        /* an argument is out of range or inconsistent       */
    DC_ENOMEM = 2,        /* a device or host allocation failed                */
    DC_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed       */
    DC_ETIMEOUT = 4,      /* a bounded device-side wait gave up                */
    DC_EUNSUPPORTED = 5   /* the request is valid but not implemented          */
} dc_status;

#define DC_DEVICE_PTRS 1u  /* flags: pointer arguments are device memory */
#define DC_BATCH_DENSITY 2u  /* batch flags: also recompute the density-dependent steps */

/* Forms of the lateral density correction (Algorithm A1 step 11). */
#define DC_LATERAL_ISO 0   /* the paper's: f(rho(r)), f(rho_hat(r)) at the dose voxel          */
#define DC_LATERAL_AXIS 1  /* densities sampled along the beam's axes (3 x 16 trilinear taps)  */
#define DC_LATERAL_MLP 2   /* the trained network's prediction of the AXIS densities          */

/* Value types of the dose-deposition matrix. */
#define DC_F32 0
#define DC_BF16 1

/* Voxel grid (Section 2.3: CT resampled to a regular grid). */
typedef struct {
    int32_t nx, ny, nz;
    float dx, dy, dz;      /* voxel size                                   */
    float ox, oy, oz;      /* centre of voxel (0, 0, 0)                    */
} dc_grid;

/* One beam (Table 1: gantry/couch angles; Section 2.1: SAD). The field
 * sizes are measured in the isocentre plane and must be whole multiples of
 * the beamlet size. */
typedef struct {
    float gantry_deg, couch_deg, coll_deg;
    float sad;             /* source-to-axis distance                     */
    float iso[3];          /* isocentre                                   */
    float field_x, field_y;
} dc_beam;

/*
 * Commissioned beam model (Section 2.1; Algorithm A1 steps 9-11), as tables
 * looked up by clamped linear interpolation:
 *   A       [a_ntheta][a_nt]  A(t_eq = j a_dt, theta = l a_dtheta), bilinear;
 *   water   [4][w_n]          u_1^w, u_2^w, omega_1^w, omega_2^w at t = j w_dt;
 *   dens    [6][f_n]          f_u1, f_u2, f_omega1, f_omega2, b_1, b_2 at
 *                             rho = f_rho0 + j f_drho (the commissioned density
 *                             range: densities outside it are clamped into it).
 * Every table needs at least 2 entries per axis and a positive step.
 * roi_radius: radius of the ROI cylinder about each beamlet axis (the paper
 * uses 5 cm, footnote to Algorithm A1). smooth_sigma: sigma of the Gaussian
 * that gives rho_hat (step 1), truncated at ceil(3 sigma / delta) voxels per
 * axis. rho_surface: the body surface is where a beamlet axis first/last meets
 * a voxel of density > rho_surface (step 4). density_correction = 0 skips
 * step 11 (conventional FSPB with depth correction only, Algorithm A2 Kernel 5).
 * The host arrays are copied during dc_fspb_create and not kept.
 */
typedef struct {
    const float* A;
    int32_t a_nt, a_ntheta;
    float a_dt, a_dtheta;
    const float* water;
    int32_t w_n;
    float w_dt;
    const float* dens;
    int32_t f_n;
    float f_rho0, f_drho;
    float roi_radius;
    float smooth_sigma;
    float rho_surface;
    int32_t density_correction;
    int32_t lateral_mode;  /* DC_LATERAL_ISO or DC_LATERAL_AXIS at creation (DC_LATERAL_MLP
                              needs weights: see dc_fspb_set_surrogate)                   */
    int32_t reserved[2];   /* must be zero */
} dc_kernel_coeffs;

typedef struct dc_plan dc_plan;
typedef struct dc_batch dc_batch;
typedef struct dc_mlp dc_mlp;

/* Message describing the calling thread's most recent failed call ("" if none). */
const char* dc_last_error(void);
/* Static name of a status code. */
const char* dc_status_str(dc_status s);

/*
 * Builds a plan: uploads the density, computes rho_hat (Algorithm A1 step 1,
 * A2 Kernel 1), the beamlet geometry and angle theta (steps 2-3, Kernel 2),
 * the body entry/exit of every beamlet axis by an FP64 Siddon ray trace
 * (step 4, Kernel 3) and the radiological-depth and omega_corr tables sampled
 * every d = min(dx, dy, dz)/2 (steps 5-6, Kernel 4; Section 2.2).
 *   ct_density  [nz][ny][nx] relative densities >= 0 and finite (host, or
 *               device with DC_DEVICE_PTRS);
 *   beams       n_beams >= 1 host records; the sources must lie outside the grid;
 *   coeffs      host record and host tables;
 *   cuda_stream cudaStream_t on which all of the plan's work runs (NULL = the
 *               legacy default stream); it must outlive the plan.
 * On success *out receives the plan; on failure *out is NULL and nothing leaks.
 * Errors: DC_EINVAL (bad sizes, negative/NaN density, source inside the grid,
 * field not a multiple of the beamlet), DC_ENOMEM, DC_ECUDA.
 */
dc_status dc_fspb_create(const float* ct_density, const dc_grid* grid, const dc_beam* beams,
                         int32_t n_beams, float beamlet_x, float beamlet_y,
                         const dc_kernel_coeffs* coeffs, uint32_t flags, void* cuda_stream,
                         dc_plan** out);

/*
 * Replaces the plan's density with a new one on the same grid (the daily CT of
 * online adaptive replanning, Section 1) and recomputes Algorithm A1 steps 1-6
 * (A2 Kernels 1-4) in place, without reallocating: rho_hat, the per-voxel
 * correction factors, every beamlet's body entry/exit and its tables.  The
 * cached pair count and matrix pattern are invalidated.  Same density rules
 * and pointer flags as dc_fspb_create; with host memory the call returns once
 * the new tables are computed, with DC_DEVICE_PTRS once the work is queued.
 */
dc_status dc_fspb_set_density(dc_plan* plan, const float* ct_density, uint32_t flags);

/* Releases the plan and all memory it owns (NULL is accepted). */
dc_status dc_fspb_destroy(dc_plan* plan);

/* Number of beamlets B (the length of a fluence vector). */
dc_status dc_fspb_n_beamlets(const dc_plan* plan, int32_t* n);

/* Number of voxels V = nx ny nz. */
dc_status dc_fspb_n_voxels(const dc_plan* plan, int64_t* n);
/* Number of (voxel, beam) entries in the plan's beam's-eye-view voxel lists:
 * the units of work of the per-(voxel, beam) lateral-factor passes (the AXIS
 * stencils or the network).  Synchronises.  Errors: DC_EINVAL, DC_ECUDA. */
dc_status dc_fspb_list_entries(dc_plan* plan, int64_t* n);

/*
 * Eq. (1): dose[v] = sum_i f_i D_i(r_v) over the pairs whose voxel lies in
 * beamlet i's ROI cylinder and between its body entry and exit (Algorithm A1
 * steps 7-14, A2 Kernel 5), evaluated in FP32 with fast exponentials.
 *   fluence [B] >= 0; dose [V] written in full (no accumulation).
 * Errors: DC_EINVAL (NULL pointers), DC_ECUDA.
 */
dc_status dc_fspb_dose(dc_plan* plan, const float* fluence, float* dose, uint32_t flags);

/*
 * Eq. (1) for k fluence vectors at once: dose[q][v] = sum_i fluence[q][i] D_i(r_v),
 * each D_i(r_v) evaluated once and applied to all k vectors (1 <= k <= 64):
 * one pass of 16, 32 or 64 vectors (the smallest that holds k), with the
 * beamlets' fluences staged beside their records.  For k > 1 each vector's
 * dose is the same, bit for bit, whatever k it is computed with.
 *   fluence [k][B]; dose [k][V].
 * Scratch, kept by the plan: per-beam partial doses, n_beams * width * V
 * floats (width 16, 32 or 64; 64 in the tensor-core form of
 * DC_PRECISION_BF16), and in that form the fluences packed as B * 64 BF16.
 * Errors: DC_EINVAL (NULL pointers, k outside [1, 64]), DC_ENOMEM, DC_ECUDA.
 */
dc_status dc_fspb_dose_batch(dc_plan* plan, const float* fluence, int32_t k, float* dose,
                             uint32_t flags);

/*
 * Number of (voxel, beamlet) pairs that eq. (1) sums (the nonzero pattern of
 * the dose-deposition matrix); computed on first use and cached. *pairs is
 * host memory.
 */
dc_status dc_fspb_pair_count(dc_plan* plan, int64_t* pairs);

/*
 * Dose-deposition matrix M[v][i] = D_i(r_v) (unit fluence) over the same
 * pairs, as CSR by voxel row with ascending beamlet columns:
 *   rowptr [V + 1] int64, cols [nnz] int32, vals [nnz] float32 (value_dtype
 *   DC_F32) or bfloat16 bits (DC_BF16, round-to-nearest-even of the FP32 value);
 *   nnz = dc_fspb_pair_count().  All three buffers are caller-owned, and all
 *   host or all device memory per `flags`.
 */
dc_status dc_fspb_dose_matrix(dc_plan* plan, int32_t value_dtype, int64_t* rowptr, int32_t* cols,
                              void* vals, uint32_t flags);

/*
 * dc_fspb_dose and dc_fspb_dose_matrix from ONE evaluation of each pair: the
 * CSR fill pass also accumulates eq. (1) for `fluence` [B] into `dose` [V].
 * Results are identical to the two separate calls (same pairs, same order of
 * the sums).  rowptr, cols, vals as for dc_fspb_dose_matrix; fluence and dose
 * host memory, or all five device memory with DC_DEVICE_PTRS.  When the row
 * pattern is not yet known a pair-count pass runs first.
 * Errors: as dc_fspb_dose_matrix.
 */
dc_status dc_fspb_dose_and_matrix(dc_plan* plan, const float* fluence, float* dose, int32_t value_dtype,
                                  int64_t* rowptr, int32_t* cols, void* vals, uint32_t flags);

/*
 * Builds, inside the plan, the dose-deposition matrix of dc_fspb_dose_matrix
 * (M[v][i] = D_i(r_v) over the pairs of eq. 1) with BF16 values, stored
 * block-sparse for the tensor cores: per beam, the voxels of the beam's
 * eye-view binning are cut into row-blocks of 128, and each row-block's
 * nonzeros are covered by dense 128 x 16 tiles, one per 4 x 4 patch of the
 * beam's beamlet grid that holds a pair of the row-block.  The values come
 * straight from the pair evaluation (the same BF16 values, round-to-nearest-even
 * of the FP32 D_i(r), as dc_fspb_dose_matrix with DC_BF16); no CSR is built.
 * Must be called again after dc_fspb_set_density or dc_fspb_autotune.
 * Synchronises the plan's stream.
 * Errors: DC_ENOMEM, DC_ECUDA, DC_EUNSUPPORTED (a beam of > 32768 beamlets).
 */
dc_status dc_fspb_spmm_prepare(dc_plan* plan);

/* Tiles (*chunks, 4 KiB each) and row-blocks of the prepared matrix. */
dc_status dc_fspb_spmm_info(const dc_plan* plan, int64_t* chunks, int64_t* row_blocks);

/*
 * Eq. (1) for k fluence vectors at once as a sparse-dense product on the
 * tensor cores: Y[v][q] = sum_i M[v][i] F[i][q], with M the BF16 matrix of
 * dc_fspb_spmm_prepare, F rounded to BF16 (round-to-nearest-even), products
 * accumulated in FP32 (tcgen05.mma, tensor memory), and the per-beam partial
 * sums of a voxel added in beam order with compensated (Neumaier) summation.
 *   F [B][k] float32 row-major (beamlet-major), 1 <= k <= 64;
 *   Y [V][k] float32 row-major (voxel-major), written in full.
 * Errors: DC_EINVAL (not prepared, bad k), DC_ECUDA, DC_ETIMEOUT (a bounded
 * device-side wait gave up; with DC_DEVICE_PTRS this is reported by the next
 * dc_fspb_device_status).
 */
dc_status dc_fspb_spmm(dc_plan* plan, const float* F, int32_t k, float* Y, uint32_t flags);

/* Limits of dc_fspb_spmm_noalloc's static scratch (per device: 1.05 MiB of
 * packed BF16 fluences and 16 MiB of per-beam partial rows). */
#define DC_SPMM_STATIC_MAX_BEAMLETS 8192
#define DC_SPMM_STATIC_MAX_PARTIALS 4194304

/*
 * dc_fspb_spmm for device buffers, allocating no device memory: the packed
 * fluences and the per-beam partial rows live in file-scope device arrays of
 * fixed size.  The paper has no counterpart; this entry point serves callers
 * that cannot allocate during the call: an optimiser or serving loop that has
 * handed the device's free memory to its own pool (a cudaMalloc would fail or
 * evict), and latency-bound loops where a cudaFree would synchronise the whole
 * device.  Same arithmetic and result as dc_fspb_spmm.
 *   F [B][k] float32, Y [V][k] float32: device memory, caller-owned; the call
 *   is asynchronous on the plan's stream.
 * Limits: the beamlets, counted per beam in whole 4 x 4 patches of its M x N
 * beamlet grid (4 ceil(M/4) x 4 ceil(N/4)), <= DC_SPMM_STATIC_MAX_BEAMLETS
 * and, for plans of more than one beam, (entries of all beam voxel lists) x k
 * <= DC_SPMM_STATIC_MAX_PARTIALS; larger problems are rejected with DC_EINVAL
 * (use dc_fspb_spmm).
 * Set-up: the first call on a device looks up the arrays' device addresses
 * (cudaGetSymbolAddress with that device current); make that first call
 * before any stream capture.
 * The arrays are shared by all plans on a device: calls whose executions
 * overlap (other streams, other plans, other threads) race on them and give
 * undefined results; serialise them.
 * Errors: DC_EINVAL (not prepared, bad k, over the limits), DC_ECUDA;
 * DC_ETIMEOUT of a bounded device-side wait is reported by the next
 * dc_fspb_device_status.
 */
dc_status dc_fspb_spmm_noalloc(dc_plan* plan, const float* F, int32_t k, float* Y);

/* ---- Lateral density correction forms (Algorithm A1 step 11) ----
 *
 * DC_LATERAL_ISO is the paper's reading: f_u1(rho(r)), f_u2/f_omega(rho_hat(r))
 * at the dose voxel.  DC_LATERAL_AXIS samples, for each (voxel r, beam), 16
 * trilinear density taps at (j - 7.5) d, j = 0..15, along each of the beam's
 * axes e_x', e_y', e_z' through r, averages each axis with normalised Gaussian
 * weights (sigma = smooth_sigma) and takes f_u2 at the x and y averages (the
 * penumbra along x and along y) and f_omega at the mean of the three; f_u1
 * stays at rho(r).  DC_LATERAL_MLP predicts the three averages from 48
 * nearest-voxel taps with the surrogate network below, falling back to the
 * AXIS computation for stencils with a density outside [rho_lo, rho_hi].  The
 * factors are computed per density (dc_fspb_create, dc_fspb_set_density) for
 * every (voxel, beam) entry of the beams' voxel lists.
 */

/*
 * Loads the surrogate network into the plan: params [7491] host float32,
 * packed W1[48][64], b1[64], W2[64][64], b2[64], W3[64][3], b3[3]; the network
 * maps x = taps - 1 (48) through two SiLU layers of 64 to y (3) and predicts the
 * effective densities 1 + y (mean, x, y).  Inference runs in BF16 with FP32
 * accumulation.  [rho_lo, rho_hi] is the density range of its training data.
 * Recomputes the factors when the plan is in the network form.  Synchronises.
 * Errors: DC_EINVAL (NULL, non-finite parameter, rho_lo >= rho_hi), DC_ECUDA.
 */
dc_status dc_fspb_set_surrogate(dc_plan* plan, const float* params, float rho_lo, float rho_hi);

/* Selects the lateral form (DC_LATERAL_*; DC_LATERAL_MLP needs
 * dc_fspb_set_surrogate first) and recomputes the per-entry factors.
 * Asynchronous on the plan's stream.  Errors: DC_EINVAL, DC_ECUDA. */
dc_status dc_fspb_set_lateral_mode(dc_plan* plan, int32_t mode);

/* ---- Commissioning (Section 2.1: u, omega, f and b fitted to reference doses) ----
 *
 * Section 2.1 obtains the model's parameters u, omega, f(.) and b(.) by
 * fitting the DC-FSPB dose to reference doses of a slab phantom.  These two
 * calls are what such a fit needs from the engine: new tables for a plan, and
 * the gradient of a weighted dose sum with respect to them.
 *
 * dc_fspb_set_tables replaces the plan's water tables water [4][w_n]
 * (u_1^w, u_2^w, omega_1^w, omega_2^w) and density functions dens [6][f_n]
 * (f_u1, f_u2, f_omega1, f_omega2, b_1, b_2), on the sampling given at
 * creation (host float32; copied before return), and recomputes the
 * density-dependent steps for the plan's current density (the omega_corr
 * tables integrate b).  The depth-dose table A stays.  Errors: DC_EINVAL
 * (NULL, non-finite entry), DC_ECUDA.
 */
dc_status dc_fspb_set_tables(dc_plan* plan, const float* water, const float* dens);

/*
 * Backward pass of eq. (1) with respect to the tables (the vector-Jacobian
 * product of the dose): for voxel weights weights [V] and fluence [B],
 *   g_water[q][j] = sum_v weights[v] dD(v)/d water[q][j]   (q = u_1^w, u_2^w,
 *                                                          omega_1^w, omega_2^w)
 *   g_dens[q][j]  = sum_v weights[v] dD(v)/d dens[q][j]    (q = f_u1, f_u2,
 *                                                          f_omega1, f_omega2)
 *   g_corr[i]     = d/ds at s = 1 of sum_v weights[v] D(v) with b_i scaled
 *                   by s (omega_i^corr scales with b_i), i = 1, 2.
 * The derivative of a table lookup is the weight of the entry in its linear
 * interpolation; a clamp at a table's end puts it on the end entry; where
 * omega_i is clamped at 0 its derivatives are 0.  The b tables enter only
 * through that common scale (their entries act through the ray integrals).
 * Needs the density correction on and DC_LATERAL_ISO (else DC_EUNSUPPORTED).
 * FP32 arithmetic; the sums are accumulated with atomics, so their order (and
 * the last bits) may change between calls.  Pointers host or device
 * (DC_DEVICE_PTRS for all).  Errors: DC_EINVAL, DC_EUNSUPPORTED (also when
 * 4 (w_n + f_n) floats of bins do not fit in shared memory), DC_ENOMEM, DC_ECUDA.
 */
dc_status dc_fspb_dose_vjp(dc_plan* plan, const float* fluence, const float* weights, float* g_water,
                           float* g_dens, float* g_corr, uint32_t flags);

/* ---- Arithmetic of the direct pair evaluation ----
 *
 * Section 2.2 evaluates the exponentials of eq. (4) with the fast,
 * reduced-accuracy hardware function.  DC_PRECISION_FP32 (the default) does
 * the same in FP32.  DC_PRECISION_BF16 is this library's reduced-precision
 * form: the two exponentials of each profile kind of eq. (4) are taken for
 * the x and the y profile at once, as one packed BF16 pair (arguments and
 * results rounded to 8 significant bits); geometry, lookups, eq. (3), eq. (2)
 * and the sum of eq. (1) stay FP32.  Its error against the FP64 oracle is
 * measured against the surrogate bar of 1 % of the maximum dose, not
 * guaranteed.  It applies to dc_fspb_dose (and dc_fspb_dose_batch with k = 1)
 * and to the plan's share of a multi-plan batch.  dc_fspb_dose_batch with
 * k > 1 takes the tensor-core form instead: each pair value D_i(r_v) (FP32
 * exponentials, as in DC_PRECISION_FP32) and each fluence are rounded to BF16
 * (nearest even), and their products for all k <= 64 vectors are summed by
 * mma.m16n8k16 with FP32 accumulators, 16 beamlets of 32 voxels at a time, in
 * one pass; the per-beam sums stay FP32, in beam order.  The matrix calls and
 * the SpMM do not depend on the setting.  Takes effect at the next call; a
 * batch picks it up at its next run.  Errors: DC_EINVAL (NULL plan, unknown
 * value).
 */
#define DC_PRECISION_FP32 0
#define DC_PRECISION_BF16 1
dc_status dc_fspb_set_precision(dc_plan* plan, int32_t precision);

/* Entries of the last network-form factor pass that fell back to the AXIS
 * computation (0 in the other forms).  Synchronises. */
dc_status dc_fspb_lateral_fallbacks(dc_plan* plan, int64_t* n);

/*
 * Network training and test samples for n (voxel, beam) pairs: X [n][48] the
 * nearest-voxel densities at the 3 x 16 tap points (axis-major: e_x', e_y',
 * e_z'), T [n][3] the AXIS effective densities (mean, x, y) of the pair.
 * vox [n] voxel indices, beam [n] beam indices.  Host buffers, or all device
 * buffers with DC_DEVICE_PTRS (then out-of-range indices give NaN rows instead
 * of DC_EINVAL).  Errors: DC_EINVAL (NULL, n < 0, index out of range), DC_ECUDA.
 */
dc_status dc_fspb_stencils(dc_plan* plan, const int32_t* vox, const int32_t* beam, int32_t n, float* X, float* T,
                           uint32_t flags);

/* ---- The surrogate network's trainer (FP32 forward, backward and Adam) ---- */

/* A trainer holding parameters (initial values params [7491], host) and Adam
 * state on the device; its work runs on cuda_stream.  Errors: DC_EINVAL,
 * DC_ENOMEM, DC_ECUDA. */
dc_status dc_mlp_create(const float* params, void* cuda_stream, dc_mlp** out);
dc_status dc_mlp_destroy(dc_mlp* m);
/* Current parameters into out [7491] (host).  Synchronises. */
dc_status dc_mlp_get_params(const dc_mlp* m, float* out);
/* Checkpoint and resume of training (no counterpart in the paper, which
 * trains nothing): the parameters, Adam's first and second moments (each
 * [7491], host float32) and the step count.  A trainer given a saved state
 * continues exactly as the trainer it was saved from would have.
 * Synchronise.  Errors: DC_EINVAL (NULL; set_state: a non-finite value, a
 * negative second moment or step), DC_ECUDA. */
dc_status dc_mlp_get_state(const dc_mlp* m, float* theta, float* m1, float* m2, int64_t* step);
/* Arithmetic of the trainer's gradient (dc_mlp_gradient, dc_mlp_train):
 * DC_PRECISION_FP32 (default, FP32 throughout) or DC_PRECISION_BF16 (the
 * forward and backward products on the tensor cores with BF16 operands and
 * FP32 accumulation, FP32 master parameters and Adam state; per-CTA partial
 * gradients summed in a fixed order, so both stay deterministic).  The
 * network has no counterpart in the paper (it stands in for the AXIS
 * sampling).  Errors: DC_EINVAL. */
dc_status dc_mlp_set_precision(dc_mlp* m, int32_t precision);
dc_status dc_mlp_set_state(dc_mlp* m, const float* theta, const float* m1, const float* m2, int64_t step);
/*
 * Gradient grad [7491] (host) and loss (host, may be NULL) of
 * L = sum_s sum_o (1 + y_so - T_so)^2 / (3 n) over the n samples X [n][48],
 * T [n][3] at the current parameters, in FP32 with per-CTA partial sums added
 * in a fixed order (deterministic).  X, T host, or device with DC_DEVICE_PTRS.
 */
dc_status dc_mlp_gradient(dc_mlp* m, const float* X, const float* T, int32_t n, float* grad, float* loss,
                          uint32_t flags);
/*
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) over `epochs` passes
 * of the samples in the given order, in whole mini-batches of `batch` (a
 * remainder is skipped); *loss (if not NULL) receives L over all n samples
 * after training.  Synchronises.  Errors: DC_EINVAL, DC_ENOMEM, DC_ECUDA.
 */
dc_status dc_mlp_train(dc_mlp* m, const float* X, const float* T, int32_t n, int32_t batch, int32_t epochs,
                       float lr, float* loss, uint32_t flags);
/* Effective densities Y [n][3] = 1 + network(X - 1) with the BF16 tensor-core
 * inference of the dose path, for params [7491] (host).  X, Y host, or device
 * with DC_DEVICE_PTRS.  Synchronises cuda_stream. */
dc_status dc_mlp_predict(const float* params, const float* X, int32_t n, float* Y, uint32_t flags,
                         void* cuda_stream);

/* ---- Several plans in one launch ----
 *
 * Eq. (1) for n plans of uneven grids and beam counts (one fluence vector per
 * plan) as ONE persistent launch of the pair kernel over the work units of all
 * plans (units of the costliest plans first), followed by one launch of the
 * per-plan beam sums, replayed from a CUDA graph built on the first run
 * (dc_fspb_batch_autotune may instead put the plans' own dose launches, one
 * after another, into the graph).  With
 * DC_BATCH_DENSITY the graph also holds each plan's density-dependent work
 * (Algorithm A1 steps 1-6, the beam's-eye-view binning, the lateral factors of
 * step 11) from the plan's resident density, one graph branch per plan, so a
 * run recomputes the whole plans.  Each plan gives the same dose as its own
 * dc_fspb_dose (same per-pair arithmetic; the plans' table and lateral
 * variants are chosen per work unit).
 */

/*
 * plans [n] (1 <= n <= 64, distinct, all on the current device).  The batch
 * owns one device fluence buffer [B_i] (zeroed) and one device dose buffer
 * [V_i] per plan; runs are enqueued on cuda_stream (NULL: legacy default).
 * The plans stay owned by the caller and must outlive the batch; a run is
 * ordered after the work already enqueued on each plan's stream and before
 * work enqueued there afterwards.  Changing a plan (dc_fspb_autotune,
 * dc_fspb_set_lateral_mode, dc_fspb_set_surrogate, a larger
 * dc_fspb_dose_batch) is detected at the next run, which rebuilds the graph.
 * Errors: DC_EINVAL, DC_ENOMEM, DC_ECUDA.
 */
dc_status dc_fspb_batch_create(dc_plan* const* plans, int32_t n, void* cuda_stream, dc_batch** out);

/* Frees the batch (waits for its stream first); NULL is a no-op. */
dc_status dc_fspb_batch_destroy(dc_batch* batch);

/* Device pointers of plan i's fluence [B_i] and dose [V_i] buffers (either out
 * pointer may be NULL).  They stay valid for the batch's lifetime. */
dc_status dc_fspb_batch_buffers(dc_batch* batch, int32_t i, float** fluence, float** dose);

/* Replays the batch graph on the batch's stream (asynchronous): dose_i = D of
 * plan i for the fluence in its batch buffer.  flags: 0 or DC_BATCH_DENSITY.
 * A DC_BATCH_DENSITY run waits for each plan's stream on the host and drops
 * the plans' matrix pattern and SpMM tiles (rebuilt on their next use). */
dc_status dc_fspb_batch_run(dc_batch* batch, uint32_t flags);

/* Copies fluence[i] [B_i] into the batch buffers, runs, copies the doses out
 * to dose[i] [V_i], and waits.  All buffers host memory, or all device memory
 * with DC_DEVICE_PTRS in flags; DC_BATCH_DENSITY as for dc_fspb_batch_run. */
dc_status dc_fspb_batch_dose(dc_batch* batch, const float* const* fluence, float* const* dose, uint32_t flags);

/*
 * Autotuner of the batch's dose graph: replays it (twice, after a warm-up) for
 * each form of the pair work and keeps the fastest: the persistent multi-plan
 * kernel with the register budget for 4 CTAs per SM (variant 0) or for 5
 * (variant 1), or the plans' own dose launches one after another inside the
 * graph (variant 2: each pair kernel specialised for its plan alone, which
 * pays off when every plan fills the GPU by itself).  *variant and *ms (mean
 * replay time) may be NULL.  The doses are the same in every variant.  Runs
 * the batch (its dose buffers are written) and synchronises.
 * Errors: DC_EINVAL, DC_ECUDA.
 */
dc_status dc_fspb_batch_autotune(dc_batch* batch, int32_t* variant, float* ms);

/* Sets the batch's form of the pair work without timing: variant 0, 1 or 2 as
 * dc_fspb_batch_autotune numbers them (the graphs are rebuilt at the next run).
 * Errors: DC_EINVAL (NULL batch, variant out of range). */
dc_status dc_fspb_batch_set_variant(dc_batch* batch, int32_t variant);

/* Waits for the batch's stream. */
dc_status dc_fspb_batch_synchronize(dc_batch* batch);

/* Kernel launches in one replay of the graph for `flags` (0 before the first
 * run with those flags). */
dc_status dc_fspb_batch_kernels(const dc_batch* batch, uint32_t flags, int32_t* kernels);

/* Waits for the plan's stream and reports DC_ETIMEOUT if a bounded
 * device-side wait of an earlier call gave up, else DC_OK. */
dc_status dc_fspb_device_status(dc_plan* plan);

/* ---- Inspection of the plan's intermediate results (for verification) ---- */

/* rho_hat [V] (Algorithm A1 step 1). */
dc_status dc_fspb_get_smoothed(const dc_plan* plan, float* out, uint32_t flags);

/*
 * Per-beamlet geometry (steps 2-4), 16 floats per beamlet into rec [B][16]
 * (host memory): n[3], e_x''[3], e_y''[3], theta, hit (0/1), L_in, L_out,
 * K (number of table samples), 0, 0.
 */
dc_status dc_fspb_get_beamlets(const dc_plan* plan, float* rec);

/*
 * Beamlet i's tables (steps 5-6) at t = k d, k < min(K, kmax), into host
 * arrays teq, w1, w2 (omega_1^corr, omega_2^corr); *K receives the sample count.
 */
dc_status dc_fspb_get_tables(const dc_plan* plan, int32_t i, float* teq, float* w1, float* w2,
                             int32_t kmax, int32_t* K);

/*
 * Autotuner of the plan's work decomposition.  The pair traversal of
 * dc_fspb_dose / dc_fspb_dose_matrix bins, per beam, the voxels by their
 * projection into the isocentre plane (tiles of `tile` cm) and their depth
 * along the beam axis (slabs of `slab` cm), 32 voxels per warp.  This call
 * times dc_fspb_dose for each candidate (tile in {0.35, 0.5, 0.75} cm, slab in
 * {0.5, 1, 2, 4} cm) with `fluence` [B] (host, or device with DC_DEVICE_PTRS), keeps
 * the fastest for the plan, and returns it in *tile, *slab and its time in
 * *best_ms (each output may be NULL).  Results do not depend on the choice
 * (every voxel sums the same pairs in the same order).
 * dc_fspb_set_density keeps the chosen cell size.  Synchronises the plan's
 * stream.  Errors: DC_EINVAL, DC_ECUDA.
 */
dc_status dc_fspb_autotune(dc_plan* plan, const float* fluence, uint32_t flags, float* tile, float* slab,
                           float* best_ms);

/* Number of CUDA kernels this library has launched in the calling process
 * (all plans, all threads), for accounting of GPU work. */
dc_status dc_fspb_launch_count(uint64_t* n);

/* ---- Fluence maps from MLC leaf sequences ----
 *
 * Section 2.3: each plan's leaf sequences and monitor units are converted
 * into a fluence map on the beamlet grid (0.2 x 0.5 cm, 0.2 cm along the leaf
 * motion), which is the fluence eq. (1) weights the beamlets with.  The paper
 * gives no formula; the reading here is the delivered fluence: for beamlet
 * i of a beam, with its rectangle [xa, xb] x [ya, yb] in the isocentre plane of
 * the collimator frame first clipped to the jaws,
 *   f_i = 1/(bx by) * sum over leaf pairs j, control-point intervals c of
 *         h_ij * [ (1 - tau) * (area of the (x, meterset) region that pair j
 *                  leaves open between control points c and c+1, within
 *                  [xa, xb]) + tau * (xb - xa) * (mu_c+1 - mu_c) ]
 * where h_ij is the length of [ya, yb] inside the pair's band and the leaf
 * tips move linearly in meterset between control points.  A step-and-shoot
 * segment is two control points with equal positions; leaf moves between
 * segments sit at a repeated meterset value and deliver nothing.  Outside the
 * leaf bank and the jaws the fluence is zero.  f_i is in meterset units.
 */
typedef struct {
    int32_t n_leaves;     /* leaf pairs, >= 1                                      */
    int32_t n_cp;         /* control points, >= 1 (one control point: no fluence)  */
    const float* edges;   /* [n_leaves + 1] pair boundaries along y (cm), increasing */
    const float* mu;      /* [n_cp] cumulative meterset, non-decreasing             */
    const float* left;    /* [n_cp][n_leaves] tip of the -x bank (cm)               */
    const float* right;   /* [n_cp][n_leaves] tip of the +x bank (cm), >= left      */
    float jaw_x1, jaw_x2; /* jaws along x (cm), x1 <= x2                            */
    float jaw_y1, jaw_y2; /* jaws along y (cm), y1 <= y2                            */
    float transmission;   /* fraction passing closed leaves, in [0, 1]              */
} dc_leaf_sequence;

/*
 * fluence [B] (beamlet order of the plan: beam by beam, row n of a beam at
 * n M + m) from seqs [n_beams], one sequence per beam in the plan's beam
 * order.  The sequences are host memory (read during the call); fluence is
 * host memory, or device memory with DC_DEVICE_PTRS in flags.  The work runs
 * on the plan's stream: with a host fluence the call waits for it; with a
 * device fluence it returns once the kernel is enqueued, so a following
 * dc_fspb_dose on the same plan is ordered after it.  At most 2^28 sequence
 * values in all.
 * Errors: DC_EINVAL (NULL arguments, sizes, non-increasing edges, decreasing
 * or non-finite meterset, left > right, non-finite positions, bad jaws or
 * transmission), DC_ENOMEM, DC_ECUDA.
 */
dc_status dc_fluence_from_leaves(dc_plan* plan, const dc_leaf_sequence* seqs, float* fluence, uint32_t flags);

/* ---- Gamma-index comparison of two dose distributions ----
 *
 * Section 3 (accuracy evaluation) compares each computed dose with a reference
 * dose by the 3-D gamma index at 3 %-3 mm, the percentage taken of the
 * reference's maximum dose, and reports gamma_max over the whole distribution,
 * the mean gamma inside the reference's 50 % isodose line and the percentage
 * of voxels there with gamma < 1 (Tables 2-3).  The paper does not say how the
 * evaluated dose is searched; here, for each reference voxel centre r:
 *   gamma(r) = min(R / dta, min over whole-voxel offsets o, |o| <= R, r + o in
 *              the grid, of sqrt(|o|^2 / dta^2 + (D_eval(r + o) - D_ref(r))^2 / dD^2))
 * with dD = dose_pct / 100 * max D_ref and R = search_cm (gamma is capped at
 * R / dta: any point farther away has a larger distance term alone).
 */
typedef struct {
    double gamma_max;      /* over all voxels                              */
    double gamma_avg50;    /* mean over voxels with D_ref >= 0.5 max D_ref */
    double pass50_pct;     /* % of those voxels with gamma < 1              */
    int64_t n50;           /* number of those voxels                       */
    float dose_max;        /* max D_ref                                    */
} dc_gamma_stats;

/*
 * ref, eval: dose [nz][ny][nx] on `grid` (x fastest); gamma: output of the
 * same size, or NULL for the statistics only; all three host memory, or
 * device memory of the current device with DC_DEVICE_PTRS in `flags`
 * (caller-owned).  dose_pct > 0, dta_cm > 0, search_cm >= dta_cm (<= 64
 * voxels along each axis).  The work runs on `cuda_stream` (NULL: the legacy
 * default stream); the call synchronises it and returns the statistics in
 * *stats (may be NULL).  Results are deterministic.
 * Errors: DC_EINVAL (NULL arguments, bad sizes or criteria, a reference dose
 * that is zero everywhere), DC_ENOMEM, DC_ECUDA.
 */
dc_status dc_gamma_index(const float* ref, const float* eval, const dc_grid* grid, float dose_pct, float dta_cm,
                         float search_cm, float* gamma, dc_gamma_stats* stats, void* cuda_stream,
                         uint32_t flags);

#ifdef __cplusplus
}
#endif

#endif /* DC_FSPB_H */
