// C ABI of the DC-FSPB engine: argument checks, plan memory and the order of
// the kernels on the plan's stream.  Every numerical step runs in the kernels
// of k_prep.cu and k_dose.cu.
#include <math.h>
#include <string.h>

#include <stdlib.h>

#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "dc_internal.cuh"

namespace dc {

static thread_local std::string g_last_error;
static unsigned long long g_launches = 0;

void count_launches(int n) { __atomic_fetch_add(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED); }

void set_error(const std::string& msg) { g_last_error = msg; }

dc_status cuda_fail(cudaError_t e, const char* what)
{
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? DC_ENOMEM : DC_ECUDA;
}

static dc_status invalid(const std::string& msg)
{
    set_error(msg);
    return DC_EINVAL;
}

cudaError_t dev_malloc_bytes(void** p, size_t bytes)
{
    static std::mutex mu;
    static std::string armed;     // value of DC_FSPB_FAIL_ALLOC_AT the count belongs to
    static long long count = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        const char* s = getenv("DC_FSPB_FAIL_ALLOC_AT");
        const std::string now = s ? s : "";
        if (now != armed) {
            armed = now;
            count = 0;
        }
        if (!armed.empty()) {
            const long long at = atoll(armed.c_str());
            if (++count == at) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
        }
    }
    return cudaMalloc(p, bytes);
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n)
{
    return dev_malloc(p, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
}

}  // namespace dc

using namespace dc;

dc::PlanView dc_plan::view() const
{
    PlanView v{};
    v.nx = grid.nx; v.ny = grid.ny; v.nz = grid.nz;
    v.n_beams = n_beams;
    v.B = B;
    v.Kmax = Kmax;
    v.dx = grid.dx; v.dy = grid.dy; v.dz = grid.dz;
    v.ox = grid.ox; v.oy = grid.oy; v.oz = grid.oz;
    v.d = d;
    v.inv_d = 1.0f / d;
    v.roi = coeffs.roi_radius;
    v.R2 = coeffs.roi_radius * coeffs.roi_radius;
    v.bx = bx; v.by = by;
    v.x0 = 0.5f * bx; v.y0 = 0.5f * by;
    v.wscale = coeffs.density_correction ? 1.0f : 0.0f;
    v.arow = d_arow; v.a_nt = coeffs.a_nt; v.inv_adt = 1.0f / coeffs.a_dt;
    v.water = d_water; v.w_n = coeffs.w_n; v.inv_wdt = 1.0f / coeffs.w_dt;
    v.fac = d_fac;
    v.beams = d_beams;
    v.bl = d_bl;
    v.tab = d_tab;
    v.tabm = d_tabm;
    v.lfac = d_lfac;
    v.rho = d_rho;
    v.rhos = d_rhos;
    v.dens = d_dens;
    v.f_n = coeffs.f_n;
    v.f_rho0 = coeffs.f_rho0;
    v.inv_drho = 1.0f / coeffs.f_drho;
    v.idx = 1.0f / grid.dx;
    v.idy = 1.0f / grid.dy;
    v.idz = 1.0f / grid.dz;
    for (int j = 0; j < 16; ++j) v.gw[j] = gw[j];
    v.merged_rt = merged ? 1 : 0;
    v.a_hi = (float)(coeffs.a_nt - 1);
    v.w_hi = (float)(coeffs.w_n - 1);
    v.item_rt = (coeffs.density_correction && lateral_mode != DC_LATERAL_ISO) ? 1 : 0;
    v.prec_rt = precision;
    v.chk = d_chk;
    return v;
}

static void free_plan(dc_plan* p)
{
    if (!p) return;
    void* bufs[] = {p->d_rho, p->d_rhos, p->d_tmp, p->d_fac, p->d_beams, p->d_bl, p->d_theta, p->d_ray, p->d_lio,
                    p->d_tab, p->d_arow, p->d_tabm, p->d_A, p->d_water, p->d_dens, p->d_beamin, p->d_fluence,
                    p->d_dose, p->d_rowcount, p->d_rowptr, p->d_scan_tmp, p->d_mcols, p->d_mvals,
                    p->d_bin, p->d_bounds, p->d_cellof, p->d_hist, p->d_nitems, p->d_bstart, p->d_bscan,
                    p->d_base, p->d_work,
                    p->d_items, p->d_part, p->d_bcount, p->d_sp_fp, p->d_sp_p, p->d_err,
                    p->d_lfac, p->d_mlp_frag, p->d_mlp_bias, p->d_nfall, p->d_leaf, p->d_chk, p->d_grad};
    for (void* b : bufs)
        if (b) cudaFree(b);
    p->spmm_free();
    delete p;
}

extern "C" {

const char* dc_last_error(void) { return g_last_error.c_str(); }

const char* dc_status_str(dc_status s)
{
    switch (s) {
        case DC_OK: return "DC_OK";
        case DC_EINVAL: return "DC_EINVAL";
        case DC_ENOMEM: return "DC_ENOMEM";
        case DC_ECUDA: return "DC_ECUDA";
        case DC_ETIMEOUT: return "DC_ETIMEOUT";
        case DC_EUNSUPPORTED: return "DC_EUNSUPPORTED";
    }
    return "DC_UNKNOWN";
}

// Beam frame in FP64, same convention as the geometry kernel: at gantry 0 the
// beam travels +y with e_x' = +x, e_y' = +z; gantry about +z, couch about +y,
// collimator about the beam axis; source = iso - SAD e_z'.
static void beam_frame_host(const dc_beam& bm, double* ex, double* ey, double* ez, double* src)
{
    const double deg = M_PI / 180.0;
    double fx[3] = {1, 0, 0}, fy[3] = {0, 0, 1}, fz[3] = {0, 1, 0};
    double* v3[3] = {fx, fy, fz};
    const double cg = cos(bm.gantry_deg * deg), sg = sin(bm.gantry_deg * deg);
    const double cc = cos(bm.couch_deg * deg), sc = sin(bm.couch_deg * deg);
    for (double* v : v3) {
        double x = v[0], y = v[1];
        v[0] = cg * x - sg * y;
        v[1] = sg * x + cg * y;
        x = v[0];
        double z = v[2];
        v[0] = cc * x + sc * z;
        v[2] = -sc * x + cc * z;
    }
    const double ck = cos(bm.coll_deg * deg), sk = sin(bm.coll_deg * deg);
    for (int q = 0; q < 3; ++q) {
        ex[q] = ck * fx[q] + sk * fy[q];
        ey[q] = -sk * fx[q] + ck * fy[q];
        ez[q] = fz[q];
        src[q] = bm.iso[q] - bm.sad * fz[q];
    }
}

// Beam's-eye-view binning: default cell size and the autotuner's candidates
// (the plan's binning buffers are sized for the largest grid among them all).
// The default 0.5 x 0.5 cm cell was within 5 % of the tuned dose time on
// thorax9, slab64, H5 and a head-and-neck plan of the 16-plan batch (a 2 cm slab
// was 6-25 % slower on the same plans).
static const float kDefaultTile = 0.5f, kDefaultSlab = 0.5f;
static const float kTuneTiles[] = {0.35f, 0.5f, 0.75f};
static const float kTuneSlabs[] = {0.5f, 1.0f, 2.0f, 4.0f};

// Beam's-eye-view binning grid of each beam (see k_bin.cu).
static void bin_geometry(dc_plan* p, float tile, float slab)
{
    p->bin_tile = tile;
    p->bin_slab = slab;
    const dc_grid& g = p->grid;
    p->bin_host.clear();
    p->tiles_max = 0;
    p->cells_max = 0;
    for (int b = 0; b < p->n_beams; ++b) {
        const dc_beam& bm = p->beams[b];
        double ex[3], ey[3], ez[3], src[3];
        beam_frame_host(bm, ex, ey, ez, src);
        double zmin = 1e300, zmax = -1e300;
        for (int corner = 0; corner < 8; ++corner) {
            const double c[3] = {g.ox + ((corner & 1) ? (g.nx - 1) * (double)g.dx : 0.0),
                                 g.oy + ((corner & 2) ? (g.ny - 1) * (double)g.dy : 0.0),
                                 g.oz + ((corner & 4) ? (g.nz - 1) * (double)g.dz : 0.0)};
            const double zz = (c[0] - src[0]) * ez[0] + (c[1] - src[1]) * ez[1] + (c[2] - src[2]) * ez[2];
            zmin = fmin(zmin, zz);
            zmax = fmax(zmax, zz);
        }
        const double hfx = 0.5 * bm.field_x, hfy = 0.5 * bm.field_y, sad = bm.sad;
        const double inv_cos = sqrt(sad * sad + hfx * hfx + hfy * hfy) / sad;
        BinGeom G;
        G.tile = tile;
        G.slab = slab;
        G.rw_max = (float)(p->coeffs.roi_radius * (sad / zmin) * inv_cos * 1.001 + 2e-3);
        const double ea = hfx + G.rw_max + tile, ec = hfy + G.rw_max + tile;
        G.a0 = (float)-ea;
        G.c0 = (float)-ec;
        G.nta = (int)ceil(2 * ea / tile);
        G.ntc = (int)ceil(2 * ec / tile);
        G.zz0 = (float)(zmin - 1e-3);
        G.nzs = std::max(1, (int)ceil((zmax - zmin + 2e-3) / slab));
        G.cells = G.nta * G.ntc * G.nzs;
        p->bin_host.push_back(G);
        p->tiles_max = std::max(p->tiles_max, G.nta * G.ntc);
        p->cells_max = std::max(p->cells_max, G.cells);
    }
}

// Tiles and cells per beam that any binning the plan can be given needs: the
// default cell and every autotuner candidate.  Leaves the default geometry set.
static void bin_capacity(dc_plan* p, int& tiles_cap, int& cells_cap)
{
    tiles_cap = 0;
    cells_cap = 0;
    for (float t : kTuneTiles)
        for (float sl : kTuneSlabs) {
            bin_geometry(p, t, sl);
            tiles_cap = std::max(tiles_cap, p->tiles_max);
            cells_cap = std::max(cells_cap, p->cells_max);
        }
    bin_geometry(p, kDefaultTile, kDefaultSlab);
    tiles_cap = std::max(tiles_cap, p->tiles_max);
    cells_cap = std::max(cells_cap, p->cells_max);
}

static dc_status check_inputs(const float* ct, const dc_grid* g, const dc_beam* beams, int32_t nb,
                              float bx, float by, const dc_kernel_coeffs* c, uint32_t flags)
{
    if (!ct || !g || !beams || !c) return invalid("dc_fspb_create: NULL argument");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return invalid("dc_fspb_create: empty grid");
    if ((int64_t)g->nx * g->ny * g->nz > (int64_t)1 << 31)
        return invalid("dc_fspb_create: grid larger than 2^31 voxels");
    if (!(g->dx > 0 && g->dy > 0 && g->dz > 0) || !isfinite(g->ox) || !isfinite(g->oy) || !isfinite(g->oz))
        return invalid("dc_fspb_create: voxel size must be positive and the origin finite");
    if (nb < 1 || nb > 64) return invalid("dc_fspb_create: n_beams must be in [1, 64]");
    if (!(bx > 0 && by > 0)) return invalid("dc_fspb_create: beamlet size must be positive");
    if (!c->A || !c->water || !c->dens) return invalid("dc_fspb_create: NULL commissioning table");
    if (c->a_nt < 2 || c->a_ntheta < 2 || c->w_n < 2 || c->f_n < 2)
        return invalid("dc_fspb_create: every table needs at least 2 entries per axis");
    if (!(c->a_dt > 0 && c->a_dtheta > 0 && c->w_dt > 0 && c->f_drho > 0))
        return invalid("dc_fspb_create: table steps must be positive");
    if (!(c->roi_radius > 0) || !(c->smooth_sigma >= 0) || !isfinite(c->rho_surface))
        return invalid("dc_fspb_create: bad roi_radius, smooth_sigma or rho_surface");
    if (c->reserved[0] || c->reserved[1])
        return invalid("dc_fspb_create: reserved fields must be zero");
    if (c->lateral_mode != DC_LATERAL_ISO && c->lateral_mode != DC_LATERAL_AXIS)
        return invalid("dc_fspb_create: lateral_mode must be DC_LATERAL_ISO or DC_LATERAL_AXIS "
                       "(the network form is enabled with dc_fspb_set_surrogate)");
    size_t sm = 2 * sizeof(float4) * c->w_n;
    if (sm > 96 * 1024) {
        set_error("dc_fspb_create: the water table exceeds 96 KiB of shared memory (w_n > 3072)");
        return DC_EUNSUPPORTED;
    }
    double vmin = fmin((double)g->dx, fmin((double)g->dy, (double)g->dz));
    if (c->smooth_sigma > 0 && ceil(3.0 * c->smooth_sigma / vmin) > 64) {
        set_error("dc_fspb_create: smoothing radius above 64 voxels");
        return DC_EUNSUPPORTED;
    }
    const double lo[3] = {g->ox - 0.5 * g->dx, g->oy - 0.5 * g->dy, g->oz - 0.5 * g->dz};
    const double hi[3] = {g->ox + (g->nx - 0.5) * g->dx, g->oy + (g->ny - 0.5) * g->dy,
                          g->oz + (g->nz - 0.5) * g->dz};
    for (int b = 0; b < nb; ++b) {
        const dc_beam& bm = beams[b];
        if (!(bm.sad > 0) || !(bm.field_x > 0) || !(bm.field_y > 0))
            return invalid("dc_fspb_create: beam " + std::to_string(b) + " has a non-positive SAD or field");
        double mx = bm.field_x / bx, my = bm.field_y / by;
        if (fabs(mx - round(mx)) > 1e-3 || fabs(my - round(my)) > 1e-3)
            return invalid("dc_fspb_create: beam " + std::to_string(b) + " field is not a multiple of the beamlet size");
        double ex[3], ey[3], ez[3], src[3];
        beam_frame_host(bm, ex, ey, ez, src);
        // every grid corner must lie in front of the source
        for (int corner = 0; corner < 8; ++corner) {
            double p[3] = {(corner & 1) ? hi[0] : lo[0], (corner & 2) ? hi[1] : lo[1],
                           (corner & 4) ? hi[2] : lo[2]};
            double zz = (p[0] - src[0]) * ez[0] + (p[1] - src[1]) * ez[1] + (p[2] - src[2]) * ez[2];
            if (!(zz > 1e-2))
                return invalid("dc_fspb_create: beam " + std::to_string(b) +
                               ": the grid must lie entirely in front of the source");
        }
    }
    if (!(flags & DC_DEVICE_PTRS)) {
        int64_t V = (int64_t)g->nx * g->ny * g->nz;
        for (int64_t v = 0; v < V; ++v)
            if (!(ct[v] >= 0.f) || !isfinite(ct[v]))
                return invalid("dc_fspb_create: density must be finite and >= 0 (voxel " + std::to_string(v) + ")");
    }
    return DC_OK;
}

// Algorithm A1 steps 1-6 on the plan's stream for the density in d_rho.
static dc_status rerun_density_steps(dc_plan* p)
{
    DC_CUDA(launch_smooth(p, p->coeffs.smooth_sigma));
    DC_CUDA(launch_factors(p));
    DC_CUDA(launch_beamlets(p));
    DC_CUDA(launch_binning(p));
    if (p->coeffs.density_correction && p->lateral_mode != DC_LATERAL_ISO) DC_CUDA(launch_lateral(p));
    p->pairs = -1;
    p->counts_fresh = false;
    if (p->sp_ready) p->spmm_invalidate();   // the SpMM tiles follow the voxel lists
    return DC_OK;
}

// The same for density `ct` (host or device memory).
static dc_status compute_density_steps(dc_plan* p, const float* ct, uint32_t flags)
{
    cudaMemcpyKind k = (flags & DC_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    DC_CUDA(cudaMemcpyAsync(p->d_rho, ct, p->V * sizeof(float), k, p->stream));
    return rerun_density_steps(p);
}

// Water tables (value + slope per depth sample) and density functions to the
// device: (u_1^w, du_1^w, u_2^w, du_2^w), (omega_1^w, domega_1^w, omega_2^w,
// domega_2^w) per sample; dens as given.  Synchronises (the host arrays may
// be released on return).
static dc_status upload_tables(dc_plan* p, const float* water, const float* dens)
{
    const dc_kernel_coeffs& c = p->coeffs;
    std::vector<float4> w(2 * (size_t)c.w_n);
    auto vs = [&](int q, int j, float* val, float* slope) {
        const float* r = water + (size_t)q * c.w_n;
        *val = r[j];
        *slope = j + 1 < c.w_n ? r[j + 1] - r[j] : 0.f;
    };
    for (int j = 0; j < c.w_n; ++j) {
        float a[8];
        for (int q = 0; q < 4; ++q) vs(q, j, &a[2 * q], &a[2 * q + 1]);
        w[2 * j] = make_float4(a[0], a[1], a[2], a[3]);
        w[2 * j + 1] = make_float4(a[4], a[5], a[6], a[7]);
    }
    DC_CUDA(cudaMemcpyAsync(p->d_water, w.data(), w.size() * sizeof(float4), cudaMemcpyHostToDevice, p->stream));
    DC_CUDA(cudaMemcpyAsync(p->d_dens, dens, sizeof(float) * 6 * (size_t)c.f_n, cudaMemcpyHostToDevice, p->stream));
    DC_CUDA(cudaStreamSynchronize(p->stream));
    return DC_OK;
}

// Normalised Gaussian weights of the 16 lateral-stencil taps at (j - 7.5) d.
static void stencil_weights(dc_plan* p)
{
    double w[16], s = 0.0;
    const double sg = p->coeffs.smooth_sigma;
    for (int j = 0; j < 16; ++j) {
        const double x = (j - 7.5) * (double)p->d;
        w[j] = sg > 0 ? exp(-x * x / (2.0 * sg * sg)) : 1.0;
        s += w[j];
    }
    for (int j = 0; j < 16; ++j) p->gw[j] = (float)(w[j] / s);
}

static dc_status create_impl(dc_plan* p, const float* ct, uint32_t flags)
{
    const dc_grid& g = p->grid;
    const dc_kernel_coeffs& c = p->coeffs;
    stencil_weights(p);
    p->lateral_mode = c.lateral_mode;
    const int64_t V = p->V;
    double diag = sqrt((double)g.nx * g.dx * g.nx * g.dx + (double)g.ny * g.dy * g.ny * g.dy +
                       (double)g.nz * g.dz * g.nz * g.dz);
    p->Kmax = (int)ceil(diag / p->d) + 3;
    // the pair kernels address the per-beamlet tables with 32-bit offsets
    if ((double)p->B * 3.0 * p->Kmax >= 2147483648.0 || (double)p->B * c.a_nt >= 2147483648.0) {
        set_error("dc_fspb_create: beamlets x table samples exceed the 32-bit table offsets");
        return DC_EUNSUPPORTED;
    }

    DC_CUDA(dalloc(&p->d_rho, V));
    DC_CUDA(dalloc(&p->d_rhos, V));
    DC_CUDA(dalloc(&p->d_tmp, V));
    DC_CUDA(dalloc(&p->d_fac, V));
    DC_CUDA(dalloc(&p->d_beams, p->n_beams));
    DC_CUDA(dalloc(&p->d_beamin, p->n_beams));
    DC_CUDA(dalloc(&p->d_bl, p->B));
    DC_CUDA(dalloc(&p->d_theta, p->B));
    DC_CUDA(dalloc(&p->d_ray, 8 * (size_t)p->B));
    DC_CUDA(dalloc(&p->d_lio, p->B));
    DC_CUDA(dalloc(&p->d_tab, 2 * (size_t)p->B * p->Kmax));
    DC_CUDA(dalloc(&p->d_arow, (size_t)p->B * c.a_nt));
    p->merged = c.w_dt == p->d;
    if (p->merged) DC_CUDA(dalloc(&p->d_tabm, 3 * (size_t)p->B * p->Kmax));
    DC_CUDA(dalloc(&p->d_A, (size_t)c.a_nt * c.a_ntheta));
    DC_CUDA(dalloc(&p->d_water, 2 * (size_t)c.w_n));
    DC_CUDA(dalloc(&p->d_dens, 6 * (size_t)c.f_n));
    size_t nscan = (size_t)((V + 4095) / 4096) + 2;
    DC_CUDA(dc::dev_malloc(&p->d_scan_tmp, nscan * sizeof(int64_t)));
    p->scan_tmp_bytes = nscan * sizeof(int64_t);

    // beam's-eye-view voxel lists and per-beam partial results
    // capacity for every binning the plan can be given; the default is set
    int tiles_cap = 0, cells_cap = 0;
    bin_capacity(p, tiles_cap, cells_cap);
    const size_t nb = (size_t)p->n_beams;
    DC_CUDA(dalloc(&p->d_bounds, nb * (size_t)tiles_cap));
    DC_CUDA(dalloc(&p->d_hist, nb * (size_t)cells_cap));
    p->tiles_cap = tiles_cap;
    p->cells_cap = cells_cap;
    if (p->tiles_max > p->tiles_cap || p->cells_max > p->cells_cap)
        return invalid("dc_fspb_create: binning grid larger than allocated");
    DC_CUDA(dalloc(&p->d_bin, nb));
    DC_CUDA(dalloc(&p->d_cellof, nb * V));
    DC_CUDA(dalloc(&p->d_nitems, nb));
    DC_CUDA(dalloc(&p->d_bstart, nb + 1));
    DC_CUDA(dalloc(&p->d_bscan, (nb * (size_t)p->cells_cap + 4095) / 4096 + 2));
    DC_CUDA(dalloc(&p->d_base, nb + 1));
    DC_CUDA(dalloc(&p->d_work, 2));
    DC_CUDA(dalloc(&p->d_items, nb * (V + 32)));
    DC_CUDA(dalloc(&p->d_part, nb * V));
    p->part_cap = nb * V;
    DC_CUDA(dalloc(&p->d_bcount, nb * V));
    DC_CUDA(dalloc(&p->d_lfac, nb * (V + 32)));
    DC_CUDA(dalloc(&p->d_nfall, 1));
    DC_CUDA(dalloc(&p->d_chk, 1));
    DC_CUDA(cudaMemsetAsync(p->d_chk, 0, sizeof(int32_t), p->stream));
    DC_CUDA(cudaMemcpyAsync(p->d_bin, p->bin_host.data(), nb * sizeof(BinGeom), cudaMemcpyHostToDevice,
                            p->stream));

    dc_status st = upload_tables(p, c.water, c.dens);
    if (st != DC_OK) return st;
    DC_CUDA(cudaMemcpyAsync(p->d_A, c.A, sizeof(float) * (size_t)c.a_nt * c.a_ntheta,
                            cudaMemcpyHostToDevice, p->stream));
    DC_CUDA(cudaMemcpyAsync(p->d_beamin, p->beams.data(), sizeof(dc_beam) * p->n_beams,
                            cudaMemcpyHostToDevice, p->stream));
    dc_status s = compute_density_steps(p, ct, flags);
    if (s != DC_OK) return s;
    DC_CUDA(cudaStreamSynchronize(p->stream));
    // the host copies of the tables are not kept
    p->coeffs.A = nullptr;
    p->coeffs.water = nullptr;
    p->coeffs.dens = nullptr;
    return DC_OK;
}

dc_status dc_fspb_create(const float* ct_density, const dc_grid* grid, const dc_beam* beams,
                         int32_t n_beams, float beamlet_x, float beamlet_y,
                         const dc_kernel_coeffs* coeffs, uint32_t flags, void* cuda_stream,
                         dc_plan** out)
{
    DC_NVTX("dc_fspb_create");
    if (!out) return invalid("dc_fspb_create: out is NULL");
    *out = nullptr;
    dc_status s = check_inputs(ct_density, grid, beams, n_beams, beamlet_x, beamlet_y, coeffs, flags);
    if (s != DC_OK) return s;
    dc_plan* p = new (std::nothrow) dc_plan();
    if (!p) {
        set_error("dc_fspb_create: host allocation failed");
        return DC_ENOMEM;
    }
    p->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    p->grid = *grid;
    p->V = (int64_t)grid->nx * grid->ny * grid->nz;
    p->n_beams = n_beams;
    p->bx = beamlet_x;
    p->by = beamlet_y;
    p->coeffs = *coeffs;
    p->d = 0.5f * fminf(grid->dx, fminf(grid->dy, grid->dz));
    p->beams.assign(beams, beams + n_beams);
    int B = 0;
    for (int b = 0; b < n_beams; ++b) {
        int M = (int)lround(beams[b].field_x / beamlet_x), N = (int)lround(beams[b].field_y / beamlet_y);
        p->M.push_back(M);
        p->N.push_back(N);
        p->first.push_back(B);
        B += M * N;
    }
    p->B = B;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "cudaGetDevice");
    }
    s = create_impl(p, ct_density, flags);
    if (s != DC_OK) {
        free_plan(p);
        return s;
    }
    *out = p;
    return DC_OK;
}

dc_status dc_fspb_set_density(dc_plan* plan, const float* ct_density, uint32_t flags)
{
    DC_NVTX("dc_fspb_set_density");
    if (!plan || !ct_density) return invalid("dc_fspb_set_density: NULL argument");
    if (!(flags & DC_DEVICE_PTRS)) {
        for (int64_t v = 0; v < plan->V; ++v)
            if (!(ct_density[v] >= 0.f) || !isfinite(ct_density[v]))
                return invalid("dc_fspb_set_density: density must be finite and >= 0 (voxel " +
                               std::to_string(v) + ")");
    }
    dc_status s = compute_density_steps(plan, ct_density, flags);
    if (s != DC_OK) return s;
    if (!(flags & DC_DEVICE_PTRS)) DC_CUDA(cudaStreamSynchronize(plan->stream));
    return DC_OK;
}

static dc_status ensure_staging(dc_plan* p, size_t nflu, size_t ndose);

// Re-bins every beam's voxels with the given cell size (see k_bin.cu).
static dc_status rebin(dc_plan* p, float tile, float slab)
{
    bin_geometry(p, tile, slab);
    if (p->tiles_max > p->tiles_cap || p->cells_max > p->cells_cap) {
        set_error("rebin: binning grid larger than allocated");
        return DC_EINVAL;
    }
    DC_CUDA(cudaMemcpyAsync(p->d_bin, p->bin_host.data(), p->bin_host.size() * sizeof(BinGeom),
                            cudaMemcpyHostToDevice, p->stream));
    DC_CUDA(launch_binning(p));
    if (p->coeffs.density_correction && p->lateral_mode != DC_LATERAL_ISO) DC_CUDA(launch_lateral(p));
    p->pairs = -1;
    p->counts_fresh = false;
    if (p->sp_ready) p->spmm_invalidate();
    ++p->layout_gen;
    return DC_OK;
}

dc_status dc_fspb_autotune(dc_plan* plan, const float* fluence, uint32_t flags, float* tile, float* slab,
                           float* best_ms)
{
    DC_NVTX("dc_fspb_autotune");
    if (!plan || !fluence) return invalid("dc_fspb_autotune: NULL argument");
    const float* f = fluence;
    dc_status s = ensure_staging(plan, (size_t)plan->B, (size_t)plan->V);
    if (s != DC_OK) return s;
    if (!(flags & DC_DEVICE_PTRS)) {
        DC_CUDA(cudaMemcpyAsync(plan->d_fluence, fluence, plan->B * sizeof(float), cudaMemcpyHostToDevice,
                                plan->stream));
        f = plan->d_fluence;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DC_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    float best = 3.0e38f, bt = kDefaultTile, bs = kDefaultSlab;
    s = DC_OK;
    for (float t : kTuneTiles) {
        for (float sl : kTuneSlabs) {
            s = rebin(plan, t, sl);
            if (s != DC_OK) break;
            float ms = 0.f;
            ce = launch_dose(plan, f, 1, plan->B, plan->d_dose, plan->V);
            if (ce == cudaSuccess) ce = cudaEventRecord(e0, plan->stream);
            if (ce == cudaSuccess) ce = launch_dose(plan, f, 1, plan->B, plan->d_dose, plan->V);
            if (ce == cudaSuccess) ce = cudaEventRecord(e1, plan->stream);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (ce != cudaSuccess) {
                s = cuda_fail(ce, "dc_fspb_autotune");
                break;
            }
            if (ms < best) {
                best = ms;
                bt = t;
                bs = sl;
            }
        }
        if (s != DC_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != DC_OK) return s;
    s = rebin(plan, bt, bs);
    if (s != DC_OK) return s;
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    if (tile) *tile = bt;
    if (slab) *slab = bs;
    if (best_ms) *best_ms = best;
    return DC_OK;
}

dc_status dc_fspb_launch_count(uint64_t* n)
{
    if (!n) return invalid("dc_fspb_launch_count: NULL argument");
    *n = __atomic_load_n(&g_launches, __ATOMIC_RELAXED);
    return DC_OK;
}

dc_status dc_fspb_destroy(dc_plan* plan)
{
    DC_NVTX("dc_fspb_destroy");
    if (plan) {
        cudaStreamSynchronize(plan->stream);
        free_plan(plan);
    }
    return DC_OK;
}

dc_status dc_fspb_n_beamlets(const dc_plan* plan, int32_t* n)
{
    if (!plan || !n) return invalid("dc_fspb_n_beamlets: NULL argument");
    *n = plan->B;
    return DC_OK;
}

dc_status dc_fspb_n_voxels(const dc_plan* plan, int64_t* n)
{
    if (!plan || !n) return invalid("dc_fspb_n_voxels: NULL argument");
    *n = plan->V;
    return DC_OK;
}

dc_status dc_fspb_list_entries(dc_plan* plan, int64_t* n)
{
    if (!plan || !n) return invalid("dc_fspb_list_entries: NULL argument");
    std::vector<int32_t> items(plan->n_beams);
    DC_CUDA(cudaMemcpyAsync(items.data(), plan->d_nitems, plan->n_beams * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            plan->stream));
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    int64_t s = 0;
    for (int32_t x : items) s += x;
    *n = s;
    return DC_OK;
}

// Per-beam partial dose buffer of at least `need` floats.
static dc_status ensure_part(dc_plan* p, size_t need)
{
    if (need <= p->part_cap) return DC_OK;
    DC_CUDA(cudaStreamSynchronize(p->stream));
    cudaFree(p->d_part);
    p->d_part = nullptr;
    p->part_cap = 0;
    DC_CUDA(dalloc(&p->d_part, need));
    p->part_cap = need;
    ++p->layout_gen;
    return DC_OK;
}

static dc_status ensure_staging(dc_plan* p, size_t nflu, size_t ndose)
{
    if (nflu > p->fluence_cap) {
        if (p->d_fluence) cudaFree(p->d_fluence);
        p->d_fluence = nullptr;
        p->fluence_cap = 0;
        DC_CUDA(dalloc(&p->d_fluence, nflu));
        p->fluence_cap = nflu;
    }
    if (ndose > p->dose_cap) {
        if (p->d_dose) cudaFree(p->d_dose);
        p->d_dose = nullptr;
        p->dose_cap = 0;
        DC_CUDA(dalloc(&p->d_dose, ndose));
        p->dose_cap = ndose;
    }
    return DC_OK;
}

dc_status dc_fspb_dose_batch(dc_plan* plan, const float* fluence, int32_t k, float* dose, uint32_t flags)
{
    DC_NVTX("dc_fspb_dose_batch");
    if (!plan || !fluence || !dose) return invalid("dc_fspb_dose: NULL argument");
    if (k < 1 || k > 64) return invalid("dc_fspb_dose_batch: k must be in [1, 64]");
    const size_t nf = (size_t)k * plan->B, nd = (size_t)k * plan->V;
    // per-beam partial doses of one pass (up to 64 fluence vectors); the
    // tensor-core form (reduced precision, k > 1) also packs the fluences
    const bool tc = k > 1 && plan->precision == DC_PRECISION_BF16;
    dc_status ps = ensure_part(plan, (size_t)plan->n_beams * (tc ? 64 : dose_pass_width(k)) * plan->V);
    if (ps != DC_OK) return ps;
    if (tc && plan->sp_fp_cap < (size_t)plan->B * 64) {
        if (plan->d_sp_fp) cudaFree(plan->d_sp_fp);
        plan->d_sp_fp = nullptr;
        plan->sp_fp_cap = 0;
        DC_CUDA(dc::dev_malloc(&plan->d_sp_fp, (size_t)plan->B * 64 * sizeof(uint16_t)));
        plan->sp_fp_cap = (size_t)plan->B * 64;
    }
    // a single-fluence pass records the pair counts of the matrix pattern
    // while the pattern is unknown (every pair test is made there anyway)
    const bool record = k == 1 && plan->pairs < 0 && !plan->counts_fresh;
    if (flags & DC_DEVICE_PTRS) {
        DC_CUDA(launch_dose(plan, fluence, k, plan->B, dose, plan->V, record));
        if (record) plan->counts_fresh = true;
        return DC_OK;
    }
    dc_status s = ensure_staging(plan, nf, nd);
    if (s != DC_OK) return s;
    DC_CUDA(cudaMemcpyAsync(plan->d_fluence, fluence, nf * sizeof(float), cudaMemcpyHostToDevice, plan->stream));
    DC_CUDA(launch_dose(plan, plan->d_fluence, k, plan->B, plan->d_dose, plan->V, record));
    if (record) plan->counts_fresh = true;
    DC_CUDA(cudaMemcpyAsync(dose, plan->d_dose, nd * sizeof(float), cudaMemcpyDeviceToHost, plan->stream));
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    return DC_OK;
}

dc_status dc_fspb_dose(dc_plan* plan, const float* fluence, float* dose, uint32_t flags)
{
    return dc_fspb_dose_batch(plan, fluence, 1, dose, flags);
}

static dc_status ensure_pattern(dc_plan* p)
{
    if (p->pairs >= 0) return DC_OK;
    if (!p->d_rowcount) DC_CUDA(dalloc(&p->d_rowcount, p->V));
    if (!p->d_rowptr) DC_CUDA(dalloc(&p->d_rowptr, p->V + 1));
    if (p->counts_fresh)
        DC_CUDA(launch_rowsum(p, p->d_rowcount));
    else
        DC_CUDA(launch_count(p, p->d_rowcount));
    p->counts_fresh = true;
    int64_t* total = reinterpret_cast<int64_t*>(p->d_scan_tmp) + (p->scan_tmp_bytes / sizeof(int64_t) - 1);
    DC_CUDA(launch_scan_counts(p, p->d_rowcount, p->d_rowptr, total));
    int64_t h = 0;
    DC_CUDA(cudaMemcpyAsync(&h, total, sizeof(int64_t), cudaMemcpyDeviceToHost, p->stream));
    DC_CUDA(cudaStreamSynchronize(p->stream));
    p->pairs = h;
    return DC_OK;
}

dc_status dc_fspb_pair_count(dc_plan* plan, int64_t* pairs)
{
    DC_NVTX("dc_fspb_pair_count");
    if (!plan || !pairs) return invalid("dc_fspb_pair_count: NULL argument");
    dc_status s = ensure_pattern(plan);
    if (s != DC_OK) return s;
    *pairs = plan->pairs;
    return DC_OK;
}

// The CSR matrix, and with a fluence also eq. (1), from one fill pass.
static dc_status matrix_impl(dc_plan* plan, int32_t value_dtype, int64_t* rowptr, int32_t* cols, void* vals,
                             const float* fluence, float* dose, uint32_t flags, const char* who)
{
    if (!plan || !rowptr || !cols || !vals) return invalid(std::string(who) + ": NULL argument");
    if (value_dtype != DC_F32 && value_dtype != DC_BF16)
        return invalid(std::string(who) + ": value_dtype must be DC_F32 or DC_BF16");
    if (fluence) {
        dc_status s = ensure_part(plan, (size_t)plan->n_beams * plan->V);
        if (s != DC_OK) return s;
    }
    dc_status s = ensure_pattern(plan);
    if (s != DC_OK) return s;
    const size_t nnz = (size_t)plan->pairs, vsz = value_dtype == DC_BF16 ? 2 : 4;
    if (flags & DC_DEVICE_PTRS) {
        DC_CUDA(cudaMemcpyAsync(rowptr, plan->d_rowptr, (plan->V + 1) * sizeof(int64_t),
                                cudaMemcpyDeviceToDevice, plan->stream));
        DC_CUDA(launch_fill(plan, plan->d_rowptr, cols, vals, value_dtype, fluence, dose));
        return DC_OK;
    }
    const size_t need = nnz * sizeof(int32_t) + 16;
    if (need > plan->mstage_bytes) {
        if (plan->d_mcols) cudaFree(plan->d_mcols);
        if (plan->d_mvals) cudaFree(plan->d_mvals);
        plan->d_mcols = nullptr;
        plan->d_mvals = nullptr;
        plan->mstage_bytes = 0;
        DC_CUDA(dc::dev_malloc(&plan->d_mcols, need));
        DC_CUDA(dc::dev_malloc(&plan->d_mvals, need));
        plan->mstage_bytes = need;
    }
    if (fluence) {
        s = ensure_staging(plan, plan->B, plan->V);
        if (s != DC_OK) return s;
        DC_CUDA(cudaMemcpyAsync(plan->d_fluence, fluence, plan->B * sizeof(float), cudaMemcpyHostToDevice,
                                plan->stream));
    }
    int32_t* dcols = plan->d_mcols;
    void* dvals = plan->d_mvals;
    cudaError_t e = launch_fill(plan, plan->d_rowptr, dcols, dvals, value_dtype, fluence ? plan->d_fluence : nullptr,
                                fluence ? plan->d_dose : nullptr);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rowptr, plan->d_rowptr, (plan->V + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                            plan->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cols, dcols, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, plan->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vals, dvals, nnz * vsz, cudaMemcpyDeviceToHost, plan->stream);
    if (e == cudaSuccess && fluence)
        e = cudaMemcpyAsync(dose, plan->d_dose, plan->V * sizeof(float), cudaMemcpyDeviceToHost, plan->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return DC_OK;
}

dc_status dc_fspb_dose_matrix(dc_plan* plan, int32_t value_dtype, int64_t* rowptr, int32_t* cols,
                              void* vals, uint32_t flags)
{
    DC_NVTX("dc_fspb_dose_matrix");
    return matrix_impl(plan, value_dtype, rowptr, cols, vals, nullptr, nullptr, flags, "dc_fspb_dose_matrix");
}

dc_status dc_fspb_dose_and_matrix(dc_plan* plan, const float* fluence, float* dose, int32_t value_dtype,
                                  int64_t* rowptr, int32_t* cols, void* vals, uint32_t flags)
{
    DC_NVTX("dc_fspb_dose_and_matrix");
    if (!fluence || !dose) return invalid("dc_fspb_dose_and_matrix: NULL argument");
    return matrix_impl(plan, value_dtype, rowptr, cols, vals, fluence, dose, flags, "dc_fspb_dose_and_matrix");
}

dc_status dc_fspb_set_tables(dc_plan* plan, const float* water, const float* dens)
{
    DC_NVTX("dc_fspb_set_tables");
    if (!plan || !water || !dens) return invalid("dc_fspb_set_tables: NULL argument");
    const dc_kernel_coeffs& c = plan->coeffs;
    for (size_t q = 0; q < 4 * (size_t)c.w_n; ++q)
        if (!isfinite(water[q])) return invalid("dc_fspb_set_tables: non-finite water table entry");
    for (size_t q = 0; q < 6 * (size_t)c.f_n; ++q)
        if (!isfinite(dens[q])) return invalid("dc_fspb_set_tables: non-finite density-function entry");
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    dc_status s = upload_tables(plan, water, dens);
    if (s != DC_OK) return s;
    return rerun_density_steps(plan);
}

dc_status dc_fspb_dose_vjp(dc_plan* plan, const float* fluence, const float* weights, float* g_water, float* g_dens,
                           float* g_corr, uint32_t flags)
{
    DC_NVTX("dc_fspb_dose_vjp");
    if (!plan || !fluence || !weights || !g_water || !g_dens || !g_corr)
        return invalid("dc_fspb_dose_vjp: NULL argument");
    if (!plan->coeffs.density_correction || plan->lateral_mode != DC_LATERAL_ISO) {
        set_error("dc_fspb_dose_vjp: needs the density correction on and the paper's lateral form (DC_LATERAL_ISO)");
        return DC_EUNSUPPORTED;
    }
    const dc_kernel_coeffs& c = plan->coeffs;
    const size_t nw = 4 * (size_t)c.w_n, nd = 4 * (size_t)c.f_n;
    if (2 * sizeof(float4) * c.w_n + sizeof(float) * (nw + nd + 2) > 200 * 1024) {
        set_error("dc_fspb_dose_vjp: water and density tables too long for the shared-memory gradient bins");
        return DC_EUNSUPPORTED;
    }
    if (flags & DC_DEVICE_PTRS) {
        DC_CUDA(launch_dose_vjp(plan, fluence, weights, g_water, g_dens, g_corr));
        return DC_OK;
    }
    // host buffers: staged through the plan's fluence/dose staging plus one
    // gradient block
    dc_status s = ensure_staging(plan, plan->B, plan->V);
    if (s != DC_OK) return s;
    if (!plan->d_grad) {   // the plan's gradient block, kept for later calls
        DC_CUDA(dalloc(&plan->d_grad, nw + nd + 2));
    }
    float* d_g = plan->d_grad;
    cudaError_t e = cudaMemcpyAsync(plan->d_fluence, fluence, plan->B * sizeof(float), cudaMemcpyHostToDevice,
                                    plan->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(plan->d_dose, weights, plan->V * sizeof(float), cudaMemcpyHostToDevice, plan->stream);
    if (e == cudaSuccess) e = launch_dose_vjp(plan, plan->d_fluence, plan->d_dose, d_g, d_g + nw, d_g + nw + nd);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_water, d_g, nw * sizeof(float), cudaMemcpyDeviceToHost, plan->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g_dens, d_g + nw, nd * sizeof(float), cudaMemcpyDeviceToHost, plan->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g_corr, d_g + nw + nd, 2 * sizeof(float), cudaMemcpyDeviceToHost, plan->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
    if (e != cudaSuccess) return cuda_fail(e, "dc_fspb_dose_vjp");
    return DC_OK;
}

static dc_status check_device_status(dc_plan* p)
{
    if (p->d_chk) {
        int32_t c = 0;
        DC_CUDA(cudaMemcpyAsync(&c, p->d_chk, sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream));
        DC_CUDA(cudaStreamSynchronize(p->stream));
        if (c != 0) {
            static const char* what[] = {"", "depth-table sample", "A-row sample", "water-table sample",
                                         "voxel-list work unit", "beamlet record or fluence", "CSR row segment",
                                         "patch bitmap word"};
            set_error(std::string("bounds check: a pair kernel's ") + (c > 0 && c < 8 ? what[c] : "index") +
                      " index was out of range (DC_BOUNDS_CHECK build)");
            return DC_ECUDA;
        }
    }
    if (!p->d_err) return DC_OK;
    int32_t h = 0;
    DC_CUDA(cudaMemcpyAsync(&h, p->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream));
    DC_CUDA(cudaStreamSynchronize(p->stream));
    if (h != 0) {
        set_error("a bounded device-side wait gave up (tensor-core pipeline did not complete)");
        return DC_ETIMEOUT;
    }
    return DC_OK;
}

dc_status dc_fspb_device_status(dc_plan* plan)
{
    if (!plan) return invalid("dc_fspb_device_status: NULL argument");
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    return check_device_status(plan);
}

dc_status dc_fspb_spmm_prepare(dc_plan* plan)
{
    DC_NVTX("dc_fspb_spmm_prepare");
    if (!plan) return invalid("dc_fspb_spmm_prepare: NULL argument");
    // the tiles come straight from the pair evaluation (no CSR in between)
    return spmm_prepare(plan);
}

dc_status dc_fspb_spmm_info(const dc_plan* plan, int64_t* chunks, int64_t* row_blocks)
{
    if (!plan) return invalid("dc_fspb_spmm_info: NULL argument");
    if (!plan->sp_ready) return invalid("dc_fspb_spmm_info: call dc_fspb_spmm_prepare first");
    if (chunks) *chunks = plan->sp_chunks;
    if (row_blocks) *row_blocks = plan->sp_n_rb;
    return DC_OK;
}

dc_status dc_fspb_spmm(dc_plan* plan, const float* F, int32_t k, float* Y, uint32_t flags)
{
    DC_NVTX("dc_fspb_spmm");
    if (!plan || !F || !Y) return invalid("dc_fspb_spmm: NULL argument");
    if (k < 1 || k > 64) return invalid("dc_fspb_spmm: k must be in [1, 64]");
    if (!plan->sp_ready) return invalid("dc_fspb_spmm: call dc_fspb_spmm_prepare first");
    if (flags & DC_DEVICE_PTRS) {
        DC_CUDA(spmm_run(plan, F, k, Y));
        return DC_OK;
    }
    const size_t nf = (size_t)k * plan->B, ny = (size_t)k * plan->V;
    dc_status s = ensure_staging(plan, nf, ny);
    if (s != DC_OK) return s;
    DC_CUDA(cudaMemcpyAsync(plan->d_fluence, F, nf * sizeof(float), cudaMemcpyHostToDevice, plan->stream));
    DC_CUDA(spmm_run(plan, plan->d_fluence, k, plan->d_dose));
    DC_CUDA(cudaMemcpyAsync(Y, plan->d_dose, ny * sizeof(float), cudaMemcpyDeviceToHost, plan->stream));
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    return check_device_status(plan);
}

dc_status dc_fspb_spmm_noalloc(dc_plan* plan, const float* F, int32_t k, float* Y)
{
    DC_NVTX("dc_fspb_spmm_noalloc");
    if (!plan || !F || !Y) return invalid("dc_fspb_spmm_noalloc: NULL argument");
    if (k < 1 || k > 64) return invalid("dc_fspb_spmm_noalloc: k must be in [1, 64]");
    if (!plan->sp_ready) return invalid("dc_fspb_spmm_noalloc: call dc_fspb_spmm_prepare first");
    if (plan->sp_cols > DC_SPMM_STATIC_MAX_BEAMLETS)
        return invalid("dc_fspb_spmm_noalloc: " + std::to_string(plan->sp_cols) +
                       " beamlets (in whole 4 x 4 patches per beam) exceed the static scratch limit of " +
                       std::to_string(DC_SPMM_STATIC_MAX_BEAMLETS) + "; use dc_fspb_spmm");
    if (plan->n_beams > 1 && plan->sp_items_total * (int64_t)k > (int64_t)DC_SPMM_STATIC_MAX_PARTIALS)
        return invalid("dc_fspb_spmm_noalloc: " + std::to_string(plan->sp_items_total) + " beam-list entries x k = " +
                       std::to_string(k) + " partial values exceed the static scratch limit of " +
                       std::to_string(DC_SPMM_STATIC_MAX_PARTIALS) + "; use dc_fspb_spmm");
    DC_CUDA(spmm_run_static(plan, F, k, Y));
    return DC_OK;
}

dc_status dc_fspb_get_smoothed(const dc_plan* plan, float* out, uint32_t flags)
{
    if (!plan || !out) return invalid("dc_fspb_get_smoothed: NULL argument");
    cudaMemcpyKind k = (flags & DC_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    DC_CUDA(cudaMemcpyAsync(out, plan->d_rhos, plan->V * sizeof(float), k, plan->stream));
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    return DC_OK;
}

dc_status dc_fspb_get_beamlets(const dc_plan* plan, float* rec)
{
    if (!plan || !rec) return invalid("dc_fspb_get_beamlets: NULL argument");
    std::vector<BeamletDev> bl(plan->B);
    std::vector<float> th(plan->B);
    DC_CUDA(cudaMemcpyAsync(bl.data(), plan->d_bl, sizeof(BeamletDev) * plan->B, cudaMemcpyDeviceToHost,
                            plan->stream));
    DC_CUDA(cudaMemcpyAsync(th.data(), plan->d_theta, sizeof(float) * plan->B, cudaMemcpyDeviceToHost,
                            plan->stream));
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    for (int i = 0; i < plan->B; ++i) {
        float* r = rec + 16 * (size_t)i;
        const BeamletDev& b = bl[i];
        r[0] = b.n_lin.x; r[1] = b.n_lin.y; r[2] = b.n_lin.z;
        r[3] = b.exy_xy.x; r[4] = b.exy_xy.z; r[5] = b.exy_z.x;
        r[6] = b.exy_xy.y; r[7] = b.exy_xy.w; r[8] = b.exy_z.y;
        r[9] = th[i];
        r[10] = (float)b.meta.z;
        r[11] = b.n_lin.w;
        r[12] = b.exy_z.z;
        r[13] = (float)b.meta.x;
        r[14] = r[15] = 0.f;
    }
    return DC_OK;
}

dc_status dc_fspb_get_tables(const dc_plan* plan, int32_t i, float* teq, float* w1, float* w2, int32_t kmax,
                             int32_t* K)
{
    if (!plan || !teq || !w1 || !w2 || !K) return invalid("dc_fspb_get_tables: NULL argument");
    if (i < 0 || i >= plan->B) return invalid("dc_fspb_get_tables: beamlet index out of range");
    BeamletDev b;
    DC_CUDA(cudaMemcpyAsync(&b, plan->d_bl + i, sizeof(b), cudaMemcpyDeviceToHost, plan->stream));
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    *K = b.meta.x;
    int n = b.meta.x < kmax ? b.meta.x : kmax;
    if (n <= 0) return DC_OK;
    std::vector<float4> t(2 * (size_t)n);
    DC_CUDA(cudaMemcpyAsync(t.data(), plan->d_tab + 2 * (size_t)i * plan->Kmax, 2 * n * sizeof(float4),
                            cudaMemcpyDeviceToHost, plan->stream));
    DC_CUDA(cudaStreamSynchronize(plan->stream));
    for (int k = 0; k < n; ++k) {
        teq[k] = t[2 * k].x;
        w1[k] = t[2 * k].z;
        w2[k] = t[2 * k + 1].x;
    }
    return DC_OK;
}

}  // extern "C"
