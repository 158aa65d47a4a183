// Beam's-eye-view binning of voxels, per beam, for the pair traversal.
//
// For beam b every voxel r is projected into the isocentre plane
// (a, c) = SAD (r - s).(e_x', e_y') / (r - s).e_z' and binned into cells of
// `tile` x `tile` cm in (a, c) and `slab` cm in depth (r - s).e_z'.  The voxels
// of one warp then share almost the same set of beamlets whose ROI cylinder
// can hold them (Algorithm A1 step 8), so the warp's traversal wastes few
// lanes.  A voxel is dropped from beam b's list when no beamlet near its
// projection can reach it in depth: every pair needs L_in <= |r_a| <= |r - s|
// and sqrt(|r - s|^2 - R^2) <= |r_a| <= L_out, so a voxel with
// |r - s| < min L_in or sqrt(|r - s|^2 - R^2) > max L_out over those beamlets
// is in no pair.  The bounds are taken per tile over all beamlets whose axes
// pass within (window radius + tile half-diagonal) of the tile centre.
#include <math.h>

#include "dc_internal.cuh"

namespace dc {
namespace {

constexpr float kBig = 3.0e38f;

// Per (beam, tile): min L_in and max L_out of the hit beamlets whose centre
// lies within rw_max + half the tile diagonal of the tile's centre (in the
// isocentre plane).  One warp per tile: the lanes run along each row of
// beamlets inside that disc, then a warp reduction.
constexpr int kBoundsWarps = 8;
__global__ void __launch_bounds__(32 * kBoundsWarps) k_bev_bounds(const BinGeom* __restrict__ G, int n_beams,
                                                                  const BeamDev* __restrict__ beams,
                                                                  const float2* __restrict__ lio, float bx,
                                                                  float by, float2* __restrict__ bounds,
                                                                  int tiles_max)
{
    const int b = blockIdx.y;
    if (b >= n_beams) return;
    const int lane = threadIdx.x & 31;
    const BinGeom g = G[b];
    const int ntile = g.nta * g.ntc;
    const int M = beams[b].M, N = beams[b].N, first = beams[b].first;
    const float hfx = beams[b].half_fx, hfy = beams[b].half_fy;
    const float reach = g.rw_max + 0.7072f * g.tile;
    const int nwarps = gridDim.x * kBoundsWarps;
    for (int t = blockIdx.x * kBoundsWarps + (threadIdx.x >> 5); t < ntile; t += nwarps) {
        const int ta = t % g.nta, tc = t / g.nta;
        const float ca = g.a0 + (ta + 0.5f) * g.tile, cc = g.c0 + (tc + 0.5f) * g.tile;
        const int n0 = max(0, (int)floorf((cc - reach + hfy) / by - 0.5f));
        const int n1 = min(N - 1, (int)ceilf((cc + reach + hfy) / by - 0.5f));
        float lmin = kBig, lmax = -kBig;
        for (int n = n0; n <= n1; ++n) {
            const float dc_ = cc - (-hfy + (n + 0.5f) * by);
            // the row's beamlets within the disc's chord, one beamlet of slack
            // each side (the exact test below decides)
            const float h = sqrtf(fmaxf(reach * reach - dc_ * dc_, 0.f));
            const int m0 = max(0, (int)floorf((ca - h + hfx) / bx - 1.5f));
            const int m1 = min(M - 1, (int)ceilf((ca + h + hfx) / bx + 0.5f));
            for (int m = m0 + lane; m <= m1; m += 32) {
                const float da = ca - (-hfx + (m + 0.5f) * bx);
                if (da * da + dc_ * dc_ > reach * reach) continue;
                const float2 r = __ldg(lio + first + n * M + m);
                if (r.y < 0.f) continue;             // axis misses the body
                lmin = fminf(lmin, r.x);
                lmax = fmaxf(lmax, r.y);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lmin = fminf(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
            lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        }
        if (lane == 0) bounds[(size_t)b * tiles_max + t] = make_float2(lmin, lmax);
    }
}

__device__ __forceinline__ int voxel_cell(const BinGeom& g, const BeamDev& bm, const float2* bounds,
                                          float R2, float rx, float ry, float rz)
{
    const float vx = rx - bm.src[0], vy = ry - bm.src[1], vz = rz - bm.src[2];
    const float zz = vx * bm.ez[0] + vy * bm.ez[1] + vz * bm.ez[2];
    if (!(zz > 1e-3f)) return -1;
    const float s = bm.sad / zz;
    const float a = (vx * bm.ex[0] + vy * bm.ex[1] + vz * bm.ex[2]) * s;
    const float c = (vx * bm.ey[0] + vy * bm.ey[1] + vz * bm.ey[2]) * s;
    const int ta = (int)floorf((a - g.a0) / g.tile), tc = (int)floorf((c - g.c0) / g.tile);
    if (ta < 0 || ta >= g.nta || tc < 0 || tc >= g.ntc) return -1;
    const float2 lb = bounds[tc * g.nta + ta];
    const float d2 = vx * vx + vy * vy + vz * vz;
    const float dist = sqrtf(d2);
    if (dist < lb.x - 1e-3f) return -1;
    if (sqrtf(fmaxf(d2 - R2, 0.f)) > lb.y + 1e-3f) return -1;
    const int zs = min(max((int)floorf((zz - g.zz0) / g.slab), 0), g.nzs - 1);
    return (tc * g.nta + ta) * g.nzs + zs;
}

// Pass 1: cell of every (beam, voxel) (-1: not in the beam's list) and cell histograms.
__global__ void __launch_bounds__(256) k_bin_hist(const PlanView P, const BinGeom* __restrict__ G,
                                                  const float2* __restrict__ bounds, int tiles_max,
                                                  int cells_max, int32_t* __restrict__ cellof,
                                                  int32_t* __restrict__ hist)
{
    const int b = blockIdx.y;
    const BinGeom g = G[b];
    const BeamDev bm = P.beams[b];
    const int64_t V = (int64_t)P.nx * P.ny * P.nz;
    const int lane = threadIdx.x & 31;
    // whole warps iterate together: the lanes of a warp that fall into the
    // same cell add to its count with one atomic
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); v0 < V; v0 += step) {
        const int64_t v = v0 + lane;
        int cell = -1;
        if (v < V) {
            // voxel indices fit 32 bits (the voxel lists hold int32): 32-bit division
            const uint32_t u = (uint32_t)v, nx = (uint32_t)P.nx, ny = (uint32_t)P.ny;
            const uint32_t q = u / nx;
            const int ix = (int)(u - q * nx), iy = (int)(q % ny), iz = (int)(q / ny);
            cell = voxel_cell(g, bm, bounds + (size_t)b * tiles_max, P.R2, fmaf((float)ix, P.dx, P.ox),
                              fmaf((float)iy, P.dy, P.oy), fmaf((float)iz, P.dz, P.oz));
            cellof[(size_t)b * V + v] = cell;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, cell);
        if (cell >= 0 && lane == __ffs(peers) - 1) atomicAdd(hist + (size_t)b * cells_max + cell, __popc(peers));
    }
}

// Pass 2: exclusive scan of all beams' cell histograms, [n_beams][cells_max]
// in one range, in place (the histogram becomes the cell cursors); beam b's
// cells start at bstart[b] in that range and bstart[n_beams] is the total.
// Three kernels: chunk sums, a scan of the chunk sums, and the scan inside
// each chunk plus its chunk's offset.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanChunk = kScanThreads * kScanPer;

__device__ __forceinline__ int32_t block_exclusive_scan32(int32_t x, int32_t* s_warp, int32_t* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
        int32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    const int32_t r = incl - x + s_warp[warp];
    *total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_cell_scan_sums(const int32_t* __restrict__ h, int64_t n,
                                                                 int32_t* __restrict__ sums)
{
    __shared__ int32_t sw[33];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    int32_t s = 0;
    for (int q = 0; q < kScanPer; ++q)
        if (base + q < n) s += h[base + q];
    int32_t tot;
    block_exclusive_scan32(s, sw, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_cell_scan_top(int32_t* __restrict__ sums, int nb,
                                                                int32_t* __restrict__ bstart, int n_beams)
{
    __shared__ int32_t sw[33];
    int32_t carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        const int q = base + threadIdx.x;
        const int32_t x = q < nb ? sums[q] : 0;
        int32_t tot;
        const int32_t e = block_exclusive_scan32(x, sw, &tot);
        if (q < nb) sums[q] = e + carry;
        carry += tot;
    }
    if (threadIdx.x == 0) bstart[n_beams] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_cell_scan_apply(int32_t* __restrict__ h, int64_t n,
                                                                  const int32_t* __restrict__ sums, int cells_max,
                                                                  int32_t* __restrict__ bstart)
{
    __shared__ int32_t sw[33];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    int32_t x[kScanPer];
    int32_t s = 0;
    for (int q = 0; q < kScanPer; ++q) {
        x[q] = base + q < n ? h[base + q] : 0;
        s += x[q];
    }
    int32_t tot;
    int32_t e = block_exclusive_scan32(s, sw, &tot) + sums[blockIdx.x];
    for (int q = 0; q < kScanPer; ++q) {
        const int64_t i = base + q;
        if (i < n) {
            h[i] = e;
            if (i % cells_max == 0) bstart[i / cells_max] = e;
        }
        e += x[q];
    }
}

// Pass 3 (one thread): each beam's item count, the start of its item list
// (padded to whole warps) and the total number of warp work units.
__global__ void k_bin_bases(int n_beams, const int32_t* __restrict__ bstart, int32_t* __restrict__ n_items,
                            int64_t* __restrict__ base, int32_t* __restrict__ work)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t s = 0;
    for (int b = 0; b < n_beams; ++b) {
        const int32_t nb = bstart[b + 1] - bstart[b];
        n_items[b] = nb;
        base[b] = s;
        s += ((int64_t)nb + 31) / 32 * 32;
    }
    base[n_beams] = s;
    work[0] = (int32_t)(s / 32);
}

// Pass 4: scatter voxel indices into their beam's list, grouped by cell;
// padding slots get -1.
__global__ void __launch_bounds__(256) k_bin_scatter(int64_t V, int n_beams, int cells_max,
                                                     const int32_t* __restrict__ cellof,
                                                     int32_t* __restrict__ cursor,
                                                     const int32_t* __restrict__ n_items,
                                                     const int32_t* __restrict__ bstart,
                                                     const int64_t* __restrict__ base,
                                                     int32_t* __restrict__ items)
{
    const int b = blockIdx.y;
    const int64_t b0 = base[b];
    const int lane = threadIdx.x & 31;
    // one atomic per cell and warp; the warp's voxels of a cell keep their
    // order (lane order) inside the cell's list
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); v0 < V; v0 += step) {
        const int64_t v = v0 + lane;
        const int cell = v < V ? cellof[(size_t)b * V + v] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, cell);
        const int leader = __ffs(peers) - 1;
        int first = 0;
        if (cell >= 0 && lane == leader) first = atomicAdd(cursor + (size_t)b * cells_max + cell, __popc(peers));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (cell >= 0) {
            const int pos = first + __popc(peers & ((1u << lane) - 1u)) - bstart[b];
            items[b0 + pos] = (int32_t)v;
        }
    }
    const int64_t n = n_items[b], pad_end = base[b + 1];
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b0 + n + t < pad_end) items[b0 + n + t] = -1;
}

}  // namespace

cudaError_t launch_binning(const dc_plan* p)
{
    const PlanView P = p->view();
    cudaError_t e = cudaMemsetAsync(p->d_hist, 0, sizeof(int32_t) * (size_t)p->n_beams * p->cells_max, p->stream);
    if (e != cudaSuccess) return e;
    dim3 gb((p->tiles_max + kBoundsWarps - 1) / kBoundsWarps, p->n_beams);
    k_bev_bounds<<<gb, 32 * kBoundsWarps, 0, p->stream>>>(p->d_bin, p->n_beams, p->d_beams, p->d_lio, p->bx,
                                                          p->by, p->d_bounds, p->tiles_max);
    int gx = (int)std::min<int64_t>((p->V + 255) / 256, 2048);
    dim3 gv(gx, p->n_beams);
    k_bin_hist<<<gv, 256, 0, p->stream>>>(P, p->d_bin, p->d_bounds, p->tiles_max, p->cells_max, p->d_cellof,
                                          p->d_hist);
    const int64_t ncell = (int64_t)p->n_beams * p->cells_max;
    const int nchunk = (int)((ncell + kScanChunk - 1) / kScanChunk);
    k_cell_scan_sums<<<nchunk, kScanThreads, 0, p->stream>>>(p->d_hist, ncell, p->d_bscan);
    k_cell_scan_top<<<1, kScanThreads, 0, p->stream>>>(p->d_bscan, nchunk, p->d_bstart, p->n_beams);
    k_cell_scan_apply<<<nchunk, kScanThreads, 0, p->stream>>>(p->d_hist, ncell, p->d_bscan, p->cells_max,
                                                              p->d_bstart);
    k_bin_bases<<<1, 32, 0, p->stream>>>(p->n_beams, p->d_bstart, p->d_nitems, p->d_base, p->d_work);
    k_bin_scatter<<<gv, 256, 0, p->stream>>>(p->V, p->n_beams, p->cells_max, p->d_cellof, p->d_hist,
                                             p->d_nitems, p->d_bstart, p->d_base, p->d_items);
    count_launches(7);
    return cudaGetLastError();
}

}  // namespace dc
