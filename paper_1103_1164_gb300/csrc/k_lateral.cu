// Lateral density correction per (voxel, beam) and its learned surrogate.
//
// Step 11 of Algorithm A1 widens the penumbra and re-weights the scatter term
// with the density around the dose point.  Besides the paper's rho(r) and
// rho_hat(r) (k_prep.cu), the engine offers an axis-stencil form: for voxel r
// and beam b, 16 trilinear density taps at (j - 7.5) d along each of the beam's
// axes e_x', e_y', e_z' through r, averaged per axis with normalised Gaussian
// weights; f_u2 is taken at the x and y averages (penumbra along x and along
// y), f_omega at the mean of the three.  The factors depend on (voxel, beam)
// only, so they are computed once per density for every entry of every beam's
// voxel list (k_bin.cu) and the pair kernel loads them per work unit.
//
// The surrogate replaces the 48 trilinear taps (8 loads each) by 48
// nearest-voxel taps and a 48-64-64-3 SiLU network that predicts the three
// effective densities; it runs on the tensor cores (mma.sync BF16 with FP32
// accumulation, one warp per 32 list entries).  A stencil with a density
// outside the training range falls back to the plain computation.  The
// network is trained by the FP32 forward/backward/Adam kernels at the end of
// this file, on (nearest taps, effective densities) samples produced by
// k_stencils from the plain computation.
#include <math.h>

#include "dc_internal.cuh"

namespace dc {
namespace {

constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float lut_rho(const float* f, int n, float x0, float inv_h, float x)
{
    const float s = fminf(fmaxf((x - x0) * inv_h, 0.f), (float)(n - 1));
    const int j = min((int)s, n - 2);
    const float w = s - (float)j;
    const float f0 = __ldg(f + j), f1 = __ldg(f + j + 1);
    return fmaf(w, f1 - f0, f0);
}

__device__ __forceinline__ float rho_at(const PlanView& P, int i, int j, int k)
{
    return __ldg(P.rho + ((int64_t)k * P.ny + j) * P.nx + i);
}

// Trilinear density at a point, clamp-to-edge.
__device__ float rho_trilinear(const PlanView& P, float px, float py, float pz)
{
    const int n[3] = {P.nx, P.ny, P.nz};
    const float u[3] = {(px - P.ox) * P.idx, (py - P.oy) * P.idy, (pz - P.oz) * P.idz};
    int i0[3], i1[3];
    float w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float c = fminf(fmaxf(u[a], 0.f), (float)(n[a] - 1));
        const int f = min((int)c, max(n[a] - 2, 0));
        i0[a] = f;
        i1[a] = n[a] > 1 ? f + 1 : f;
        w[a] = n[a] > 1 ? c - (float)f : 0.f;
    }
    const float c00 = fmaf(w[0], rho_at(P, i1[0], i0[1], i0[2]) - rho_at(P, i0[0], i0[1], i0[2]), rho_at(P, i0[0], i0[1], i0[2]));
    const float c10 = fmaf(w[0], rho_at(P, i1[0], i1[1], i0[2]) - rho_at(P, i0[0], i1[1], i0[2]), rho_at(P, i0[0], i1[1], i0[2]));
    const float c01 = fmaf(w[0], rho_at(P, i1[0], i0[1], i1[2]) - rho_at(P, i0[0], i0[1], i1[2]), rho_at(P, i0[0], i0[1], i1[2]));
    const float c11 = fmaf(w[0], rho_at(P, i1[0], i1[1], i1[2]) - rho_at(P, i0[0], i1[1], i1[2]), rho_at(P, i0[0], i1[1], i1[2]));
    const float c0 = fmaf(w[1], c10 - c00, c00), c1 = fmaf(w[1], c11 - c01, c01);
    return fmaf(w[2], c1 - c0, c0);
}

// Density of the voxel nearest to a point (clamp-to-edge).
__device__ __forceinline__ float rho_nearest(const PlanView& P, float px, float py, float pz)
{
    const int i = min(max((int)floorf(fmaf(px - P.ox, P.idx, 0.5f)), 0), P.nx - 1);
    const int j = min(max((int)floorf(fmaf(py - P.oy, P.idy, 0.5f)), 0), P.ny - 1);
    const int k = min(max((int)floorf(fmaf(pz - P.oz, P.idz, 0.5f)), 0), P.nz - 1);
    return rho_at(P, i, j, k);
}

__device__ __forceinline__ void voxel_centre(const PlanView& P, int64_t v, float& rx, float& ry, float& rz)
{
    // plan grids hold at most 2^31 voxels: 32-bit division
    const uint32_t u = (uint32_t)v, q = u / (uint32_t)P.nx;
    const int ix = (int)(u - q * (uint32_t)P.nx), iy = (int)(q % (uint32_t)P.ny), iz = (int)(q / (uint32_t)P.ny);
    rx = fmaf((float)ix, P.dx, P.ox);
    ry = fmaf((float)iy, P.dy, P.oy);
    rz = fmaf((float)iz, P.dz, P.oz);
}

__device__ __forceinline__ float3 beam_axis(const BeamDev& bm, int a)
{
    const float* e = a == 0 ? bm.ex : (a == 1 ? bm.ey : bm.ez);
    return make_float3(__ldg(e), __ldg(e + 1), __ldg(e + 2));
}

// Effective densities of the axis stencil: (mean of the axis averages, x, y).
__device__ float3 axis_densities(const PlanView& P, const BeamDev& bm, float rx, float ry, float rz)
{
    float avg[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float3 e = beam_axis(bm, a);
        float s = 0.f;
        for (int j = 0; j < 16; ++j) {
            const float sj = ((float)j - 7.5f) * P.d;
            s = fmaf(P.gw[j], rho_trilinear(P, fmaf(sj, e.x, rx), fmaf(sj, e.y, ry), fmaf(sj, e.z, rz)), s);
        }
        avg[a] = s;
    }
    return make_float3((avg[0] + avg[1] + avg[2]) * (1.0f / 3.0f), avg[0], avg[1]);
}

// (log2(e) f_u2(rho_x), log2(e) f_u2(rho_y), f_w1(rho_mean), f_w2(rho_mean))
__device__ __forceinline__ float4 lateral_factors(const PlanView& P, float3 eff)
{
    const float* f = P.dens;
    const int n = P.f_n;
    return make_float4(kLog2e * lut_rho(f + 1 * n, n, P.f_rho0, P.inv_drho, eff.y),
                       kLog2e * lut_rho(f + 1 * n, n, P.f_rho0, P.inv_drho, eff.z),
                       lut_rho(f + 2 * n, n, P.f_rho0, P.inv_drho, eff.x),
                       lut_rho(f + 3 * n, n, P.f_rho0, P.inv_drho, eff.x));
}

__device__ __forceinline__ int beam_of(const int64_t* base, int n_beams, int64_t e)
{
    int b = 0;
    while (b + 1 < n_beams && base[b + 1] <= e) ++b;
    return b;
}

// Plain axis-stencil factors for every list entry.
__global__ void __launch_bounds__(128) k_axis_factors(const PlanView P, const int32_t* __restrict__ items,
                                                      const int64_t* __restrict__ base, float4* __restrict__ lfac)
{
    const int64_t total = base[P.n_beams];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int v = items[e];
        if (v < 0) continue;
        const BeamDev& bm = P.beams[beam_of(base, P.n_beams, e)];
        float rx, ry, rz;
        voxel_centre(P, v, rx, ry, rz);
        lfac[e] = lateral_factors(P, axis_densities(P, bm, rx, ry, rz));
    }
}

// ---------------------------------------------------------------------------
// The network: x = taps - 1 (48), h1 = silu(x W1 + b1) (64), h2 = silu(h1 W2 + b2)
// (64), y = h2 W3 + b3 (3), effective densities = 1 + y.  Parameters packed as
// W1[48][64], b1[64], W2[64][64], b2[64], W3[64][3], b3[3] (7491 floats).

__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint2 b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

constexpr int kXs = 56;   // bf16 row stride of the staged inputs (bank-conflict free)

// One warp evaluates the network for 32 rows of inputs staged in xs (bf16,
// [32][kXs], already offset by -1).  w: packed B fragments (see pack layout in
// api.cu: layer 1 [3][8][32] uint2, layer 2 [4][8][32], layer 3 [4][1][32]),
// bias: b1[64], b2[64], b3[3].  Writes the 3 outputs of row r to ys[r * 4 + o].
__device__ void mlp_warp_bf16(const uint2* __restrict__ w, const float* __restrict__ bias,
                              const __nv_bfloat16* __restrict__ xs, float* __restrict__ ys, int lane)
{
    const int gid = lane >> 2, tig = lane & 3;
    const uint2* w1 = w;
    const uint2* w2 = w1 + 3 * 8 * 32;
    const uint2* w3 = w2 + 4 * 8 * 32;
    const float* b1 = bias;
    const float* b2 = bias + 64;
    const float* b3 = bias + 128;
    for (int mt = 0; mt < 2; ++mt) {
        const __nv_bfloat16* x0 = xs + (mt * 16 + gid) * kXs;
        const __nv_bfloat16* x1 = x0 + 8 * kXs;
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
            uint32_t a[4];
            a[0] = *reinterpret_cast<const uint32_t*>(x0 + kt * 16 + tig * 2);
            a[1] = *reinterpret_cast<const uint32_t*>(x1 + kt * 16 + tig * 2);
            a[2] = *reinterpret_cast<const uint32_t*>(x0 + kt * 16 + tig * 2 + 8);
            a[3] = *reinterpret_cast<const uint32_t*>(x1 + kt * 16 + tig * 2 + 8);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], a, w1[(kt * 8 + nt) * 32 + lane]);
        }
        // bias + SiLU, repacked as the A fragments of layer 2 (k-tile j = n-tiles 2j, 2j+1)
        uint32_t h[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int nt = 2 * j + half, c = nt * 8 + tig * 2;
                h[j][2 * half] = pack_bf16(silu(acc[nt][0] + b1[c]), silu(acc[nt][1] + b1[c + 1]));
                h[j][2 * half + 1] = pack_bf16(silu(acc[nt][2] + b1[c]), silu(acc[nt][3] + b1[c + 1]));
            }
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const uint32_t a[4] = {h[kt][0], h[kt][1], h[kt][2], h[kt][3]};
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], a, w2[(kt * 8 + nt) * 32 + lane]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int nt = 2 * j + half, c = nt * 8 + tig * 2;
                h[j][2 * half] = pack_bf16(silu(acc[nt][0] + b2[c]), silu(acc[nt][1] + b2[c + 1]));
                h[j][2 * half + 1] = pack_bf16(silu(acc[nt][2] + b2[c]), silu(acc[nt][3] + b2[c + 1]));
            }
        }
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const uint32_t a[4] = {h[kt][0], h[kt][1], h[kt][2], h[kt][3]};
            mma_bf16(o, a, w3[kt * 32 + lane]);
        }
        // output columns tig*2, tig*2+1 of rows gid and gid + 8 (only columns 0-2 exist)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c = tig * 2 + q;
            if (c < 3) {
                ys[(mt * 16 + gid) * 4 + c] = o[q] + b3[c];
                ys[(mt * 16 + gid + 8) * 4 + c] = o[2 + q] + b3[c];
            }
        }
    }
}

constexpr int kMlpWarps = 4;
constexpr int kWfragU2 = (3 * 8 + 4 * 8 + 4) * 32;   // uint2 fragments of the three layers
constexpr int kBias = 64 + 64 + 3;

// Network factors for every list entry (one warp per 32 entries of one beam).
// Entries whose stencil has a density outside [lo, hi] use the plain stencil.
__global__ void __launch_bounds__(32 * kMlpWarps) k_mlp_factors(const PlanView P, const int32_t* __restrict__ items,
                                                                const int64_t* __restrict__ base,
                                                                const uint2* __restrict__ wfrag,
                                                                const float* __restrict__ bias, float lo, float hi,
                                                                float4* __restrict__ lfac, int32_t* __restrict__ nfall)
{
    __shared__ uint2 sw[kWfragU2];
    __shared__ float sb[kBias];
    __shared__ __align__(16) __nv_bfloat16 sx[kMlpWarps][32 * kXs];
    __shared__ float sy[kMlpWarps][32 * 4];
    for (int q = threadIdx.x; q < kWfragU2; q += blockDim.x) sw[q] = wfrag[q];
    for (int q = threadIdx.x; q < kBias; q += blockDim.x) sb[q] = bias[q];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t total = base[P.n_beams];
    const int64_t units = total / 32;
    int fall = 0;
    for (int64_t u = (int64_t)blockIdx.x * kMlpWarps + warp; u < units; u += (int64_t)gridDim.x * kMlpWarps) {
        const int64_t e = u * 32 + lane;
        const int v = items[e];
        const BeamDev& bm = P.beams[beam_of(base, P.n_beams, u * 32)];
        float rx = 0.f, ry = 0.f, rz = 0.f;
        bool in_range = true;
        if (v >= 0) {
            voxel_centre(P, v, rx, ry, rz);
            for (int a = 0; a < 3; ++a) {
                const float3 ax = beam_axis(bm, a);
                for (int j = 0; j < 16; ++j) {
                    const float sj = ((float)j - 7.5f) * P.d;
                    const float r = rho_nearest(P, fmaf(sj, ax.x, rx), fmaf(sj, ax.y, ry), fmaf(sj, ax.z, rz));
                    in_range = in_range && r >= lo && r <= hi;
                    sx[warp][lane * kXs + a * 16 + j] = __float2bfloat16_rn(r - 1.0f);
                }
            }
        } else {
            for (int q = 0; q < 48; ++q) sx[warp][lane * kXs + q] = __float2bfloat16_rn(0.f);
        }
        __syncwarp();
        mlp_warp_bf16(sw, sb, sx[warp], sy[warp], lane);
        __syncwarp();
        if (v >= 0) {
            float3 eff;
            if (in_range) {
                eff = make_float3(1.0f + sy[warp][lane * 4], 1.0f + sy[warp][lane * 4 + 1], 1.0f + sy[warp][lane * 4 + 2]);
            } else {
                eff = axis_densities(P, bm, rx, ry, rz);   // outside the training range: plain form
                ++fall;
            }
            lfac[e] = lateral_factors(P, eff);
        }
        __syncwarp();
    }
    if (fall) atomicAdd(nfall, fall);
}

// Training / evaluation samples: for (voxel, beam) pairs, the 48 nearest-voxel
// taps (network input) and the plain effective densities (network target).
__global__ void __launch_bounds__(128) k_stencils(const PlanView P, const int32_t* __restrict__ vox,
                                                  const int32_t* __restrict__ beam, int n, float* __restrict__ X,
                                                  float* __restrict__ T)
{
    const int64_t V = (int64_t)P.nx * P.ny * P.nz;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        if (vox[s] < 0 || vox[s] >= V || beam[s] < 0 || beam[s] >= P.n_beams) {   // skip bad indices
            for (int q = 0; q < 48; ++q) X[(size_t)s * 48 + q] = __int_as_float(0x7fc00000);
            for (int q = 0; q < 3; ++q) T[(size_t)s * 3 + q] = __int_as_float(0x7fc00000);
            continue;
        }
        const BeamDev& bm = P.beams[beam[s]];
        float rx, ry, rz;
        voxel_centre(P, vox[s], rx, ry, rz);
        for (int a = 0; a < 3; ++a) {
            const float3 ax = beam_axis(bm, a);
            for (int j = 0; j < 16; ++j) {
                const float sj = ((float)j - 7.5f) * P.d;
                X[(size_t)s * 48 + a * 16 + j] = rho_nearest(P, fmaf(sj, ax.x, rx), fmaf(sj, ax.y, ry), fmaf(sj, ax.z, rz));
            }
        }
        const float3 t = axis_densities(P, bm, rx, ry, rz);
        T[(size_t)s * 3 + 0] = t.x;
        T[(size_t)s * 3 + 1] = t.y;
        T[(size_t)s * 3 + 2] = t.z;
    }
}

// BF16 tensor-core inference on given inputs (for measuring the network's error
// exactly as the dose path evaluates it): Y[n][3] = effective densities.
__global__ void __launch_bounds__(32 * kMlpWarps) k_mlp_predict_bf16(const float* __restrict__ X, int n,
                                                                     const uint2* __restrict__ wfrag,
                                                                     const float* __restrict__ bias,
                                                                     float* __restrict__ Y)
{
    __shared__ uint2 sw[kWfragU2];
    __shared__ float sb[kBias];
    __shared__ __align__(16) __nv_bfloat16 sx[kMlpWarps][32 * kXs];
    __shared__ float sy[kMlpWarps][32 * 4];
    for (int q = threadIdx.x; q < kWfragU2; q += blockDim.x) sw[q] = wfrag[q];
    for (int q = threadIdx.x; q < kBias; q += blockDim.x) sb[q] = bias[q];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int units = (n + 31) / 32;
    for (int u = blockIdx.x * kMlpWarps + warp; u < units; u += gridDim.x * kMlpWarps) {
        const int s = u * 32 + lane;
        for (int q = 0; q < 48; ++q)
            sx[warp][lane * kXs + q] = __float2bfloat16_rn(s < n ? X[(size_t)s * 48 + q] - 1.0f : 0.f);
        __syncwarp();
        mlp_warp_bf16(sw, sb, sx[warp], sy[warp], lane);
        __syncwarp();
        if (s < n)
            for (int o = 0; o < 3; ++o) Y[(size_t)s * 3 + o] = 1.0f + sy[warp][lane * 4 + o];
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Training in FP32: one CTA of 256 threads handles tiles of 64 samples and
// accumulates the gradient of L = sum (y - t)^2 / (3 n_batch) over its tiles in
// shared memory (every entry owned by one thread: deterministic); partial
// gradients per CTA are summed in a fixed order by k_mlp_adam.

constexpr int kTile = 64;
constexpr int kTrainThreads = 256;
constexpr int kNParam = 48 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3;   // 7491
constexpr int oW1 = 0, oB1 = 48 * 64, oW2 = oB1 + 64, oB2 = oW2 + 64 * 64, oW3 = oB2 + 64, oB3 = oW3 + 64 * 3;

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

__global__ void __launch_bounds__(kTrainThreads) k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ X,
                                                            const float* __restrict__ T, int n, float inv_norm,
                                                            float* __restrict__ partial, float* __restrict__ loss_part)
{
    extern __shared__ float sm[];
    float* W = sm;                          // kNParam
    float* G = W + kNParam;                 // kNParam
    float* xs = G + kNParam;                // [64][48]
    float* z1 = xs + kTile * 48;            // [64][64]
    float* h1 = z1 + kTile * 64;            // [64][64] (later dz1)
    float* z2 = h1 + kTile * 64;            // [64][64]
    float* h2 = z2 + kTile * 64;            // [64][64] (later dz2)
    float* dy = h2 + kTile * 64;            // [64][3]
    float* ts = dy + kTile * 4;             // [64][3]
    __shared__ float sloss[kTrainThreads];
    const int t = threadIdx.x;
    for (int q = t; q < kNParam; q += blockDim.x) {
        W[q] = theta[q];
        G[q] = 0.f;
    }
    float lacc = 0.f;
    __syncthreads();
    const int tiles = (n + kTile - 1) / kTile;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int s0 = tile * kTile, ns = min(kTile, n - s0);
        for (int q = t; q < kTile * 48; q += blockDim.x) {
            const int s = q / 48;
            xs[q] = s < ns ? X[(size_t)(s0 + s) * 48 + q % 48] - 1.0f : 0.f;
        }
        for (int q = t; q < kTile * 3; q += blockDim.x) {
            const int s = q / 3;
            ts[(q / 3) * 4 + q % 3] = s < ns ? T[(size_t)(s0 + s) * 3 + q % 3] - 1.0f : 0.f;
        }
        __syncthreads();
        for (int q = t; q < kTile * 64; q += blockDim.x) {   // layer 1
            const int s = q / 64, j = q % 64;
            float z = W[oB1 + j];
            for (int k = 0; k < 48; ++k) z = fmaf(xs[s * 48 + k], W[oW1 + k * 64 + j], z);
            z1[q] = z;
            h1[q] = z * sigm(z);
        }
        __syncthreads();
        for (int q = t; q < kTile * 64; q += blockDim.x) {   // layer 2
            const int s = q / 64, j = q % 64;
            float z = W[oB2 + j];
            for (int k = 0; k < 64; ++k) z = fmaf(h1[s * 64 + k], W[oW2 + k * 64 + j], z);
            z2[q] = z;
            h2[q] = z * sigm(z);
        }
        __syncthreads();
        for (int q = t; q < kTile * 3; q += blockDim.x) {    // layer 3 and the loss gradient
            const int s = q / 3, o = q % 3;
            float y = W[oB3 + o];
            for (int k = 0; k < 64; ++k) y = fmaf(h2[s * 64 + k], W[oW3 + k * 3 + o], y);
            const float r = s < ns ? y - ts[s * 4 + o] : 0.f;
            dy[s * 4 + o] = 2.0f * r * inv_norm;
            lacc = fmaf(r, r, lacc);
        }
        __syncthreads();
        for (int q = t; q < 64 * 3 + 3; q += blockDim.x) {   // dW3, db3
            if (q < 64 * 3) {
                const int k = q / 3, o = q % 3;
                float g = 0.f;
                for (int s = 0; s < kTile; ++s) g = fmaf(h2[s * 64 + k], dy[s * 4 + o], g);
                G[oW3 + q] += g;
            } else {
                const int o = q - 64 * 3;
                float g = 0.f;
                for (int s = 0; s < kTile; ++s) g += dy[s * 4 + o];
                G[oB3 + o] += g;
            }
        }
        __syncthreads();
        for (int q = t; q < kTile * 64; q += blockDim.x) {   // dz2 = (dy W3^T) silu'(z2), into h2
            const int s = q / 64, j = q % 64;
            const float dh = dy[s * 4 + 0] * W[oW3 + j * 3 + 0] + dy[s * 4 + 1] * W[oW3 + j * 3 + 1] +
                             dy[s * 4 + 2] * W[oW3 + j * 3 + 2];
            const float z = z2[q], sg = sigm(z);
            h2[q] = dh * sg * (1.0f + z * (1.0f - sg));
        }
        __syncthreads();
        for (int q = t; q < 64 * 64 + 64; q += blockDim.x) {  // dW2, db2
            if (q < 64 * 64) {
                const int k = q / 64, j = q % 64;
                float g = 0.f;
                for (int s = 0; s < kTile; ++s) g = fmaf(h1[s * 64 + k], h2[s * 64 + j], g);
                G[oW2 + q] += g;
            } else {
                const int j = q - 64 * 64;
                float g = 0.f;
                for (int s = 0; s < kTile; ++s) g += h2[s * 64 + j];
                G[oB2 + j] += g;
            }
        }
        __syncthreads();
        for (int q = t; q < kTile * 64; q += blockDim.x) {   // dz1 = (dz2 W2^T) silu'(z1), into h1
            const int s = q / 64, k = q % 64;
            float dh = 0.f;
            for (int j = 0; j < 64; ++j) dh = fmaf(h2[s * 64 + j], W[oW2 + k * 64 + j], dh);
            const float z = z1[q], sg = sigm(z);
            h1[q] = dh * sg * (1.0f + z * (1.0f - sg));
        }
        __syncthreads();
        for (int q = t; q < 48 * 64 + 64; q += blockDim.x) {  // dW1, db1
            if (q < 48 * 64) {
                const int k = q / 64, j = q % 64;
                float g = 0.f;
                for (int s = 0; s < kTile; ++s) g = fmaf(xs[s * 48 + k], h1[s * 64 + j], g);
                G[oW1 + q] += g;
            } else {
                const int j = q - 48 * 64;
                float g = 0.f;
                for (int s = 0; s < kTile; ++s) g += h1[s * 64 + j];
                G[oB1 + j] += g;
            }
        }
        __syncthreads();
    }
    for (int q = t; q < kNParam; q += blockDim.x) partial[(size_t)blockIdx.x * kNParam + q] = G[q];
    sloss[t] = lacc;
    __syncthreads();
    if (t == 0) {
        float s = 0.f;
        for (int q = 0; q < kTrainThreads; ++q) s += sloss[q];
        loss_part[blockIdx.x] = s;
    }
}

// Sums the per-CTA gradients in CTA order; optionally stores the gradient and
// applies one Adam step (lr > 0).
__global__ void __launch_bounds__(256) k_mlp_adam(const float* __restrict__ partial, int nparts, float* __restrict__ theta,
                                                  float* __restrict__ m1, float* __restrict__ m2, float* __restrict__ grad,
                                                  float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kNParam; q += gridDim.x * blockDim.x) {
        float g = 0.f;
        for (int c = 0; c < nparts; ++c) g += partial[(size_t)c * kNParam + q];
        if (grad) grad[q] = g;
        if (lr > 0.f) {
            const float a = fmaf(b1, m1[q], (1.f - b1) * g);
            const float b = fmaf(b2, m2[q], (1.f - b2) * g * g);
            m1[q] = a;
            m2[q] = b;
            theta[q] -= lr * (a * c1) / (sqrtf(b * c2) + eps);
        }
    }
}

}  // namespace

size_t mlp_grad_smem() { return sizeof(float) * (2 * kNParam + kTile * 48 + 4 * kTile * 64 + 2 * kTile * 4); }

cudaError_t launch_lateral(const dc_plan* p)
{
    const PlanView P = p->view();
    int64_t total = (int64_t)p->n_beams * (p->V + 32);
    int g = (int)std::min<int64_t>((total + 127) / 128, 152 * 16);
    if (p->lateral_mode == DC_LATERAL_AXIS) {
        k_axis_factors<<<g, 128, 0, p->stream>>>(P, p->d_items, p->d_base, p->d_lfac);
        count_launches(1);
    } else if (p->lateral_mode == DC_LATERAL_MLP) {
        cudaError_t e = cudaMemsetAsync(p->d_nfall, 0, sizeof(int32_t), p->stream);
        if (e != cudaSuccess) return e;
        k_mlp_factors<<<152 * 4, 32 * kMlpWarps, 0, p->stream>>>(P, p->d_items, p->d_base, p->d_mlp_frag,
                                                                 p->d_mlp_bias, p->mlp_lo, p->mlp_hi, p->d_lfac,
                                                                 p->d_nfall);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_stencils(const dc_plan* p, const int32_t* vox, const int32_t* beam, int n, float* X, float* T)
{
    k_stencils<<<std::max(1, std::min((n + 127) / 128, 152 * 8)), 128, 0, p->stream>>>(p->view(), vox, beam, n, X, T);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_predict_bf16(cudaStream_t s, const float* X, int n, const uint2* wfrag, const float* bias, float* Y)
{
    k_mlp_predict_bf16<<<std::max(1, std::min((n + 127) / 128, 152 * 8)), 32 * kMlpWarps, 0, s>>>(X, n, wfrag, bias, Y);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(cudaStream_t s, int nctas, const float* theta, const float* X, const float* T, int n,
                            float* partial, float* loss_part)
{
    const size_t sm = mlp_grad_smem();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_mlp_grad<<<nctas, kTrainThreads, sm, s>>>(theta, X, T, n, 1.0f / (3.0f * (float)n), partial, loss_part);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(cudaStream_t s, const float* partial, int nparts, float* theta, float* m1, float* m2,
                            float* grad, float lr, float b1, float b2, float eps, int step)
{
    const float c1 = 1.0f / (1.0f - powf(b1, (float)step)), c2 = 1.0f / (1.0f - powf(b2, (float)step));
    k_mlp_adam<<<(kNParam + 255) / 256, 256, 0, s>>>(partial, nparts, theta, m1, m2, grad, lr, b1, b2, eps, c1, c2);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dc
