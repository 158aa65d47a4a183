// Gamma-index comparison of two dose distributions (the 3 %-3 mm 3-D gamma
// of the paper's accuracy evaluation, Section 3 and Tables 2-3):
//   gamma(r) = min(R / dta, min over whole-voxel offsets o, |o| <= R, r + o in
//              the grid, of sqrt(|o|^2 / dta^2 + (D_eval(r + o) - D_ref(r))^2 / dD^2)),
// dD = pct / 100 * max D_ref, and its statistics (gamma_max, the mean gamma
// and the pass rate gamma < 1 inside the reference's 50 % isodose line).
//
// One thread per reference voxel walks the offsets in order of increasing
// length and stops at the first whose distance term alone is not below the
// best value so far (no later offset can do better); consecutive threads hold
// consecutive x, so each offset's evaluated doses are read coalesced.  The
// reductions (max dose, statistics) run in a fixed order, so results do not
// depend on scheduling.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "dc_internal.cuh"

namespace dc {
namespace {

constexpr int kGammaThreads = 256;
constexpr int kRedBlocks = 512;     // partials of the fixed-order reductions
constexpr int kMaxReach = 64;       // search radius in voxels along each axis

struct GammaArgs {
    const float* ref;
    const float* ev;
    float* gamma;
    int nx, ny, nz;
    const int4* off;     // (i, j, k, bits of |o|^2 / dta^2), |o| ascending
    int n_off;
    const float* dmax;   // max D_ref (device)
    float frac;          // pct / 100
    float cap2;          // (R / dta)^2
};

__global__ void __launch_bounds__(kGammaThreads) k_gamma(const GammaArgs a)
{
    const int64_t V = (int64_t)a.nx * a.ny * a.nz;
    const float dD = a.frac * __ldg(a.dmax);
    const float inv = 1.0f / (dD * dD);
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(v % a.nx), y = (int)((v / a.nx) % a.ny), z = (int)(v / ((int64_t)a.nx * a.ny));
        const float dr = __ldg(a.ref + v);
        float best = a.cap2;
        for (int q = 0; q < a.n_off; ++q) {
            const int4 o = __ldg(a.off + q);
            const float d2 = __int_as_float(o.w);
            if (d2 >= best) break;
            const int xx = x + o.x, yy = y + o.y, zz = z + o.z;
            if ((unsigned)xx >= (unsigned)a.nx || (unsigned)yy >= (unsigned)a.ny || (unsigned)zz >= (unsigned)a.nz)
                continue;
            const float diff = __ldg(a.ev + ((int64_t)zz * a.ny + yy) * a.nx + xx) - dr;
            best = fminf(best, fmaf(diff * diff, inv, d2));
        }
        a.gamma[v] = sqrtf(best);
    }
}

// Block-wide reduction in a fixed order (tree over the threads' values).
template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T x, T* sh, Op op)
{
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] = op(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const T r = sh[0];
    __syncthreads();
    return r;
}

// part[b] = max of block b's contiguous chunk of d (values >= 0).
__global__ void __launch_bounds__(kGammaThreads) k_max_part(const float* __restrict__ d, int64_t n,
                                                            float* __restrict__ part)
{
    __shared__ float sh[kGammaThreads];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    float m = 0.f;
    for (int64_t v = lo + threadIdx.x; v < hi; v += blockDim.x) m = fmaxf(m, __ldg(d + v));
    m = block_reduce(m, sh, [](float p, float q) { return fmaxf(p, q); });
    if (threadIdx.x == 0) part[blockIdx.x] = m;
}

__global__ void __launch_bounds__(kGammaThreads) k_max_final(const float* __restrict__ part, int n,
                                                             float* __restrict__ out)
{
    __shared__ float sh[kGammaThreads];
    float m = 0.f;
    for (int q = threadIdx.x; q < n; q += blockDim.x) m = fmaxf(m, part[q]);
    m = block_reduce(m, sh, [](float p, float q) { return fmaxf(p, q); });
    if (threadIdx.x == 0) *out = m;
}

// Per block: max gamma, sum of gamma, voxel count and pass count inside the
// 50 % isodose of the reference.
struct GammaPart {
    double sum50;
    long long n50, pass50;
    float gmax;
    float pad;
};

__global__ void __launch_bounds__(kGammaThreads) k_gamma_part(const float* __restrict__ g,
                                                              const float* __restrict__ ref, int64_t n,
                                                              const float* __restrict__ dmax,
                                                              GammaPart* __restrict__ part)
{
    __shared__ double shd[kGammaThreads];
    __shared__ long long shl[kGammaThreads];
    __shared__ float shf[kGammaThreads];
    const float half = 0.5f * __ldg(dmax);
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
    float gm = 0.f;
    double s = 0.0;
    long long c = 0, p = 0;
    for (int64_t v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const float gv = __ldg(g + v);
        gm = fmaxf(gm, gv);
        if (__ldg(ref + v) >= half) {
            s += (double)gv;
            ++c;
            p += gv < 1.0f ? 1 : 0;
        }
    }
    auto add_d = [](double x, double y) { return x + y; };
    auto add_l = [](long long x, long long y) { return x + y; };
    gm = block_reduce(gm, shf, [](float x, float y) { return fmaxf(x, y); });
    s = block_reduce(s, shd, add_d);
    c = block_reduce(c, shl, add_l);
    p = block_reduce(p, shl, add_l);
    if (threadIdx.x == 0) part[blockIdx.x] = GammaPart{s, c, p, gm, 0.f};
}

__global__ void __launch_bounds__(kGammaThreads) k_gamma_final(const GammaPart* __restrict__ part, int n,
                                                               GammaPart* __restrict__ out)
{
    __shared__ double shd[kGammaThreads];
    __shared__ long long shl[kGammaThreads];
    __shared__ float shf[kGammaThreads];
    float gm = 0.f;
    double s = 0.0;
    long long c = 0, p = 0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        gm = fmaxf(gm, part[q].gmax);
        s += part[q].sum50;
        c += part[q].n50;
        p += part[q].pass50;
    }
    auto add_d = [](double x, double y) { return x + y; };
    auto add_l = [](long long x, long long y) { return x + y; };
    gm = block_reduce(gm, shf, [](float x, float y) { return fmaxf(x, y); });
    s = block_reduce(s, shd, add_d);
    c = block_reduce(c, shl, add_l);
    p = block_reduce(p, shl, add_l);
    if (threadIdx.x == 0) *out = GammaPart{s, c, p, gm, 0.f};
}

int float_bits(float f)
{
    int i;
    memcpy(&i, &f, sizeof(i));
    return i;
}

// Device buffers of one call, freed on every return path.
struct GammaBuffers {
    std::vector<void*> ptrs;
    ~GammaBuffers()
    {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    cudaError_t get(T** p, size_t n)
    {
        void* q = nullptr;
        const cudaError_t e = dc::dev_malloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = reinterpret_cast<T*>(q);
        return e;
    }
};

}  // namespace
}  // namespace dc

using namespace dc;

extern "C" dc_status dc_gamma_index(const float* ref, const float* eval, const dc_grid* grid, float dose_pct,
                                    float dta_cm, float search_cm, float* gamma, dc_gamma_stats* stats,
                                    void* cuda_stream, uint32_t flags)
{
    DC_NVTX("dc_gamma_index");
    if (!ref || !eval || !grid) {
        set_error("dc_gamma_index: NULL argument");
        return DC_EINVAL;
    }
    const dc_grid g = *grid;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1 || !(g.dx > 0 && g.dy > 0 && g.dz > 0)) {
        set_error("dc_gamma_index: empty grid or non-positive voxel size");
        return DC_EINVAL;
    }
    if (!(dose_pct > 0 && dta_cm > 0 && search_cm >= dta_cm)) {
        set_error("dc_gamma_index: need dose_pct > 0, dta_cm > 0 and search_cm >= dta_cm");
        return DC_EINVAL;
    }
    const int ri = (int)floor(search_cm / g.dx + 1e-9), rj = (int)floor(search_cm / g.dy + 1e-9),
              rk = (int)floor(search_cm / g.dz + 1e-9);
    if (ri > kMaxReach || rj > kMaxReach || rk > kMaxReach) {
        set_error("dc_gamma_index: the search radius spans more than 64 voxels along an axis");
        return DC_EINVAL;
    }
    const int64_t V = (int64_t)g.nx * g.ny * g.nz;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);

    // offsets within the search sphere, by increasing length (ties in a fixed order)
    struct Off {
        double d2;
        int i, j, k;
    };
    std::vector<Off> offs;
    const double R2 = (double)search_cm * search_cm * (1 + 1e-12);
    for (int k = -rk; k <= rk; ++k)
        for (int j = -rj; j <= rj; ++j)
            for (int i = -ri; i <= ri; ++i) {
                const double d2 = (i * (double)g.dx) * (i * (double)g.dx) + (j * (double)g.dy) * (j * (double)g.dy) +
                                  (k * (double)g.dz) * (k * (double)g.dz);
                if (d2 <= R2) offs.push_back(Off{d2, i, j, k});
            }
    std::stable_sort(offs.begin(), offs.end(), [](const Off& a, const Off& b) { return a.d2 < b.d2; });
    std::vector<int4> h_off(offs.size());
    const double inv_dta2 = 1.0 / ((double)dta_cm * dta_cm);
    for (size_t q = 0; q < offs.size(); ++q) {
        const float d2 = (float)(offs[q].d2 * inv_dta2);
        h_off[q] = make_int4(offs[q].i, offs[q].j, offs[q].k, float_bits(d2));
    }

    GammaBuffers buf;
    const bool dev = (flags & DC_DEVICE_PTRS) != 0;
    const float* d_ref = ref;
    const float* d_ev = eval;
    float* d_g = dev ? gamma : nullptr;
    int4* d_off = nullptr;
    float *d_part = nullptr, *d_max = nullptr;
    GammaPart *d_gpart = nullptr, *d_gout = nullptr;
    DC_CUDA(buf.get(&d_off, h_off.size()));
    DC_CUDA(buf.get(&d_part, kRedBlocks));
    DC_CUDA(buf.get(&d_max, 1));
    DC_CUDA(buf.get(&d_gpart, kRedBlocks));
    DC_CUDA(buf.get(&d_gout, 1));
    if (!dev) {
        float *r = nullptr, *e = nullptr;
        DC_CUDA(buf.get(&r, V));
        DC_CUDA(buf.get(&e, V));
        DC_CUDA(cudaMemcpyAsync(r, ref, V * sizeof(float), cudaMemcpyHostToDevice, s));
        DC_CUDA(cudaMemcpyAsync(e, eval, V * sizeof(float), cudaMemcpyHostToDevice, s));
        d_ref = r;
        d_ev = e;
    }
    if (!d_g) DC_CUDA(buf.get(&d_g, V));
    DC_CUDA(cudaMemcpyAsync(d_off, h_off.data(), h_off.size() * sizeof(int4), cudaMemcpyHostToDevice, s));

    // max D_ref (needed for dD and the 50 % isodose), checked on the host
    k_max_part<<<kRedBlocks, kGammaThreads, 0, s>>>(d_ref, V, d_part);
    k_max_final<<<1, kGammaThreads, 0, s>>>(d_part, kRedBlocks, d_max);
    count_launches(2);
    float dmax = 0.f;
    DC_CUDA(cudaMemcpyAsync(&dmax, d_max, sizeof(float), cudaMemcpyDeviceToHost, s));
    DC_CUDA(cudaStreamSynchronize(s));
    if (!(dmax > 0.f)) {
        set_error("dc_gamma_index: the reference dose is zero everywhere");
        return DC_EINVAL;
    }

    GammaArgs a;
    a.ref = d_ref;
    a.ev = d_ev;
    a.gamma = d_g;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.off = d_off;
    a.n_off = (int)h_off.size();
    a.dmax = d_max;
    a.frac = dose_pct / 100.f;
    a.cap2 = (float)(((double)search_cm / dta_cm) * ((double)search_cm / dta_cm));
    int sms = 0, device = 0;
    DC_CUDA(cudaGetDevice(&device));
    DC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int64_t want = (V + kGammaThreads - 1) / kGammaThreads;
    const int grid_g = (int)std::min<int64_t>(want, (int64_t)sms * 16);
    k_gamma<<<grid_g, kGammaThreads, 0, s>>>(a);
    k_gamma_part<<<kRedBlocks, kGammaThreads, 0, s>>>(d_g, d_ref, V, d_max, d_gpart);
    k_gamma_final<<<1, kGammaThreads, 0, s>>>(d_gpart, kRedBlocks, d_gout);
    count_launches(3);
    DC_CUDA(cudaGetLastError());
    GammaPart h{};
    DC_CUDA(cudaMemcpyAsync(&h, d_gout, sizeof(h), cudaMemcpyDeviceToHost, s));
    if (gamma && !dev) DC_CUDA(cudaMemcpyAsync(gamma, d_g, V * sizeof(float), cudaMemcpyDeviceToHost, s));
    DC_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        stats->gamma_max = h.gmax;
        stats->n50 = h.n50;
        stats->gamma_avg50 = h.n50 > 0 ? h.sum50 / (double)h.n50 : 0.0;
        stats->pass50_pct = h.n50 > 0 ? 100.0 * (double)h.pass50 / (double)h.n50 : 0.0;
        stats->dose_max = dmax;
    }
    return DC_OK;
}
