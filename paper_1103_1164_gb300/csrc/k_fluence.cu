// Beamlet fluence from MLC leaf sequences (Section 2.3: the plans' leaf
// sequences and monitor units become a fluence map on the 0.2 x 0.5 cm
// beamlet grid, 0.2 cm along the leaf motion).
//
// For beamlet (m, n) of a beam, its rectangle [xa, xb] x [ya, yb] clipped to
// the jaws, the delivered fluence is
//   f = 1/(bx by) sum_j h_j sum_c (mu_c+1 - mu_c) [(1 - tau) (C(r) - C(l)) + tau (xb - xa)]
// with h_j the y-overlap of leaf pair j and C(z) the mean over the interval of
// clip(z(s), xa, xb) for the tip z moving linearly from z_c to z_c+1: while
// the pair's gap is (l, r), l <= r, the open length inside [xa, xb] is
// clip(r) - clip(l).  clip(z(s)) is linear between the points where z crosses
// xa and xb, so the trapezoid rule on those (at most three) pieces is exact.
//
// One thread per beamlet, one grid row per beam; the threads of a warp share
// a beamlet row, so they read the same leaf pair's positions (broadcast).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "dc_internal.cuh"

namespace dc {
namespace {

constexpr int kFluenceThreads = 128;

struct LeafBeam {
    int n_leaves, n_cp;
    int off_edges, off_mu, off_left, off_right;   // offsets into the packed data (floats)
    int M, N, first;
    float hfx, hfy;
    float x1, x2, y1, y2, tau;
};

struct LeafArgs {
    LeafBeam b[kMaxBeams];
    const float* data;
    float* out;
    float bx, by;
};

// Mean over s in [0, 1] of clip(z0 + (z1 - z0) s, a, b), a < b.
__device__ __forceinline__ float clip_mean(float z0, float z1, float a, float b)
{
    const float dz = z1 - z0;
    if (dz == 0.f) return fminf(fmaxf(z0, a), b);
    const float sa = (a - z0) / dz, sb = (b - z0) / dz;
    const float s1 = fminf(fmaxf(fminf(sa, sb), 0.f), 1.f);
    const float s2 = fminf(fmaxf(fmaxf(sa, sb), 0.f), 1.f);
    const float g0 = fminf(fmaxf(z0, a), b);
    const float g1 = fminf(fmaxf(fmaf(dz, s1, z0), a), b);
    const float g2 = fminf(fmaxf(fmaf(dz, s2, z0), a), b);
    const float g3 = fminf(fmaxf(z1, a), b);
    return 0.5f * (s1 * (g0 + g1) + (s2 - s1) * (g1 + g2) + (1.f - s2) * (g2 + g3));
}

__global__ void __launch_bounds__(kFluenceThreads) k_leaf_fluence(const __grid_constant__ LeafArgs A)
{
    const LeafBeam& L = A.b[blockIdx.y];
    const int e = blockIdx.x * kFluenceThreads + threadIdx.x;
    if (e >= L.M * L.N) return;
    const int m = e % L.M, n = e / L.M;
    const float xa0 = fmaf((float)m, A.bx, -L.hfx), ya0 = fmaf((float)n, A.by, -L.hfy);
    const float xa = fmaxf(xa0, L.x1), xb = fminf(xa0 + A.bx, L.x2);
    const float ya = fmaxf(ya0, L.y1), yb = fminf(ya0 + A.by, L.y2);
    float total = 0.f;
    if (xb > xa && yb > ya) {
        const float* E = A.data + L.off_edges;
        const float* mu = A.data + L.off_mu;
        const float* left = A.data + L.off_left;
        const float* right = A.data + L.off_right;
        const int nl = L.n_leaves;
        // first leaf pair whose band ends above ya
        int lo = 0, hi = nl;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(E + mid + 1) > ya) hi = mid;
            else lo = mid + 1;
        }
        const float open_w = 1.f - L.tau, leak = L.tau * (xb - xa);
        for (int j = lo; j < nl && __ldg(E + j) < yb; ++j) {
            const float h = fminf(yb, __ldg(E + j + 1)) - fmaxf(ya, __ldg(E + j));
            if (!(h > 0.f)) continue;
            float acc = 0.f;
            float m0 = __ldg(mu), l0 = __ldg(left + j), r0 = __ldg(right + j);
            for (int c = 1; c < L.n_cp; ++c) {
                const float m1 = __ldg(mu + c);
                const float l1 = __ldg(left + (size_t)c * nl + j), r1 = __ldg(right + (size_t)c * nl + j);
                const float dmu = m1 - m0;
                if (dmu > 0.f) {
                    const float open = clip_mean(r0, r1, xa, xb) - clip_mean(l0, l1, xa, xb);
                    acc = fmaf(dmu, fmaf(open_w, open, leak), acc);
                }
                m0 = m1;
                l0 = l1;
                r0 = r1;
            }
            total = fmaf(h, acc, total);
        }
    }
    A.out[L.first + e] = total / (A.bx * A.by);
}

dc_status leaf_invalid(const std::string& msg)
{
    set_error("dc_fluence_from_leaves: " + msg);
    return DC_EINVAL;
}

bool finite_all(const float* p, size_t n)
{
    for (size_t k = 0; k < n; ++k)
        if (!isfinite(p[k])) return false;
    return true;
}

}  // namespace
}  // namespace dc

using namespace dc;

extern "C" dc_status dc_fluence_from_leaves(dc_plan* plan, const dc_leaf_sequence* seqs, float* fluence,
                                            uint32_t flags)
{
    DC_NVTX("dc_fluence_from_leaves");
    if (!plan || !seqs || !fluence) return leaf_invalid("NULL argument");
    const int nb = plan->n_beams;
    LeafArgs A{};
    A.bx = plan->bx;
    A.by = plan->by;
    size_t total = 0;
    int max_mn = 1;
    for (int b = 0; b < nb; ++b) {
        const dc_leaf_sequence& s = seqs[b];
        const std::string at = "beam " + std::to_string(b) + ": ";
        if (s.n_leaves < 1 || s.n_cp < 1) return leaf_invalid(at + "n_leaves and n_cp must be >= 1");
        if (!s.edges || !s.mu || !s.left || !s.right) return leaf_invalid(at + "NULL array");
        const size_t nlc = (size_t)s.n_leaves * (size_t)s.n_cp;
        if (nlc > (size_t)1 << 27) return leaf_invalid(at + "sequence too large");
        if (!finite_all(s.edges, s.n_leaves + 1) || !finite_all(s.mu, s.n_cp) || !finite_all(s.left, nlc) ||
            !finite_all(s.right, nlc))
            return leaf_invalid(at + "non-finite value");
        for (int j = 0; j < s.n_leaves; ++j)
            if (!(s.edges[j + 1] > s.edges[j])) return leaf_invalid(at + "leaf edges must increase");
        for (int c = 1; c < s.n_cp; ++c)
            if (s.mu[c] < s.mu[c - 1]) return leaf_invalid(at + "meterset must not decrease");
        for (size_t k = 0; k < nlc; ++k)
            if (s.left[k] > s.right[k]) return leaf_invalid(at + "left tip beyond right tip");
        if (!(s.jaw_x1 <= s.jaw_x2) || !(s.jaw_y1 <= s.jaw_y2) || !isfinite(s.jaw_x1) || !isfinite(s.jaw_x2) ||
            !isfinite(s.jaw_y1) || !isfinite(s.jaw_y2))
            return leaf_invalid(at + "bad jaws");
        if (!(s.transmission >= 0.f && s.transmission <= 1.f)) return leaf_invalid(at + "transmission not in [0, 1]");
        LeafBeam& L = A.b[b];
        L.n_leaves = s.n_leaves;
        L.n_cp = s.n_cp;
        L.off_edges = (int)total;
        L.off_mu = (int)(total + s.n_leaves + 1);
        L.off_left = L.off_mu + s.n_cp;
        L.off_right = (int)(L.off_left + nlc);
        total += (size_t)s.n_leaves + 1 + s.n_cp + 2 * nlc;
        if (total > (size_t)1 << 28) return leaf_invalid("more than 2^28 sequence values");
        L.M = plan->M[b];
        L.N = plan->N[b];
        L.first = plan->first[b];
        L.hfx = 0.5f * plan->beams[b].field_x;
        L.hfy = 0.5f * plan->beams[b].field_y;
        L.x1 = s.jaw_x1;
        L.x2 = s.jaw_x2;
        L.y1 = s.jaw_y1;
        L.y2 = s.jaw_y2;
        L.tau = s.transmission;
        max_mn = std::max(max_mn, L.M * L.N);
    }
    std::vector<float> h(total);
    for (int b = 0; b < nb; ++b) {
        const dc_leaf_sequence& s = seqs[b];
        const LeafBeam& L = A.b[b];
        const size_t nlc = (size_t)s.n_leaves * (size_t)s.n_cp;
        std::copy(s.edges, s.edges + s.n_leaves + 1, h.begin() + L.off_edges);
        std::copy(s.mu, s.mu + s.n_cp, h.begin() + L.off_mu);
        std::copy(s.left, s.left + nlc, h.begin() + L.off_left);
        std::copy(s.right, s.right + nlc, h.begin() + L.off_right);
    }
    const bool dev = (flags & DC_DEVICE_PTRS) != 0;
    const size_t need = total + (dev ? 0 : (size_t)plan->B);   // host output: staged after the data
    if (need > plan->leaf_cap) {
        if (plan->d_leaf) cudaFree(plan->d_leaf);
        plan->d_leaf = nullptr;
        plan->leaf_cap = 0;
        DC_CUDA(dc::dev_malloc(&plan->d_leaf, need * sizeof(float)));
        plan->leaf_cap = need;
    }
    // pageable source: the call returns once the data is staged for the copy
    DC_CUDA(cudaMemcpyAsync(plan->d_leaf, h.data(), total * sizeof(float), cudaMemcpyHostToDevice, plan->stream));
    A.data = plan->d_leaf;
    A.out = dev ? fluence : plan->d_leaf + total;
    const dim3 grid((max_mn + kFluenceThreads - 1) / kFluenceThreads, nb);
    k_leaf_fluence<<<grid, kFluenceThreads, 0, plan->stream>>>(A);
    count_launches(1);
    DC_CUDA(cudaGetLastError());
    if (!dev) {
        DC_CUDA(cudaMemcpyAsync(fluence, A.out, (size_t)plan->B * sizeof(float), cudaMemcpyDeviceToHost,
                                plan->stream));
        DC_CUDA(cudaStreamSynchronize(plan->stream));
    }
    return DC_OK;
}
