// Training of the lateral-correction network on the tensor cores in BF16:
// forward pass, backward pass and weight gradients of
//   L = sum over samples and outputs of (y - t)^2 / (3 n)
// for x = taps - 1 (48), z1 = x W1 + b1, h1 = silu(z1) (64), z2 = h1 W2 + b2,
// h2 = silu(z2) (64), y = h2 W3 + b3 (3), with the FP32 master parameters
// rounded to BF16 for the products (FP32 accumulation), as the inference
// kernel does.  The per-CTA partial gradients (FP32) are summed in CTA order
// by the Adam kernel, so a gradient is deterministic.
//
// One CTA of four warps takes tiles of 64 samples.  Per tile, each warp runs
// 16 samples through the network and back with mma.m16n8k16 (activations and
// their gradients stay in registers, repacked from accumulator to operand
// layout); the tile's activations and gradients then go to shared memory, and
// the weight gradients W^T-products over the 64 samples are mma.m16n8k16 again
// with operands read transposed by ldmatrix: warp w owns rows 16w..16w+15 of
// dW2 and (w < 3) of dW1 for the whole run.  dW3 and the biases (few entries,
// FP32) are sums over the samples by one thread each.
#include <cuda_bf16.h>
#include <stdint.h>

#include "dc_internal.cuh"

namespace dc {
namespace {

constexpr int kT = 64;          // samples per CTA tile
constexpr int kW = 4;           // warps per CTA
constexpr int kLd = 72;         // bf16 row stride of the 64-wide tiles (conflict-free ldmatrix)
constexpr int kLdX = 56;        // bf16 row stride of the 48-wide input tile
constexpr int oW1 = 0, oB1 = 48 * 64, oW2 = oB1 + 64, oB2 = oW2 + 64 * 64, oW3 = oB2 + 64, oB3 = oW3 + 64 * 3;
constexpr int kNP = oB3 + 3;    // 7491
// small per-thread sums: dW3 (192), db1 (64), db2 (64), db3 (3)
constexpr int kSmall = 64 * 3 + 64 + 64 + 3;

__device__ __forceinline__ uint32_t pk(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float sig(float z) { return 1.0f / (1.0f + __expf(-z)); }

__device__ __forceinline__ void mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                    uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Four 8x8 BF16 matrices, transposed on the way (lane i gives the row address
// of row i % 8 of matrix i / 8).
__device__ __forceinline__ void ldsm_t4(uint32_t (&r)[4], const __nv_bfloat16* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

// B fragment (k-tile kt, n-tile nt, lane) of a K x N operand given by get(k, n).
template <typename F>
__device__ __forceinline__ uint2 bfrag(F get, int kt, int nt, int lane)
{
    const int k0 = kt * 16 + 2 * (lane & 3), n = nt * 8 + (lane >> 2);
    return make_uint2(pk(get(k0, n), get(k0 + 1, n)), pk(get(k0 + 8, n), get(k0 + 9, n)));
}

struct Smem {
    uint2 f1[3 * 8 * 32];       // W1 (K 48, N 64)
    uint2 f2[4 * 8 * 32];       // W2 (K 64, N 64)
    uint2 f3[4 * 32];           // W3 (K 64, N 3 of 8)
    uint2 g2[4 * 8 * 32];       // W2^T (K 64 = j, N 64 = k)
    uint2 g3[8 * 32];           // W3^T (K 3 of 16 = o, N 64 = j)
    float b1[64], b2[64], b3[4];
    __nv_bfloat16 x[kT * kLdX];
    __nv_bfloat16 h1[kT * kLd], h2[kT * kLd], dz1[kT * kLd], dz2[kT * kLd];
    float dy[kT * 4];
    float loss[kW];
};

__global__ void __launch_bounds__(32 * kW, 1) k_mlp_grad_bf16(const float* __restrict__ theta,
                                                              const float* __restrict__ X, const float* __restrict__ T,
                                                              int n, float inv_norm, float* __restrict__ partial,
                                                              float* __restrict__ loss_part)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem& S = *reinterpret_cast<Smem*>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gid = lane >> 2, tig = lane & 3;

    // BF16 operand fragments of the current parameters
    auto W1 = [&](int k, int j) { return __ldg(theta + oW1 + k * 64 + j); };
    auto W2 = [&](int k, int j) { return __ldg(theta + oW2 + k * 64 + j); };
    auto W3 = [&](int k, int o) { return o < 3 ? __ldg(theta + oW3 + k * 3 + o) : 0.f; };
    for (int q = tid; q < 3 * 8 * 32; q += blockDim.x) S.f1[q] = bfrag(W1, q / 256, (q / 32) % 8, q % 32);
    for (int q = tid; q < 4 * 8 * 32; q += blockDim.x) {
        S.f2[q] = bfrag(W2, q / 256, (q / 32) % 8, q % 32);
        S.g2[q] = bfrag([&](int j, int k) { return W2(k, j); }, q / 256, (q / 32) % 8, q % 32);
    }
    for (int q = tid; q < 4 * 32; q += blockDim.x) S.f3[q] = bfrag(W3, q / 32, 0, q % 32);
    for (int q = tid; q < 8 * 32; q += blockDim.x)
        S.g3[q] = bfrag([&](int o, int j) { return W3(j, o); }, 0, q / 32, q % 32);
    for (int q = tid; q < 64; q += blockDim.x) {
        S.b1[q] = __ldg(theta + oB1 + q);
        S.b2[q] = __ldg(theta + oB2 + q);
    }
    if (tid < 4) S.b3[tid] = tid < 3 ? __ldg(theta + oB3 + tid) : 0.f;
    __syncthreads();

    float gW1[8][4], gW2[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) gW1[a][b] = gW2[a][b] = 0.f;
    float small[(kSmall + 32 * kW - 1) / (32 * kW)];
#pragma unroll
    for (int q = 0; q < (kSmall + 32 * kW - 1) / (32 * kW); ++q) small[q] = 0.f;
    float lsum = 0.f;

    const int tiles = (n + kT - 1) / kT;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int s0 = tile * kT + warp * 16;        // this warp's 16 samples
        const int r0 = s0 + gid, r1 = r0 + 8;        // the two rows of this lane
        const int l0 = warp * 16 + gid, l1 = l0 + 8; // their rows in the tile
        // ---- layer 1: z1 = x W1 + b1 (x = X - 1, zero rows past n)
        float z1[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a) z1[a][0] = z1[a][1] = z1[a][2] = z1[a][3] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 3; ++kt) {
            const int c = kt * 16 + 2 * tig;
            float v[2][4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = h ? r1 : r0;
                const bool ok = r < n;
                const float* xr = X + (size_t)(ok ? r : 0) * 48;
                v[h][0] = ok ? __ldg(xr + c) - 1.f : 0.f;
                v[h][1] = ok ? __ldg(xr + c + 1) - 1.f : 0.f;
                v[h][2] = ok ? __ldg(xr + c + 8) - 1.f : 0.f;
                v[h][3] = ok ? __ldg(xr + c + 9) - 1.f : 0.f;
            }
            const uint32_t a0 = pk(v[0][0], v[0][1]), a1 = pk(v[1][0], v[1][1]);
            const uint32_t a2 = pk(v[0][2], v[0][3]), a3 = pk(v[1][2], v[1][3]);
            *reinterpret_cast<uint32_t*>(S.x + l0 * kLdX + c) = a0;
            *reinterpret_cast<uint32_t*>(S.x + l1 * kLdX + c) = a1;
            *reinterpret_cast<uint32_t*>(S.x + l0 * kLdX + c + 8) = a2;
            *reinterpret_cast<uint32_t*>(S.x + l1 * kLdX + c + 8) = a3;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint2 b = S.f1[(kt * 8 + nt) * 32 + lane];
                mma(z1[nt], a0, a1, a2, a3, b.x, b.y);
            }
        }
        // h1 = silu(z1) as the A operand of layer 2 (k-tile j = n-tiles 2j, 2j+1)
        uint32_t h[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * tig;
            z1[nt][0] += S.b1[c];
            z1[nt][1] += S.b1[c + 1];
            z1[nt][2] += S.b1[c];
            z1[nt][3] += S.b1[c + 1];
            const uint32_t u0 = pk(z1[nt][0] * sig(z1[nt][0]), z1[nt][1] * sig(z1[nt][1]));
            const uint32_t u1 = pk(z1[nt][2] * sig(z1[nt][2]), z1[nt][3] * sig(z1[nt][3]));
            h[nt >> 1][(nt & 1) * 2] = u0;
            h[nt >> 1][(nt & 1) * 2 + 1] = u1;
            *reinterpret_cast<uint32_t*>(S.h1 + l0 * kLd + c) = u0;
            *reinterpret_cast<uint32_t*>(S.h1 + l1 * kLd + c) = u1;
        }
        // ---- layer 2
        float z2[8][4];
#pragma unroll
        for (int a = 0; a < 8; ++a) z2[a][0] = z2[a][1] = z2[a][2] = z2[a][3] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint2 b = S.f2[(kt * 8 + nt) * 32 + lane];
                mma(z2[nt], h[kt][0], h[kt][1], h[kt][2], h[kt][3], b.x, b.y);
            }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * tig;
            z2[nt][0] += S.b2[c];
            z2[nt][1] += S.b2[c + 1];
            z2[nt][2] += S.b2[c];
            z2[nt][3] += S.b2[c + 1];
            const uint32_t u0 = pk(z2[nt][0] * sig(z2[nt][0]), z2[nt][1] * sig(z2[nt][1]));
            const uint32_t u1 = pk(z2[nt][2] * sig(z2[nt][2]), z2[nt][3] * sig(z2[nt][3]));
            h[nt >> 1][(nt & 1) * 2] = u0;
            h[nt >> 1][(nt & 1) * 2 + 1] = u1;
            *reinterpret_cast<uint32_t*>(S.h2 + l0 * kLd + c) = u0;
            *reinterpret_cast<uint32_t*>(S.h2 + l1 * kLd + c) = u1;
        }
        // ---- layer 3 and the loss gradient dy = 2 (y - t) / (3 n)
        float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const uint2 b = S.f3[kt * 32 + lane];
            mma(y, h[kt][0], h[kt][1], h[kt][2], h[kt][3], b.x, b.y);
        }
        float dy[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int o = 2 * tig + (q & 1), r = q < 2 ? r0 : r1, l = q < 2 ? l0 : l1;
            float d = 0.f;
            if (o < 3 && r < n) {
                const float res = y[q] + S.b3[o] - (__ldg(T + (size_t)r * 3 + o) - 1.f);
                lsum = fmaf(res, res, lsum);
                d = 2.f * res * inv_norm;
            }
            dy[q] = d;
            if (o < 4) S.dy[l * 4 + o] = d;
        }
        // ---- dz2 = (dy W3^T) silu'(z2): dy is the A operand with K = the 3 outputs
        const uint32_t da0 = pk(dy[0], dy[1]), da1 = pk(dy[2], dy[3]);
        float g[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            g[nt][0] = g[nt][1] = g[nt][2] = g[nt][3] = 0.f;
            const uint2 b = S.g3[nt * 32 + lane];
            mma(g[nt], da0, da1, 0u, 0u, b.x, b.y);
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * tig;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float s = sig(z2[nt][q]);
                g[nt][q] *= s * (1.f + z2[nt][q] * (1.f - s));
            }
            const uint32_t u0 = pk(g[nt][0], g[nt][1]), u1 = pk(g[nt][2], g[nt][3]);
            h[nt >> 1][(nt & 1) * 2] = u0;
            h[nt >> 1][(nt & 1) * 2 + 1] = u1;
            *reinterpret_cast<uint32_t*>(S.dz2 + l0 * kLd + c) = u0;
            *reinterpret_cast<uint32_t*>(S.dz2 + l1 * kLd + c) = u1;
        }
        // ---- dz1 = (dz2 W2^T) silu'(z1)
#pragma unroll
        for (int a = 0; a < 8; ++a) g[a][0] = g[a][1] = g[a][2] = g[a][3] = 0.f;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint2 b = S.g2[(kt * 8 + nt) * 32 + lane];
                mma(g[nt], h[kt][0], h[kt][1], h[kt][2], h[kt][3], b.x, b.y);
            }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * tig;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float s = sig(z1[nt][q]);
                g[nt][q] *= s * (1.f + z1[nt][q] * (1.f - s));
            }
            *reinterpret_cast<uint32_t*>(S.dz1 + l0 * kLd + c) = pk(g[nt][0], g[nt][1]);
            *reinterpret_cast<uint32_t*>(S.dz1 + l1 * kLd + c) = pk(g[nt][2], g[nt][3]);
        }
        __syncthreads();
        // ---- weight gradients over the tile's 64 samples (K = samples)
        // dW2[k][j] += sum_s h1[s][k] dz2[s][j]: rows k of warp w's m-tile
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const int ra = ks * 16 + ((lane >> 3) >> 1) * 8 + (lane & 7);   // sample row of A's matrix
            uint32_t a[4];
            ldsm_t4(a, S.h1 + ra * kLd + warp * 16 + ((lane >> 3) & 1) * 8);
            const int rb = ks * 16 + ((lane >> 3) & 1) * 8 + (lane & 7);    // sample row of B's matrix
#pragma unroll
            for (int np = 0; np < 4; ++np) {
                uint32_t b[4];
                ldsm_t4(b, S.dz2 + rb * kLd + np * 16 + ((lane >> 3) >> 1) * 8);
                mma(gW2[2 * np], a[0], a[1], a[2], a[3], b[0], b[1]);
                mma(gW2[2 * np + 1], a[0], a[1], a[2], a[3], b[2], b[3]);
            }
            if (warp < 3) {   // dW1[k][j] += sum_s x[s][k] dz1[s][j]
                ldsm_t4(a, S.x + ra * kLdX + warp * 16 + ((lane >> 3) & 1) * 8);
#pragma unroll
                for (int np = 0; np < 4; ++np) {
                    uint32_t b[4];
                    ldsm_t4(b, S.dz1 + rb * kLd + np * 16 + ((lane >> 3) >> 1) * 8);
                    mma(gW1[2 * np], a[0], a[1], a[2], a[3], b[0], b[1]);
                    mma(gW1[2 * np + 1], a[0], a[1], a[2], a[3], b[2], b[3]);
                }
            }
        }
        // dW3[k][o] = sum_s h2[s][k] dy[s][o]; db1, db2, db3 = column sums
#pragma unroll
        for (int q = 0; q < (kSmall + 32 * kW - 1) / (32 * kW); ++q) {
            const int e = tid + q * 32 * kW;
            if (e >= kSmall) break;
            float acc = 0.f;
            if (e < 192) {
                const int k = e / 3, o = e % 3;
                for (int s = 0; s < kT; ++s) acc = fmaf(__bfloat162float(S.h2[s * kLd + k]), S.dy[s * 4 + o], acc);
            } else if (e < 256) {
                for (int s = 0; s < kT; ++s) acc += __bfloat162float(S.dz1[s * kLd + (e - 192)]);
            } else if (e < 320) {
                for (int s = 0; s < kT; ++s) acc += __bfloat162float(S.dz2[s * kLd + (e - 256)]);
            } else {
                for (int s = 0; s < kT; ++s) acc += S.dy[s * 4 + (e - 320)];
            }
            small[q] += acc;
        }
        __syncthreads();
    }

    // ---- this CTA's partial gradient, every parameter written once
    float* P = partial + (size_t)blockIdx.x * kNP;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int j = nt * 8 + 2 * tig, k0 = warp * 16 + gid, k1 = k0 + 8;
        P[oW2 + k0 * 64 + j] = gW2[nt][0];
        P[oW2 + k0 * 64 + j + 1] = gW2[nt][1];
        P[oW2 + k1 * 64 + j] = gW2[nt][2];
        P[oW2 + k1 * 64 + j + 1] = gW2[nt][3];
        if (warp < 3) {
            P[oW1 + k0 * 64 + j] = gW1[nt][0];
            P[oW1 + k0 * 64 + j + 1] = gW1[nt][1];
            P[oW1 + k1 * 64 + j] = gW1[nt][2];
            P[oW1 + k1 * 64 + j + 1] = gW1[nt][3];
        }
    }
#pragma unroll
    for (int q = 0; q < (kSmall + 32 * kW - 1) / (32 * kW); ++q) {
        const int e = tid + q * 32 * kW;
        if (e >= kSmall) break;
        const int dst = e < 192 ? oW3 + e : (e < 256 ? oB1 + (e - 192) : (e < 320 ? oB2 + (e - 256) : oB3 + (e - 320)));
        P[dst] = small[q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) S.loss[warp] = lsum;
    __syncthreads();
    if (tid == 0) loss_part[blockIdx.x] = S.loss[0] + S.loss[1] + S.loss[2] + S.loss[3];
}

}  // namespace

cudaError_t launch_mlp_grad_bf16(cudaStream_t s, int nctas, const float* theta, const float* X, const float* T, int n,
                                 float* partial, float* loss_part)
{
    const size_t sm = sizeof(Smem);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_mlp_grad_bf16<<<nctas, 32 * kW, sm, s>>>(theta, X, T, n, 1.0f / (3.0f * (float)n), partial, loss_part);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dc
