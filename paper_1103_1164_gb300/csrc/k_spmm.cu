// Multi-fluence dose as a block-sparse BF16 tensor-core SpMM:
//   Y[v][q] = sum_i M[v][i] F[i][q]     (eq. 1 for k fluence vectors at once)
// with M the dose-deposition matrix (M[v][i] = D_i(r_v), BF16) and FP32
// accumulation in tensor memory.
//
// Storage.  Each beam's voxel list (k_bin.cu: voxels grouped by their cell in
// the beam's eye view) is cut into row-blocks of 128 voxels.  The beam's
// beamlets are numbered as tile columns in 4 x 4 patches (patch_col below), and
// a row-block's nonzeros are covered by K-chunks of 16 tile columns: one per
// patch that holds a pair of the row-block.  Every chunk is a dense 128 x 16
// BF16 tile stored in the UMMA "no swizzle" K-major core-matrix layout
// (8 x 8 cores of 128 contiguous bytes; core (m/8, k/8) at ((m/8) * 2 + k/8) * 128),
// so one 4 KB bulk copy puts it in shared memory ready for tcgen05.mma.  The
// tiles are written by the pair kernels straight from the pair evaluation
// (k_dose.cu: k_mark_patches, k_tile_fill).  The fluence matrix is converted
// per call into the matching K-major layout of 16 x 64 tiles, contiguous for
// every 8-aligned chunk start.
//
// Kernel.  One CTA (4 warps) per row-block at a time: thread 0 streams the
// chunks' A and F tiles through a ring of shared-memory stages with
// cp.async.bulk (completion on mbarriers) and issues one
// tcgen05.mma.kind::f16 (M = 128, N = 64, K = 16) per chunk into a 64-column
// FP32 accumulator in tensor memory; after a tcgen05.commit the four warps
// read their 32 rows back with tcgen05.ld and write them out.  Every wait is
// bounded; a wait that gives up sets an error word and the CTA stops.
// Per-beam partial results are combined with compensated (Neumaier) sums.
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "dc_internal.cuh"

namespace dc {
namespace {

constexpr int kRB = 128;             // rows (voxels) per row-block
constexpr int kKC = 16;              // beamlets per K-chunk
constexpr int kN = 64;               // fluence columns of the MMA
constexpr int kTileA = kRB * kKC * 2;     // 4096 bytes
constexpr int kTileB = kKC * kN * 2;      // 2048 bytes
constexpr int kStages = 3;
constexpr int kAcc = 1;                       // accumulators in tensor memory (kN columns each)
constexpr int kMaxCtasPerSm = 512 / (kAcc * kN);   // tensor memory holds 512 columns per SM
constexpr int kEpiWarps = 4;                  // epilogue warps (one per 32 accumulator rows)
constexpr int kSpmmThreads = 32 * (kEpiWarps + 2);
constexpr long long kSpinLimit = 1ll << 26;   // bounded mbarrier waits ...
constexpr uint64_t kWaitNs = 2000000000ull;   // ... of at most 2 s

// ---------------------------------------------------------------------------
// Small PTX helpers (sm_100 family).

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the given phase of an mbarrier; false if the wait gave up (after
// kWaitNs nanoseconds or kSpinLimit polls, whichever comes first).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase)
{
    const uint64_t t0 = global_ns();
    for (long long it = 0; it < kSpinLimit; ++it) {
        if (mbar_try_wait(bar, phase)) return true;
        if ((it & 255) == 255 && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// UMMA shared-memory matrix descriptor, no swizzle, K-major.
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((smem_u32(p) >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the sm_100 family
    return d;                 // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of tcgen05.mma.kind::f16: D FP32, A and B BF16,
// both K-major, N = kN, M = kRB.
__host__ __device__ constexpr uint32_t instr_desc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(kRB >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(instr_desc()), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

constexpr int kMaxKB = 4096;   // k-blocks of one beam (32768 tile columns)

// Tile column order: each beam's beamlets in 4 x 4 patches of its M x N
// beamlet grid (patches row by row, then the patch's rows, then its columns);
// patch cells past the grid's edge are padding columns.  The beamlets of one
// voxel form a disc in the grid (the ROI), which these patches cover with
// fewer 16-column chunks than the grid's rows do.  The CSR matrix and the
// fluence vectors keep the beamlet order of the ABI; only the tiles and the
// packed fluences use this one.
__host__ __device__ __forceinline__ int patch_col(int n, int m, int M)
{
    return ((n >> 2) * ((M + 3) >> 2) + (m >> 2)) * 16 + ((n & 3) << 2) + (m & 3);
}
__host__ __device__ __forceinline__ int patch_cols(int M, int N) { return ((M + 3) >> 2) * ((N + 3) >> 2) * 16; }

// ---------------------------------------------------------------------------
// Chunk lists of the block-sparse matrix.  The pair kernels (k_dose.cu) set,
// per row-block, the bit of every 4 x 4 beamlet patch holding one of its
// pairs; each marked patch is one chunk (16 tile columns, two k-blocks).
// Per row-block: the chunks before each bitmap word, and the chunk count.
__global__ void __launch_bounds__(256) k_patch_cover(const uint32_t* __restrict__ marks, int words, int n_rb,
                                                     uint16_t* __restrict__ wpre, int32_t* __restrict__ nchunk)
{
    for (int rb = blockIdx.x * blockDim.x + threadIdx.x; rb < n_rb; rb += gridDim.x * blockDim.x) {
        int acc = 0;
        for (int w = 0; w < words; ++w) {
            wpre[(size_t)rb * words + w] = (uint16_t)acc;
            acc += __popc(marks[(size_t)rb * words + w]);
        }
        nchunk[rb] = acc;
    }
}

// The first k-block of every chunk (twice its patch, in the all-beams tile
// column numbering), a warp per row-block.
__global__ void __launch_bounds__(256) k_patch_list(const uint32_t* __restrict__ marks,
                                                    const uint16_t* __restrict__ wpre, int words, int n_rb,
                                                    const int32_t* __restrict__ rb_first, const int4* __restrict__ beam,
                                                    int n_beams, const int64_t* __restrict__ chunk_off,
                                                    int32_t* __restrict__ chunk_kb)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int rb = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; rb < n_rb; rb += nwarps) {
        int b = 0;
        while (b + 1 < n_beams && rb_first[b + 1] <= rb) ++b;
        const int kb0 = beam[b].w / 8;
        for (int w = lane; w < words; w += 32) {
            uint32_t m = marks[(size_t)rb * words + w];
            int64_t c = chunk_off[rb] + wpre[(size_t)rb * words + w];
            while (m) {
                const int bit = __ffs((int)m) - 1;
                m &= m - 1u;
                chunk_kb[c++] = kb0 + 2 * (32 * w + bit);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// F [B][k] (FP32, row-major) -> BF16 K-major core tiles in tile column order:
// element (tile column p, fluence n) at ((p / 8) * 8 + n / 8) * 64 + (n % 8) * 8
// + p % 8; fluence columns n >= k, padding columns and columns past the last
// beam are zero.
__device__ __forceinline__ void pack_fluence(const float* __restrict__ F, int k, int nkb,
                                             const int4* __restrict__ beam, int n_beams,
                                             __nv_bfloat16* __restrict__ Fp)
{
    const int64_t n_el = (int64_t)nkb * 8 * kN;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const int kb = (int)(e / (8 * kN));
        const int r = (int)(e % (8 * kN));
        const int nb = r / 64, n_in = (r % 64) / 8, c_in = r % 8;
        const int pc = kb * 8 + c_in, n = nb * 8 + n_in;
        float x = 0.f;
        if (n < k && pc < __ldg(&beam[n_beams].w)) {
            int b = 0;
            while (b + 1 < n_beams && __ldg(&beam[b + 1].w) <= pc) ++b;
            const int4 bm = beam[b];
            const int l = pc - bm.w, patch = l >> 4, q = l & 15, MB = (bm.y + 3) >> 2;
            const int row = (patch / MB) * 4 + (q >> 2), col = (patch % MB) * 4 + (q & 3);
            if (row < bm.z && col < bm.y) x = __ldg(F + (size_t)(bm.x + row * bm.y + col) * k + n);
        }
        Fp[e] = __float2bfloat16_rn(x);
    }
}

// ---------------------------------------------------------------------------
struct SpmmArgs {
    const uint16_t* tiles;
    const int32_t* chunk_kb;
    const int64_t* chunk_off;    // [n_rb + 1]
    const __nv_bfloat16* Fp;
    const int32_t* items;
    const int64_t* base;
    const int32_t* n_items;
    const int32_t* rb_first;
    int n_beams, n_rb, k;
    float* Y;                    // single beam: [V][k]
    float* P;                    // several beams: partial rows [item][k] per beam list position
    int direct;
    int stall;                   // test only: the producer issues no copies
    int32_t* err;
    const int32_t* zero;         // single beam: voxels in no list, whose rows are written as zeros
    int64_t n_zero;
};

// Reads 32 FP32 columns of this warp's 32 accumulator rows from tensor memory.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Warp roles: warps 0-3 drain the accumulator of a finished row-block (warp w
// owns tensor-memory lanes 32w..32w+31, i.e. rows 32w.. of the row-block),
// warp 4 (one lane) streams the A and F tiles of all the CTA's row-blocks
// through the stage ring, warp 5 (one lane) issues the MMAs.  With kAcc
// accumulators in tensor memory, the MMAs of row-block j + kAcc wait for the
// epilogue of row-block j; the loads run ahead through the ring.  One
// accumulator and a 3-stage ring per CTA let 6 CTAs share an SM (measured:
// more resident CTAs per SM shorten the call, deeper rings per CTA do not).
__global__ void __launch_bounds__(kSpmmThreads) k_spmm(const SpmmArgs a)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t full[kStages], empty[kStages], acc_full[kAcc], acc_empty[kAcc], drained;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_abort;
    __shared__ float s_epi[kEpiWarps][32 * 33];   // epilogue transpose, one 32 x 32 block per warp
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

    // stage buffers, 1 KB aligned
    uint8_t* buf = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(sm) + 1023) & ~(uintptr_t)1023);
    if (t == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int q = 0; q < kAcc; ++q) {
            mbar_init(&acc_full[q], 1);
            mbar_init(&acc_empty[q], kEpiWarps);
        }
        mbar_init(&drained, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kAcc * kN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    // the launch may overlap the pre-pass (programmatic dependent launch):
    // from here on its packed fluences and status word are needed
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == kEpiWarps) {
        // ---- producer: every chunk of every row-block of this CTA, in order.
        // The whole warp loads the chunks' k-block indices 32 at a time (and
        // the row-blocks' chunk ranges 32 row-blocks at a time), so the copies
        // are not serialised behind one dependent load each; lane 0 issues
        // the copies.
        uint32_t g = 0;
        bool ok = true;
        for (int rb0 = blockIdx.x; rb0 < a.n_rb && ok; rb0 += 32 * gridDim.x) {
            const int rbl = rb0 + lane * gridDim.x;
            const int64_t my_c0 = rbl < a.n_rb ? a.chunk_off[rbl] : 0;
            const int64_t my_c1 = rbl < a.n_rb ? a.chunk_off[rbl + 1] : 0;
            for (int j = 0; j < 32 && ok; ++j) {
                const int rb = rb0 + j * gridDim.x;
                if (rb >= a.n_rb) break;
                const int64_t ch0 = __shfl_sync(0xffffffffu, my_c0, j);
                const int64_t nch = __shfl_sync(0xffffffffu, my_c1, j) - ch0;
                // test-only stall (a.stall): no copy is issued, so the
                // consumers' bounded waits run out with nothing in flight
                for (int64_t cb = 0; cb < nch && ok && !a.stall; cb += 32) {
                    const int my_kb = cb + lane < nch ? a.chunk_kb[ch0 + cb + lane] : 0;
                    const int n_in = (int)(nch - cb < 32 ? nch - cb : 32);
                    for (int c = 0; c < n_in; ++c, ++g) {
                        const int kb = __shfl_sync(0xffffffffu, my_kb, c);
                        int lok = 1;
                        if (lane == 0) {
                            const uint32_t s = g % kStages;
                            if (g >= kStages && !mbar_wait(&empty[s], ((g / kStages) - 1) & 1)) lok = 0;
                            else if (s_abort) lok = 0;
                            if (lok) {
                                uint8_t* sa = buf + s * (kTileA + kTileB);
                                mbar_expect_tx(&full[s], kTileA + kTileB);
                                bulk_g2s(sa, a.tiles + (size_t)(ch0 + cb + c) * (kRB * kKC), kTileA, &full[s]);
                                bulk_g2s(sa + kTileA, a.Fp + (size_t)kb * (8 * kN), kTileB, &full[s]);
                            }
                        }
                        if (__shfl_sync(0xffffffffu, lok, 0) == 0) {
                            ok = false;
                            break;
                        }
                    }
                }
            }
        }
        if (lane == 0) {
            if (!ok) {
                s_abort = 1;
                atomicExch(a.err, 1);
            }
            // nothing may be in flight when the CTA releases its shared memory:
            // wait (bounded) until the MMA warp has consumed, or the copies
            // have landed in, every issued stage
            for (uint32_t q = g > kStages ? g - kStages : 0; q < g; ++q)
                if (!mbar_wait(&full[q % kStages], (q / kStages) & 1)) break;
        }
    } else if (warp == kEpiWarps + 1) {
        // ---- MMA issuer
        if (lane == 0) {
            uint32_t g = 0, j = 0;
            bool ok = true;
            for (int rb = blockIdx.x; rb < a.n_rb && ok; rb += gridDim.x, ++j) {
                const int64_t nch = a.chunk_off[rb + 1] - a.chunk_off[rb];
                const uint32_t ab = j % kAcc;
                // the epilogue of row-block j - kAcc has read this accumulator
                if (j >= kAcc && !mbar_wait(&acc_empty[ab], ((j / kAcc) - 1) & 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                for (int64_t c = 0; c < nch; ++c, ++g) {
                    const uint32_t s = g % kStages;
                    if (!mbar_wait(&full[s], (g / kStages) & 1) || s_abort) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    uint8_t* sa = buf + s * (kTileA + kTileB);
                    const uint64_t da = smem_desc(sa, 128, 256);            // A: LBO along K, SBO along M
                    const uint64_t db = smem_desc(sa + kTileA, 1024, 128);  // B: LBO along K, SBO along N
                    umma_bf16(tmem + ab * kN, da, db, c > 0 ? 1u : 0u);
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&acc_full[ab]);   // arrives when this row-block's MMAs are complete
            }
            if (!ok) {
                s_abort = 1;
                atomicExch(a.err, 1);
                // no MMA may still write tensor memory when the CTA frees it:
                // one more commit arrives once every MMA this thread issued
                // has completed (at once if there is none); wait for it, bounded
                umma_commit(&drained);
                mbar_wait(&drained, 0);
            }
        }
    } else {
        // ---- epilogue (warps 0-3)
        // first, while the first accumulator fills: the rows of voxels in no
        // beam list (one-beam plans), which no row-block writes
        // (a warp per row: consecutive lanes write consecutive columns)
        for (int64_t z = blockIdx.x * (int64_t)kEpiWarps + warp; z < a.n_zero; z += (int64_t)gridDim.x * kEpiWarps) {
            float* out = a.Y + (size_t)__ldg(a.zero + z) * a.k;
            for (int q = lane; q < a.k; q += 32) out[q] = 0.f;
        }
        uint32_t j = 0;
        for (int rb = blockIdx.x; rb < a.n_rb; rb += gridDim.x, ++j) {
            // the row-block's metadata and output row are looked up before
            // waiting for its accumulator, so the loads overlap the MMAs
            const int64_t nch = a.chunk_off[rb + 1] - a.chunk_off[rb];
            int b = 0;
            while (b + 1 < a.n_beams && a.rb_first[b + 1] <= rb) ++b;
            const int e = (rb - a.rb_first[b]) * kRB + t;
            // every listed row is written (zeros for a row-block without
            // chunks), so the per-beam partial rows never hold stale values
            float* out = nullptr;
            if (e < a.n_items[b]) {
                if (a.direct) {
                    const int v = a.items[a.base[b] + e];
                    out = a.Y + (size_t)v * a.k;
                } else {
                    out = a.P + (size_t)(a.base[b] + e) * a.k;
                }
            }
            const uint32_t ab = j % kAcc;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(&acc_full[ab], (j / kAcc) & 1) && !s_abort;
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                if (lane == 0) {
                    s_abort = 1;
                    atomicExch(a.err, 1);
                }
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + ab * kN;
#pragma unroll 1
            for (int h = 0; h < kN; h += 32) {
                uint32_t r[32];
                if (nch > 0) {
                    tmem_ld32(taddr + h, r);
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q) r[q] = 0u;
                }
                if (h + 32 == kN) {
                    // the accumulator is free once the last columns are in registers
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    __syncwarp();
                    if (lane == 0)
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[ab]))
                                     : "memory");
                }
                // through shared memory, so that each store writes one row's 32
                // consecutive columns (128 contiguous bytes) instead of 16 bytes
                // of 32 different rows: lane l holds row l; row stride 33 words
                // keeps both the writes and the reads free of bank conflicts
                float* sw = s_epi[warp];
#pragma unroll
                for (int q = 0; q < 32; ++q) sw[lane * 33 + q] = __uint_as_float(r[q]);
                __syncwarp();
                const bool col_ok = h + lane < a.k;
#pragma unroll 4
                for (int row = 0; row < 32; ++row) {
                    float* o = reinterpret_cast<float*>(__shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(out), row));
                    if (o && col_ok) o[h + lane] = sw[row * 33 + lane];
                }
                __syncwarp();
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAcc * kN));
}

// Y[v][q] = sum over beams of the partial rows, in beam order, with
// Neumaier-compensated summation.  A warp per voxel: the lanes find the
// voxel's list positions of all beams at once, then add the partial rows
// column by column (lane l: columns 2l, 2l + 1), so the row reads are whole
// lines.  (One thread per output element, each looking up the positions
// itself, took 9.5 ms on a 12.6 M-voxel, 9-beam plan at k = 64.)
__device__ __forceinline__ void neumaier_add(float& s, float& c, float x)
{
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

__global__ void __launch_bounds__(256) k_spmm_reduce(const float* __restrict__ P, const int32_t* __restrict__ inv,
                                                     int n_beams, int64_t V, int k, float* __restrict__ Y)
{
    const int lane = threadIdx.x & 31, q = 2 * lane;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the voxel's position in each beam's list (at most 64 beams: two per
    // lane), looked up one voxel ahead so that the lookup of the next voxel
    // overlaps the sums of this one
    int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    auto lookup = [&](int64_t u, int32_t& a, int32_t& b) {
        a = u < V && lane < n_beams ? __ldg(inv + (size_t)lane * V + u) : -1;
        b = u < V && lane + 32 < n_beams ? __ldg(inv + (size_t)(lane + 32) * V + u) : -1;
    };
    int32_t na, nb;
    lookup(v, na, nb);
    for (; v < V; v += nwarps) {
        const int32_t pa = na, pb = nb;
        lookup(v + nwarps, na, nb);
        float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
#pragma unroll 4
        for (int b = 0; b < n_beams; ++b) {
            const int32_t pos = __shfl_sync(0xffffffffu, b < 32 ? pa : pb, b & 31);
            if (pos < 0) continue;
            const float* row = P + (size_t)pos * k;
            if (q < k) neumaier_add(s0, c0, __ldg(row + q));
            if (q + 1 < k) neumaier_add(s1, c1, __ldg(row + q + 1));
        }
        float* y = Y + (size_t)v * k;
        if (q < k) y[q] = s0 + c0;
        if (q + 1 < k) y[q + 1] = s1 + c1;
    }
}

// inv[b][v] = position of voxel v in beam b's list (-1 if absent).
__global__ void __launch_bounds__(256) k_inverse(const int32_t* __restrict__ items, const int64_t* __restrict__ base,
                                                 const int32_t* __restrict__ n_items, int64_t V, int32_t* __restrict__ inv)
{
    const int b = blockIdx.y;
    const int n = n_items[b];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int v = items[base[b] + e];
        if (v >= 0) inv[(size_t)b * V + v] = (int32_t)(base[b] + e);
    }
}

// Grid and dynamic shared memory of k_spmm.  Each CTA holds 2 x 64 columns of
// tensor memory, so at most 4 CTAs may be resident on an SM (512 columns): the
// shared-memory request is raised, if needed, so that a fifth cannot fit (an
// allocation beyond the SM's columns would wait for a resident CTA to finish).
// Resident CTAs per SM and the dynamic shared memory to request, per device
// (looked up on the first call on a device: the attribute queries cost more
// than the launch itself on small problems).
struct SpmmShape {
    int per_sm = 0, sms = 0;
    size_t req = 0;
};
constexpr int kShapeDevices = 64;
SpmmShape g_shape[kShapeDevices];
std::mutex g_shape_mu;

cudaError_t spmm_device_shape(int device, size_t smem, SpmmShape* out)
{
    int smem_sm = 0, sms = 0, reserved = 0;
    cudaError_t e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, k_spmm);
    if (e != cudaSuccess) return e;
    const size_t static_smem = fa.sharedSizeBytes;
    size_t req = smem;
    const size_t min_per_cta = (size_t)smem_sm / (kMaxCtasPerSm + 1) + 1;   // one more CTA than tensor memory holds must not fit
    if (req + static_smem + (size_t)reserved < min_per_cta) req = min_per_cta - static_smem - (size_t)reserved;
    e = cudaFuncSetAttribute(k_spmm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)req);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM from the shared-memory and register budgets
    int regs_sm = 0;
    e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, device);
    if (e != cudaSuccess) return e;
    const int by_smem = smem_sm / (int)(req + static_smem + (size_t)reserved);
    const int regs_cta = ((fa.numRegs + 7) / 8 * 8) * kSpmmThreads;
    const int by_regs = regs_cta > 0 ? regs_sm / regs_cta : 4;
    int per_sm = by_smem < by_regs ? by_smem : by_regs;
    per_sm = per_sm < 1 ? 1 : (per_sm > kMaxCtasPerSm ? kMaxCtasPerSm : per_sm);
    out->per_sm = per_sm;
    out->sms = sms;
    out->req = req;
    return cudaSuccess;
}

cudaError_t spmm_launch_shape(int device, size_t smem, int n_rb, int64_t n_zero, int* grid, size_t* smem_req)
{
    if (device < 0 || device >= kShapeDevices) return cudaErrorInvalidDevice;
    SpmmShape sh;
    {
        std::lock_guard<std::mutex> lock(g_shape_mu);
        sh = g_shape[device];
    }
    if (sh.per_sm == 0) {
        cudaError_t e = spmm_device_shape(device, smem, &sh);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(g_shape_mu);
        g_shape[device] = sh;
    }
    // enough CTAs for the row-blocks, and for the zero rows (one per epilogue warp and pass)
    const int64_t need = std::max<int64_t>(n_rb, (n_zero + kEpiWarps - 1) / kEpiWarps);
    const int g = sh.sms * sh.per_sm;
    *grid = (int)(g > need ? need : g);
    *smem_req = sh.req;
    return cudaSuccess;
}

// zero[] = the voxels that no beam list holds (inv[v] < 0), in any order.
__global__ void __launch_bounds__(256) k_unlisted(const int32_t* __restrict__ inv, int64_t V,
                                                  int32_t* __restrict__ zero, unsigned long long* __restrict__ n)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
        if (inv[v] < 0) zero[atomicAdd(n, 1ull)] = (int32_t)v;
}

// The work of one call before k_spmm: the packed fluences and the
// bounded-wait status word cleared.  k_spmm may start (its set-up) as soon as
// every CTA of this grid has begun; it waits for this grid's completion before
// it reads the packed fluences.
__global__ void __launch_bounds__(256) k_spmm_pre(const float* __restrict__ F, int k, int nkb,
                                                  const int4* __restrict__ beam, int n_beams,
                                                  __nv_bfloat16* __restrict__ Fp, int32_t* __restrict__ err)
{
    asm volatile("griddepcontrol.launch_dependents;");
    if (blockIdx.x == 0 && threadIdx.x == 0) *err = 0;
    pack_fluence(F, k, nkb, beam, n_beams, Fp);
}

// k_spmm on `stream`, allowed to overlap the tail of the preceding kernel
// (k_spmm_pre) through programmatic dependent launch.
cudaError_t launch_spmm(const SpmmArgs& a, int grid, size_t smem, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kSpmmThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_spmm, a);
}

int gsize(int64_t n)
{
    int64_t g = (n + 255) / 256;
    return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side

// Buffer slot `slot` of the plan's block-sparse storage with at least `bytes`
// (reused when it is large enough, else freed and allocated again).
template <typename T>
cudaError_t sp_buffer(dc_plan* p, int slot, T*& ptr, size_t bytes)
{
    if (ptr && p->sp_cap[slot] >= bytes) return cudaSuccess;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    p->sp_cap[slot] = 0;
    const cudaError_t e = dc::dev_malloc(&ptr, bytes);
    if (e == cudaSuccess) p->sp_cap[slot] = bytes;
    return e;
}

dc_status spmm_prepare(dc_plan* p)
{
    const int nb = p->n_beams;
    std::vector<int32_t> n_items(nb);
    DC_CUDA(cudaMemcpyAsync(n_items.data(), p->d_nitems, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, p->stream));
    DC_CUDA(cudaStreamSynchronize(p->stream));
    std::vector<int32_t> rb_first(nb + 1);
    std::vector<int4> beam(nb + 1);
    int n_rb = 0, cols_total = 0;
    for (int b = 0; b < nb; ++b) {
        rb_first[b] = n_rb;
        n_rb += (n_items[b] + kRB - 1) / kRB;
        const int M = p->M[b], N = p->N[b];
        if (patch_cols(M, N) / 8 > kMaxKB) {
            set_error("spmm: a beam has more than 32768 beamlets (4 x 4 patches included)");
            return DC_EUNSUPPORTED;
        }
        beam[b] = make_int4(p->first[b], M, N, cols_total);
        cols_total += patch_cols(M, N);
    }
    rb_first[nb] = n_rb;
    beam[nb] = make_int4(p->B, 0, 0, cols_total);
    p->spmm_invalidate();
    p->sp_n_rb = n_rb;
    DC_CUDA(sp_buffer(p, 0, p->d_sp_rbfirst, (nb + 1) * sizeof(int32_t)));
    DC_CUDA(sp_buffer(p, 1, p->d_sp_first, (nb + 1) * sizeof(int4)));
    p->sp_cols = cols_total;
    DC_CUDA(sp_buffer(p, 2, p->d_sp_nchunk, (size_t)(n_rb + 1) * sizeof(int32_t)));
    DC_CUDA(sp_buffer(p, 3, p->d_sp_off, (size_t)(n_rb + 1) * sizeof(int64_t)));
    DC_CUDA(cudaMemcpyAsync(p->d_sp_rbfirst, rb_first.data(), (nb + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                            p->stream));
    DC_CUDA(cudaMemcpyAsync(p->d_sp_first, beam.data(), (nb + 1) * sizeof(int4), cudaMemcpyHostToDevice,
                            p->stream));
    // the chunks of each row-block: the 4 x 4 patches holding one of its pairs
    int max_patch = 0;
    for (int b = 0; b < nb; ++b) max_patch = std::max(max_patch, patch_cols(p->M[b], p->N[b]) / 16);
    const int words = (max_patch + 31) / 32;
    const size_t nmark = (size_t)std::max(n_rb, 1) * words;
    DC_CUDA(sp_buffer(p, 8, p->d_sp_marks, nmark * sizeof(uint32_t)));
    DC_CUDA(sp_buffer(p, 9, p->d_sp_wpre, nmark * sizeof(uint16_t)));
    DC_CUDA(cudaMemsetAsync(p->d_sp_marks, 0, nmark * sizeof(uint32_t), p->stream));
    PatchTiles pt{p->d_sp_marks, p->d_sp_wpre, p->d_sp_rbfirst, p->d_sp_off, nullptr, words};
    if (n_rb > 0) {
        DC_CUDA(launch_mark_patches(p, pt));
        k_patch_cover<<<gsize(n_rb), 256, 0, p->stream>>>(p->d_sp_marks, words, n_rb, p->d_sp_wpre,
                                                           p->d_sp_nchunk);
        count_launches(1);
        DC_CUDA(cudaGetLastError());
    }
    std::vector<int32_t> nch(n_rb + 1, 0);
    std::vector<int64_t> off(n_rb + 1, 0);
    if (n_rb > 0)
        DC_CUDA(cudaMemcpyAsync(nch.data(), p->d_sp_nchunk, n_rb * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                p->stream));
    DC_CUDA(cudaStreamSynchronize(p->stream));
    for (int r = 0; r < n_rb; ++r) off[r + 1] = off[r] + nch[r];
    p->sp_chunks = off[n_rb];
    DC_CUDA(cudaMemcpyAsync(p->d_sp_off, off.data(), (n_rb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                            p->stream));
    DC_CUDA(sp_buffer(p, 4, p->d_sp_kb, (size_t)(p->sp_chunks + 1) * sizeof(int32_t)));
    DC_CUDA(sp_buffer(p, 5, p->d_sp_tiles, (size_t)(p->sp_chunks + 1) * kTileA));
    if (n_rb > 0) {
        k_patch_list<<<gsize((int64_t)n_rb * 32), 256, 0, p->stream>>>(p->d_sp_marks, p->d_sp_wpre, words, n_rb,
                                                                        p->d_sp_rbfirst, p->d_sp_first, nb,
                                                                        p->d_sp_off, p->d_sp_kb);
        count_launches(1);
        DC_CUDA(cudaGetLastError());
        DC_CUDA(cudaMemsetAsync(p->d_sp_tiles, 0, (size_t)p->sp_chunks * kTileA, p->stream));
        pt.tiles = reinterpret_cast<uint16_t*>(p->d_sp_tiles);
        DC_CUDA(launch_tile_fill(p, pt));
    }
    {
        // inverse of the beam lists (the reduction of several beams' partial
        // rows reads it; one-beam plans keep only the voxels in no list)
        DC_CUDA(sp_buffer(p, 6, p->d_sp_inv, (size_t)nb * p->V * sizeof(int32_t)));
        DC_CUDA(cudaMemsetAsync(p->d_sp_inv, 0xff, (size_t)nb * p->V * sizeof(int32_t), p->stream));
        int maxn = 0;
        for (int b = 0; b < nb; ++b) maxn = std::max(maxn, n_items[b]);
        dim3 g(gsize(maxn), nb);
        k_inverse<<<g, 256, 0, p->stream>>>(p->d_items, p->d_base, p->d_nitems, p->V, p->d_sp_inv);
        count_launches(1);
        DC_CUDA(cudaGetLastError());
        int64_t items_total = 0;
        for (int b = 0; b < nb; ++b) items_total += ((int64_t)n_items[b] + 31) / 32 * 32;
        p->sp_items_total = items_total;
        if (nb == 1) {
            DC_CUDA(sp_buffer(p, 7, p->d_sp_zero, (size_t)p->V * sizeof(int32_t) + sizeof(unsigned long long)));
            unsigned long long* cnt = reinterpret_cast<unsigned long long*>(p->d_sp_zero + p->V);
            DC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), p->stream));
            k_unlisted<<<gsize(p->V), 256, 0, p->stream>>>(p->d_sp_inv, p->V, p->d_sp_zero, cnt);
            count_launches(1);
            DC_CUDA(cudaGetLastError());
            unsigned long long h = 0;
            DC_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
            DC_CUDA(cudaStreamSynchronize(p->stream));
            p->sp_n_zero = (int64_t)h;
        }
    }
    if (!p->d_err) DC_CUDA(dc::dev_malloc(&p->d_err, sizeof(int32_t)));
    DC_CUDA(cudaStreamSynchronize(p->stream));
    p->sp_ready = true;
    return DC_OK;
}

// Test hook of the bounded waits: with DC_FSPB_TEST_SPMM_STALL=1 in the
// environment, k_spmm's producer issues no copies, so every consumer wait runs
// out (after its 2 s bound) with nothing in flight and the call ends with the
// status word set (dc_fspb_device_status then returns DC_ETIMEOUT).  Read on
// every call of dc_fspb_spmm; unset, the kernel runs normally.
static int spmm_test_stall()
{
    const char* s = getenv("DC_FSPB_TEST_SPMM_STALL");
    return s && s[0] == '1' ? 1 : 0;
}

cudaError_t spmm_run(dc_plan* p, const float* F, int k, float* Y)
{
    const int nkb = (p->sp_cols + 7) / 8 + 2;
    cudaError_t e = cudaSuccess;
    if (p->sp_fp_cap < (size_t)nkb * 8 * kN) {
        if (p->d_sp_fp) cudaFree(p->d_sp_fp);
        p->d_sp_fp = nullptr;
        p->sp_fp_cap = 0;
        e = dc::dev_malloc(&p->d_sp_fp, (size_t)nkb * 8 * kN * sizeof(__nv_bfloat16));
        if (e != cudaSuccess) return e;
        p->sp_fp_cap = (size_t)nkb * 8 * kN;
    }
    const bool direct = p->n_beams == 1;
    if (!direct) {
        const size_t need = (size_t)p->sp_items_total * k;
        if (p->sp_p_cap < need) {
            if (p->d_sp_p) cudaFree(p->d_sp_p);
            p->d_sp_p = nullptr;
            p->sp_p_cap = 0;
            e = dc::dev_malloc(&p->d_sp_p, need * sizeof(float));
            if (e != cudaSuccess) return e;
            p->sp_p_cap = need;
        }
    }
    k_spmm_pre<<<gsize((int64_t)nkb * 8 * kN), 256, 0, p->stream>>>(
        F, k, nkb, p->d_sp_first, p->n_beams, reinterpret_cast<__nv_bfloat16*>(p->d_sp_fp), p->d_err);
    count_launches(1);
    SpmmArgs a{};
    a.tiles = reinterpret_cast<const uint16_t*>(p->d_sp_tiles);
    a.chunk_kb = p->d_sp_kb;
    a.chunk_off = p->d_sp_off;
    a.Fp = reinterpret_cast<const __nv_bfloat16*>(p->d_sp_fp);
    a.items = p->d_items;
    a.base = p->d_base;
    a.n_items = p->d_nitems;
    a.rb_first = p->d_sp_rbfirst;
    a.n_beams = p->n_beams;
    a.n_rb = p->sp_n_rb;
    a.k = k;
    a.Y = Y;
    a.P = p->d_sp_p;
    a.direct = direct ? 1 : 0;
    a.stall = spmm_test_stall();
    a.err = p->d_err;
    a.zero = p->d_sp_zero;
    a.n_zero = direct ? p->sp_n_zero : 0;
    const size_t smem = (size_t)kStages * (kTileA + kTileB) + 1024;
    int grid = 0;
    size_t smem_req = 0;
    e = spmm_launch_shape(p->device, smem, p->sp_n_rb, a.n_zero, &grid, &smem_req);
    if (e != cudaSuccess) return e;
    if (grid > 0) {
        e = launch_spmm(a, grid, smem_req, p->stream);
        count_launches(1);
        if (e != cudaSuccess) return e;
    }
    if (!direct) {
        k_spmm_reduce<<<gsize(p->V * 32), 256, 0, p->stream>>>(p->d_sp_p, p->d_sp_inv, p->n_beams, p->V, k, Y);
        count_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

// ---------------------------------------------------------------------------
// SpMM with its scratch in static device memory (dc_fspb_spmm_noalloc).
//
// Callers that cannot allocate: an optimiser or serving loop that has handed
// the device's free memory to its own pool (a cudaMalloc there fails or has
// to evict), and a latency-bound loop where a cudaFree would synchronise the
// whole device and stall the other streams.  For them the packed fluences and
// the per-beam partial rows live in the file-scope arrays below, whose
// addresses are looked up once per device; the call itself allocates nothing.
// The arrays are shared by every plan on the device, so two such calls in
// flight at once (two streams, two plans, two threads) race on them.
namespace {

constexpr int kStaticNkb = (DC_SPMM_STATIC_MAX_BEAMLETS + 7) / 8 + 2;
constexpr size_t kStaticFp = (size_t)kStaticNkb * 8 * kN;   // BF16 elements

// Packed fluence tiles are fully rewritten by k_spmm_pre and the partial
// rows read back are exactly those k_spmm stores, so neither needs clearing.
static __device__ __align__(256) uint16_t g_static_fp[kStaticFp];
static __device__ __align__(256) float g_static_part[DC_SPMM_STATIC_MAX_PARTIALS];

constexpr int kStaticDevices = 64;
struct StaticScratch {
    __nv_bfloat16* fp = nullptr;
    float* part = nullptr;
};
StaticScratch g_scratch[kStaticDevices];
std::mutex g_scratch_mu;

// Device addresses of the static arrays on `device`, looked up on first use
// with that device current (the caller's current device is restored).
cudaError_t static_scratch(int device, StaticScratch* out)
{
    if (device < 0 || device >= kStaticDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    StaticScratch& s = g_scratch[device];
    if (!s.fp || !s.part) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return e;
        if (cur != device) {
            e = cudaSetDevice(device);
            if (e != cudaSuccess) return e;
        }
        void* fp = nullptr;
        void* part = nullptr;
        e = cudaGetSymbolAddress(&fp, g_static_fp);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&part, g_static_part);
        if (cur != device) {
            const cudaError_t e2 = cudaSetDevice(cur);
            if (e == cudaSuccess) e = e2;
        }
        if (e != cudaSuccess) return e;
        if (!fp || !part) return cudaErrorInvalidSymbol;
        s.fp = reinterpret_cast<__nv_bfloat16*>(fp);
        s.part = reinterpret_cast<float*>(part);
    }
    *out = s;
    return cudaSuccess;
}

}  // namespace

cudaError_t spmm_run_static(dc_plan* p, const float* F, int k, float* Y)
{
    const int nkb = (p->sp_cols + 7) / 8 + 2;
    const bool direct = p->n_beams == 1;
    if (nkb > kStaticNkb) return cudaErrorInvalidValue;
    if (!direct && (size_t)p->sp_items_total * k > (size_t)DC_SPMM_STATIC_MAX_PARTIALS) return cudaErrorInvalidValue;
    StaticScratch sc;
    cudaError_t e = static_scratch(p->device, &sc);
    if (e != cudaSuccess) return e;
    // the packed fluences and the bounded-wait status word read after the call
    // (k_spmm itself writes the zero rows of voxels outside every beam list)
    k_spmm_pre<<<gsize((int64_t)nkb * 8 * kN), 256, 0, p->stream>>>(F, k, nkb, p->d_sp_first, p->n_beams, sc.fp,
                                                                    p->d_err);
    count_launches(1);
    SpmmArgs a{};
    a.tiles = reinterpret_cast<const uint16_t*>(p->d_sp_tiles);
    a.chunk_kb = p->d_sp_kb;
    a.chunk_off = p->d_sp_off;
    a.Fp = sc.fp;
    a.items = p->d_items;
    a.base = p->d_base;
    a.n_items = p->d_nitems;
    a.rb_first = p->d_sp_rbfirst;
    a.n_beams = p->n_beams;
    a.n_rb = p->sp_n_rb;
    a.k = k;
    a.Y = Y;
    a.P = sc.part;
    a.direct = direct ? 1 : 0;
    a.err = p->d_err;
    a.zero = p->d_sp_zero;
    a.n_zero = direct ? p->sp_n_zero : 0;
    const size_t smem = (size_t)kStages * (kTileA + kTileB) + 1024;
    int grid = 0;
    size_t smem_req = 0;
    e = spmm_launch_shape(p->device, smem, p->sp_n_rb, a.n_zero, &grid, &smem_req);
    if (e != cudaSuccess) return e;
    if (grid > 0) {
        e = launch_spmm(a, grid, smem_req, p->stream);
        count_launches(1);
        if (e != cudaSuccess) return e;
    }
    if (!direct) {
        k_spmm_reduce<<<gsize(p->V * 32), 256, 0, p->stream>>>(sc.part, p->d_sp_inv, p->n_beams, p->V, k, Y);
        count_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace dc
