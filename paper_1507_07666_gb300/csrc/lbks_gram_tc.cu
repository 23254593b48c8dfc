// Overlap (Gram) matrix of more than eight FP32 orbitals on the fifth-
// generation tensor cores: S = h^3 Psi Psi^T, the N_O x N_O x N contraction
// behind the normalisation sigma_j = 1/||psi_j|| and the couplings
// Lambda_jk = S_jk / S_kk of each relaxation step (Sec. 3, the normalised
// update and Eq. W) and behind the Cholesky orthonormalisation that ends a cycle.
//
// Precision.  Every FP32 orbital value x is split into bf16 parts
// hi = rn(x), lo = rn(x - hi).  A shared-memory tile of 64 sites holds hi in
// rows 0..N_O-1 and lo in rows N_O..2N_O-1, and one M = 128 tcgen05.mma with
// A = B = that tile (N = 2N_O rounded up to 16) leaves the four blocks hi.hi,
// hi.lo, lo.hi, lo.lo in TMEM; A rows past 2N_O (zeros, or the next stage's
// bytes in the compact layout of TcLayout) reach only accumulator rows that
// are never read.  Their sum is the product of the FP32 values up
// to the rounding of lo (2^-17 relative, unbiased).  TMEM accumulates in FP32
// over kDrainTiles tiles; then the four blocks are folded and added to
// per-thread FP64 sums, so no FP32 sum runs over more than 512 sites.  Blocks
// and the grid finish in FP64 (the last block of each system, fixed order).
//
// Pipeline.  256 threads (320 for 33..40 orbitals, so that every thread
// splits two 4-site groups of a tile) stream the next tiles into a cp.async
// ring (or registers) while they split the current ones into 128-byte-
// swizzled K-major tiles: one tile per block barrier into two stages, or, for
// 33..40 orbitals, two tiles per barrier into four.  After each barrier one
// thread issues the tiles' K = 16 MMAs (four per tile) and commits each tile
// to its stage's mbarrier; warps 0..7 drain TMEM (warp w reads lanes
// 32 (w % 4) .. 32 (w % 4) + 31).  Every wait on an
// mbarrier is bounded (lbks_set_wait_limit polls, default 2^22): on expiry the
// block records a timeout, writes NaN partial sums (so the solve fails with a
// non-finite energy), waits (2^22 polls at most) for its own MMAs, frees its
// TMEM and returns.
#include "lbks_internal.cuh"
#include "lbks_reduce.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>

namespace lbks {
namespace {

constexpr int kTcThreads = 256;                              // 8 warps (the default block)
constexpr int kTcSites = 64;                                 // sites per tile: 64 bf16 = one 128-byte row
constexpr int kTcRows = 128;                                 // MMA M
constexpr int kTcStages = 2;                                 // bf16 stages per tile of a barrier (below)
constexpr int kTcTileBytes = kTcRows * kTcSites * 2;         // 16 KB
// Per-thread work bounds for at most MAXO orbitals: 4-site groups of a tile,
// and overlap pairs of the packed lower triangle.
template <int MAXO, int TH>
struct TcBounds {
    static constexpr int quads = (MAXO * (kTcSites / 4) + TH - 1) / TH;
    static constexpr int pairs = (MAXO * (MAXO + 1) / 2 + TH - 1) / TH;
};
constexpr int kDrainTiles = 8;
constexpr int kInStages = 4;                                 // staged FP32 tiles in flight (bulk-copy path)
// Shared-memory layout for at most MAXO orbitals and TPB tiles split between
// two block barriers (2 TPB bf16 stages).  TPB = 1: 128-row stages, the FP32
// fold buffer after the cp.async ring.  TPB > 1: a stage holds only the
// 2 MAXO rows in use (stride bytes apart, whole 1 KB swizzle groups) -- the
// M = 128 MMA reads 128 rows from a stage's start, and the rows past 2 MAXO
// (the next stage, or the slack after the last one) feed only accumulator
// rows that are never read -- and the fold buffer shares the stages' bytes
// where it fits (it is written only while no MMA is in flight).
template <int MAXO, int TPB>
struct TcLayout {
    static constexpr int stages = kTcStages * TPB;
    static constexpr int stride = TPB > 1 ? ((2 * MAXO * 128 + 1023) / 1024) * 1024 : kTcTileBytes;
    static constexpr int tiles = stages * stride + (kTcTileBytes - stride);
    static constexpr bool fold_in_tiles = TPB > 1 && 2 * MAXO * (2 * MAXO + 1) * 4 <= tiles;
};
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr int kTmemColumnsPerSm = 512;

__device__ unsigned g_tc_timeouts;
// Polls of the main mbarrier waits, read at each launch (a test can lower it
// to make the waits give up; the wait for the block's own MMAs after a
// failure keeps kWaitLimit).
std::atomic<uint32_t> g_wait_limit{kWaitLimit};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, groups of 8 rows 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu)   // start address
           | ((uint64_t)1 << 16)                // leading-dimension offset (unused with this swizzle)
           | ((uint64_t)(1024 >> 4) << 32)      // stride between 8-row groups
           | ((uint64_t)1 << 46)                // descriptor version
           | ((uint64_t)2 << 61);               // 128-byte swizzle
}

// Instruction descriptor, kind::f16: bf16 A and B, both K-major; FP32 D; M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row r, site k) in a swizzled tile: 16-byte chunk
// index XOR (row mod 8), the pattern the descriptor's swizzle mode reads.
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + (((k >> 3) ^ (r & 7)) << 4) + (k & 7) * 2);
}

// Each poll may suspend the thread until the phase completes, for at most
// kPollSuspendNs (so that waiting warps issue few instructions).
constexpr uint32_t kPollSuspendNs = 1000;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity), "n"(kPollSuspendNs)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
        :
        : "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 lanes x 16 consecutive 32-bit TMEM columns, one lane per thread of the warp.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }

}  // namespace

// 16-byte asynchronous copy global -> shared (zero-filled when src_bytes = 0).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One block per group of tiles of one system (system = blockIdx.y); tile i of
// the block is global tile blockIdx.x + i * gridDim.x.
//
// BULK (N % 4 == 0, 16-byte aligned orbitals): every thread streams its 16-byte
// pieces of the tiles kInStages - 1 ahead into a staging ring with cp.async,
// so the loads in flight do not depend on registers; a thread's ring pieces
// are its own (one block barrier per tile, before the MMAs).  Otherwise every thread
// loads its values for the next tile into registers while it converts the
// current one.
//
// TPB tiles are split between two block barriers, and one thread issues their
// MMAs together.
//
// Dynamic shared memory (TcLayout): 1 KB alignment slack, the bf16 stages,
// the staging ring (BULK), the (2N_O) x (2N_O + 1) FP32 fold buffer unless it
// shares the stages' bytes (reused for the block totals).
template <bool LAM, bool BULK, int MAXO, int TH, int TPB>
__global__ void __launch_bounds__(TH, 2)
    k_gram_tc(Grid g, double h, const float* __restrict__ psi, int NO, int drain_tiles, double* S, double* lam,
              double* sigma, Scratch sc, uint32_t wait_limit) {
    if (inactive(g)) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    using L = TcLayout<MAXO, TPB>;
    constexpr int NS = L::stages;
    const uint32_t stage_bytes = (uint32_t)NO * kTcSites * 4;  // one staged FP32 tile
    unsigned char* ring = smem + L::tiles;
    float* fold = reinterpret_cast<float*>(L::fold_in_tiles ? smem : ring + (BULK ? kInStages * stage_bytes : 0));
    __shared__ __align__(8) uint64_t mbar[NS];
    __shared__ uint32_t tmem_sh;

    constexpr int kTcQuads = TcBounds<MAXO, TH>::quads, kTcMaxPairs = TcBounds<MAXO, TH>::pairs;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int lane_base = (warp & 3) * 32, half = warp >> 2;  // TMEM lanes of this warp; column half it drains
    const uint32_t N = g.N;
    const size_t y = sys_id();
    psi += y * NO * (size_t)N;
    const int R = 2 * NO;                       // tile rows in use: hi, then lo
    const int NM = (R + 15) & ~15;              // MMA N (multiple of 16)
    const uint32_t ncols = NM <= 32 ? 32u : NM <= 64 ? 64u : 128u;
    const int ld = R + 1;                       // fold row pitch (floats)
    const int NP = NO * (NO + 1) / 2;
    const uint32_t ntiles = (N + kTcSites - 1) / kTcSites;
    const int my_tiles = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);  // >= 1: gridDim.x <= ntiles

    for (int i = tid; i < L::tiles / 16; i += TH)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    const uint32_t idesc = idesc_bf16(kTcRows, NM);
    const uint32_t tiles_u32 = smem_u32(smem);

    const int nq = NO * (kTcSites / 4);
    // This thread's 4-site groups of every tile (the same in each tile): the
    // group's first site in the tile, its orbital's offset in psi, its
    // byte offset in a staged FP32 tile and in the swizzled hi and lo rows.
    uint32_t qk[kTcQuads], qring[kTcQuads], qhi[kTcQuads], qlo[kTcQuads];
    size_t qrow[kTcQuads];
#pragma unroll
    for (int q = 0; q < kTcQuads; ++q) {
        const int i = tid + q * TH, r = i >> 4, k = 4 * (i & 15);
        qk[q] = (uint32_t)k;
        qrow[q] = (size_t)r * N;
        qring[q] = (uint32_t)(r * kTcSites + k) * 4u;
        qhi[q] = tile_off(r, k);
        qlo[q] = tile_off(NO + r, k);
    }
    // Staged copy of local tile `it` into ring slot it % kInStages: this
    // thread's 16-byte pieces, one commit group per tile (empty past the end).
    auto issue = [&](int it) {
        if (it < my_tiles) {
            const uint32_t base = (blockIdx.x + (uint32_t)it * gridDim.x) * kTcSites;
            const uint32_t slot = smem_u32(ring + (it % kInStages) * stage_bytes);
#pragma unroll
            for (int q = 0; q < kTcQuads; ++q) {
                if (tid + q * TH >= nq) continue;
                const uint32_t site = base + qk[q];
                const bool in = site < N;  // N % 4 == 0: a piece is all in or all out
                cp_async16(slot + qring[q], in ? psi + qrow[q] + site : psi, in ? 16u : 0u);
            }
        }
        cp_async_commit();
    };
    if (BULK)
        for (int it = 0; it < kInStages - 1; ++it) issue(it);

    double acc[kTcMaxPairs];
    int pr[kTcMaxPairs];  // (a << 8) | b, or -1
#pragma unroll
    for (int q = 0; q < kTcMaxPairs; ++q) {
        acc[q] = 0.0;
        const int k = tid + q * TH;
        int a = 0, b = 0;
        if (k < NP) tri_pair(k, a, b);
        pr[q] = k < NP ? (a << 8) | b : -1;
    }

    float4 cur[kTcQuads], nxt[kTcQuads];
    // Register path: values of local tile `it` (zero past N).
    auto load = [&](int it, float4(&v)[kTcQuads]) {
        const uint32_t base = (blockIdx.x + (uint32_t)it * gridDim.x) * kTcSites;
#pragma unroll
        for (int q = 0; q < kTcQuads; ++q) {
            if (tid + q * TH >= nq) continue;
            const uint32_t site = base + qk[q];
            const float* p = psi + qrow[q] + site;
            v[q].x = site < N ? __ldg(p) : 0.f;
            v[q].y = site + 1 < N ? __ldg(p + 1) : 0.f;
            v[q].z = site + 2 < N ? __ldg(p + 2) : 0.f;
            v[q].w = site + 3 < N ? __ldg(p + 3) : 0.f;
        }
    };

    bool failed = false;
    int in_chunk = 0;
    uint32_t last_bar = 0, last_parity = 0;
    if (!BULK) load(0, cur);
    for (int it0 = 0; it0 < my_tiles; it0 += TPB) {
        const int nt = min(TPB, my_tiles - it0);  // tiles before this barrier
        const bool last_group = it0 + nt == my_tiles;
        bool late = false;
#pragma unroll
        for (int u = 0; u < TPB; ++u) {
            if (u >= nt) break;
            const int it = it0 + u;
            if (BULK) {
                // this thread's pieces of tile `it` have landed; every thread
                // reads back only the pieces it copied itself, so no block
                // barrier is needed, and slot (it - 1) % kInStages, which it
                // refills now, was read into its registers for tile it - 1
                cp_async_wait<kInStages - 2>();
                issue(it + kInStages - 1);
                const uint32_t base = (blockIdx.x + (uint32_t)it * gridDim.x) * kTcSites;
                const unsigned char* stg = ring + (it % kInStages) * stage_bytes;
#pragma unroll
                for (int q = 0; q < kTcQuads; ++q) {
                    if (tid + q * TH >= nq) continue;
                    cur[q] = base + qk[q] < N ? *reinterpret_cast<const float4*>(stg + qring[q])
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            } else if (it + 1 < my_tiles) {
                load(it + 1, nxt);
            }
            const int s = it % NS;
            // the MMAs of tile it - NS read this stage
            late = late ||
                   (it >= NS && !mbar_wait(smem_u32(&mbar[s]), (uint32_t)((it / NS) + 1) & 1u, wait_limit));
            unsigned char* st = smem + s * L::stride;
#pragma unroll
            for (int q = 0; q < kTcQuads; ++q) {
                if (tid + q * TH >= nq) continue;
                const float4 v = cur[q];
                const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
                const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
                const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
                const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
                *reinterpret_cast<uint2*>(st + qhi[q]) = make_uint2(bf2_bits(h01), bf2_bits(h23));
                *reinterpret_cast<uint2*>(st + qlo[q]) = make_uint2(bf2_bits(l01), bf2_bits(l23));
            }
            if (!BULK) {
#pragma unroll
                for (int q = 0; q < kTcQuads; ++q) cur[q] = nxt[q];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (__syncthreads_or(late)) {
            failed = true;
            break;
        }
        if (tid == 0) {
            tc_fence_after();
            for (int u = 0; u < nt; ++u) {
                const int s = (it0 + u) % NS;
                const uint64_t d0 = sw128_desc(tiles_u32 + s * L::stride);
#pragma unroll
                for (int k = 0; k < kTcSites / 16; ++k)  // K = 16 bf16 = 32 bytes = 2 descriptor units
                    mma_bf16(tmem, d0 + 2 * k, d0 + 2 * k, idesc, (in_chunk > 0 || u > 0 || k > 0) ? 1u : 0u);
                mma_commit(smem_u32(&mbar[s]));
            }
        }
        const int it_last = it0 + nt - 1;
        last_bar = smem_u32(&mbar[it_last % NS]);
        last_parity = (uint32_t)(it_last / NS) & 1u;
        in_chunk += nt;
        if (in_chunk >= drain_tiles || last_group) {
            in_chunk = 0;
            // the last commit tracks every earlier MMA of the issuing thread
            const bool ok = __all_sync(0xffffffffu, mbar_wait(last_bar, last_parity, wait_limit));
            tc_fence_after();
            if (ok && warp < 8 && lane_base < R) {  // two groups of four warps drain alternate 16-column blocks
                const int row = lane_base + (tid & 31);
                for (int cb = 16 * half; cb < NM; cb += 32) {
                    uint32_t v[16];
                    tmem_ld16(tmem + ((uint32_t)lane_base << 16) + (uint32_t)cb, v);
                    if (row < R) {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (cb + e < R) fold[row * ld + cb + e] = __uint_as_float(v[e]);
                    }
                }
            }
            tc_fence_before();
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
#pragma unroll
            for (int q = 0; q < kTcMaxPairs; ++q) {
                if (pr[q] < 0) continue;
                const int a = pr[q] >> 8, b = pr[q] & 255;
                const float d00 = fold[a * ld + b], d01 = fold[a * ld + NO + b];
                const float d10 = fold[(NO + a) * ld + b], d11 = fold[(NO + a) * ld + NO + b];
                acc[q] += (double)d00 + (double)((d01 + d10) + d11);
            }
            if (L::fold_in_tiles) __syncthreads();  // the fold is read before the next tiles overwrite it
        }
    }

    if (failed) {
        if (tid == 0) atomicAdd(&g_tc_timeouts, 1u);
        // own MMAs in flight: the last commit tracks every earlier MMA of this
        // thread; always the full bound, whatever limit the main waits had
        if (last_bar) mbar_wait(last_bar, last_parity, kWaitLimit);
    }
    if (BULK) cp_async_wait<0>();  // no copy may land after the block's shared memory is gone
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }

    double* partial = sys_partial(sc);
#pragma unroll
    for (int q = 0; q < kTcMaxPairs; ++q) {
        const int k = tid + q * TH;
        if (k < NP) partial[(size_t)blockIdx.x * NP + k] = failed ? __longlong_as_double(0x7ff8000000000000ll) : acc[q];
    }
    double* tot = reinterpret_cast<double*>(fold);  // NP doubles fit in the fold buffer
    if (grid_total_rt(partial, sys_counter(sc), tot, NP))
        store_overlap_block(tot, NO, h, S + y * NO * NO, LAM ? lam + y * NO * NO : nullptr,
                            LAM ? sigma + y * NO : nullptr);
}

template <bool LAM, bool BULK, int MAXO, int TH = kTcThreads, int TPB = 1>
static cudaError_t gram_tc_launch(int NO, const Grid& g, double h, const float* psi, double* S, double* lam,
                                  double* sigma, const Scratch& sc, int B, int drain_tiles, cudaStream_t st) {
    auto kern = k_gram_tc<LAM, BULK, MAXO, TH, TPB>;
    using L = TcLayout<MAXO, TPB>;
    const int R = 2 * NO, NM = (R + 15) & ~15;
    const int ncols = NM <= 32 ? 32 : NM <= 64 ? 64 : 128;
    size_t smem = 1024 + (size_t)L::tiles + (BULK ? (size_t)kInStages * NO * kTcSites * 4 : 0) +
                  (L::fold_in_tiles ? 0 : (size_t)R * (R + 1) * sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // the largest shared-memory carveout, so that two blocks fit beside each other
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TH, smem);
    if (e != cudaSuccess) return e;
    // The occupancy query has reported one block per SM where two fit (shared
    // memory and registers both allow two, and two run when launched): take
    // the larger of it and the count from the per-SM limits.
    {
        static const int smem_sm = [] {
            int dev = 0, v = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            return v;
        }();
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && fa.numRegs > 0) {
            const int regs = (fa.numRegs + 7) & ~7;
            const int by_regs = 65536 / (regs * TH);
            const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
            occ = std::max(occ, std::min(by_regs, by_smem));
        }
    }
    // co-resident blocks must not ask for more TMEM columns than an SM has
    const int cap = kTmemColumnsPerSm / ncols;
    for (int guard = 0; occ > cap && guard < 64; ++guard) {
        smem += 4096;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TH, smem);
        if (e != cudaSuccess) return e;
    }
    if (occ < 1 || occ > cap) return cudaErrorInvalidConfiguration;
    const size_t tiles = (g.N + kTcSites - 1) / kTcSites;
    const int per = std::max(1, std::min(sc.max_blocks, occ * num_sms() / std::max(B, 1)));
    const dim3 grid((unsigned)std::max<size_t>(1, std::min<size_t>(tiles, (size_t)per)), (unsigned)B);
    kern<<<grid, TH, smem, st>>>(g, h, psi, NO, drain_tiles, S, lam, sigma, sc, g_wait_limit.load());
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gram_tc(int NO, const Grid& g, double h, const float* psi, double* S, double* lam,
                           double* sigma, const Scratch& sc, int B, cudaStream_t st, int drain_tiles) {
    if (NO < 1 || NO > kMaxOrbWide || !psi || !S || (lam && !sigma)) return cudaErrorInvalidValue;
    if (sc.max_vals < NO * (NO + 1) / 2 || sc.systems < B || drain_tiles < 0) return cudaErrorInvalidValue;
    if (drain_tiles == 0) drain_tiles = kDrainTiles;
    const bool bulk = g.N % 4 == 0 && reinterpret_cast<uintptr_t>(psi) % 16 == 0;
#define LBKS_TC(MAXO)                                                                                          \
    return lam ? (bulk ? gram_tc_launch<true, true, MAXO>(NO, g, h, psi, S, lam, sigma, sc, B, drain_tiles, st)  \
                       : gram_tc_launch<true, false, MAXO>(NO, g, h, psi, S, lam, sigma, sc, B, drain_tiles, st)) \
               : (bulk ? gram_tc_launch<false, true, MAXO>(NO, g, h, psi, S, nullptr, nullptr, sc, B, drain_tiles, st) \
                       : gram_tc_launch<false, false, MAXO>(NO, g, h, psi, S, nullptr, nullptr, sc, B, drain_tiles, st));
    if (NO <= 16) LBKS_TC(16)
    if (NO <= 32) LBKS_TC(32)
    if (NO <= 40) {  // 16 NO 4-site groups of a tile: two per thread of ten warps; two tiles per barrier
        return lam ? (bulk ? gram_tc_launch<true, true, 40, 320, 2>(NO, g, h, psi, S, lam, sigma, sc, B, drain_tiles,
                                                                    st)
                           : gram_tc_launch<true, false, 40, 320, 2>(NO, g, h, psi, S, lam, sigma, sc, B, drain_tiles,
                                                                     st))
                   : (bulk ? gram_tc_launch<false, true, 40, 320, 2>(NO, g, h, psi, S, nullptr, nullptr, sc, B,
                                                                     drain_tiles, st)
                           : gram_tc_launch<false, false, 40, 320, 2>(NO, g, h, psi, S, nullptr, nullptr, sc, B,
                                                                      drain_tiles, st));
    }
    if (NO <= 48) LBKS_TC(48)
    LBKS_TC(kMaxOrbWide)
#undef LBKS_TC
}

uint32_t set_gram_tc_wait_limit(uint32_t polls) { return g_wait_limit.exchange(polls); }
uint32_t device_wait_limit() { return g_wait_limit.load(); }

unsigned gram_tc_timeouts() {
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_tc_timeouts, sizeof(v));
    return v;
}

}  // namespace lbks
