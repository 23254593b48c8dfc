// Orbital-storage relaxation at omega = 1 fed by the tensor memory
// accelerator (TMA): the same 19-point stencil as k_relax_psi_tile,
//
//   psi'_j(r) = sigma_j [ sum_p (xi_p - dt chi_p Vc(r - v_p)) psi_j(r - v_p)
//                         - omega sum_{k<j} Lambda_jk (K_xi psi_k)(r) ],
//   (K_xi psi_k)(r) = sum_p xi_p psi_k(r - v_p),
//
// zero outside the box, for any number of orbitals: the W source is formed
// from the K_xi sums that the thread already holds for the lower orbitals of
// its site, so no W field is written or read at any orbital count.
//
// Work unit: one orbital of a tile of kTX x kTY sites of one z-plane.  Its
// input is one TMA box of psi_j -- x from x0 - pad (a 16-byte boundary) over
// bx values, y0 - 1 .. y0 + kTY, z - 1 .. z + 1 -- copied into a ring of
// shared-memory slots; the tile's Vc box (same geometry, FP64) sits in a
// ring of its own.  Out-of-range coordinates read zero, which is the
// empty-source rule of the pull.  Thread 0 issues the copies ahead of use and
// each copy signals its slot's `full` mbarrier with the byte count; the eight
// warps (one site per thread, a warp = one x-row of the tile) wait on it, sum
// the 19 neighbours from shared memory and release the slot through its
// `empty` mbarrier (one arrival per warp).  Tiles are taken
// in a block-stride loop, plane by plane, so a plane's neighbours are read
// from L2 by the blocks working next to it.
//
// Every mbarrier wait is bounded.  On expiry the block records it, writes
// NaN for the site's orbitals (and, with the overlap fused, NaN partial sums,
// so the solve fails with a non-finite energy), stops issuing copies, waits
// (bounded) for the copies already issued and returns.
//
// Needs nx a multiple of 16 / sizeof(T) and 16-byte aligned psi and Vc
// (psi_tma_applies): the tensor maps' row pitches are multiples of 16 bytes.
// Included by lbks_psi.cuh.
#pragma once

#include <cuda.h>  // CUtensorMap (the map is encoded on the host, lbks_tma.cu)

namespace lbks {

// 4-D tiled tensor map over [nw][nz][ny][nx] values (FP64 if f64, else FP32),
// box bx x by x bz x 1, zero fill out of range.  Defined in lbks_tma.cu.
cudaError_t encode_box_map(CUtensorMap* map, bool f64, const void* base, int nx, int ny, int nz, int nw, int bx,
                           int by, int bz);

template <typename T>
struct PsiTmaShape {
    static constexpr int pad = 16 / (int)sizeof(T);                         // x values per 16 bytes
    static constexpr int bx = (kTX + 1 + pad + pad - 1) / pad * pad;        // 40 (FP32), 36 (FP64)
    static constexpr int by = kTY + 2;
    static constexpr int bz = 3;
    static constexpr int box = bx * by * bz;                                // values per box
    static constexpr int slot_psi = (box * (int)sizeof(T) + 127) / 128 * 128;  // bytes, 128-byte aligned slots
    static constexpr int slot_v = (box * 8 + 127) / 128 * 128;
    static constexpr int stages = sizeof(T) == 4 ? 8 : 6;                  // psi box slots
    static constexpr int vstages = 3;                                      // Vc box slots
};

// Row pitch of -omega Lambda in shared memory: whole 16-byte loads.
template <typename T, int MAXO>
__host__ __device__ constexpr int psi_tma_pitch() {
    return (MAXO + 16 / (int)sizeof(T) - 1) / (16 / (int)sizeof(T)) * (16 / (int)sizeof(T));
}
// Bytes of -omega Lambda (MAXO rows) and sigma (MAXO, padded to 16 bytes).
template <typename T, int MAXO>
__host__ __device__ constexpr size_t psi_tma_coef_bytes() {
    return ((size_t)MAXO * psi_tma_pitch<T, MAXO>() + psi_tma_pitch<T, MAXO>()) * sizeof(T);
}
// Dynamic shared memory: psi ring, two Vc slots, -omega Lambda and sigma,
// then the mbarriers (plus 128 bytes to round the base up to 128 bytes).
template <typename T, int MAXO>
constexpr size_t psi_tma_smem() {
    using S = PsiTmaShape<T>;
    return 128 + (size_t)S::stages * S::slot_psi + S::vstages * S::slot_v + psi_tma_coef_bytes<T, MAXO>() +
           (2 * S::stages + 2 * S::vstages) * 8;
}

constexpr uint32_t kPsiWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t psi_smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void psi_mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void psi_mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void psi_mbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Waits for the completion of the barrier's phase of the given parity; false
// after kPsiWaitLimit polls or once another thread has flagged an abort.
__device__ __forceinline__ bool psi_mbar_wait(uint32_t bar, uint32_t parity, const volatile int* abort_flag) {
    for (uint32_t i = 0; i < kPsiWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (abort_flag && *abort_flag) return false;
    }
    return false;
}
// One box of a 4-D tensor map into shared memory, completion counted on bar.
__device__ __forceinline__ void psi_tma_load(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int w,
                                             uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
        : "memory");
}

// EXACT: NO == MAXO (at most kMaxOrb), overlap, Lambda and sigma fused as in
// k_relax_psi_tile.  Otherwise NO <= MAXO at run time and the overlap follows
// in its own kernel.  blockIdx.y = system.
//
// Thread 0 also issues the copies: before it takes unit u it issues every
// unit up to u + stages - 2 whose tile is less than vstages tiles ahead, so
// each wait it makes for a free slot is on units that the block has already
// passed (u - 2 or earlier), never on its own later work.
template <typename T, int MAXO, bool EXACT>
__global__ void __launch_bounds__(kThreads, (EXACT || MAXO <= 16) ? 2 : 1)
    k_relax_psi_tma(const __grid_constant__ CUtensorMap tm_psi, const __grid_constant__ CUtensorMap tm_v, Grid g,
                    Coef c, RelaxIO io, Scratch sc, int NO_rt) {
    using S = PsiTmaShape<T>;
    constexpr int NP = EXACT ? MAXO * (MAXO + 1) / 2 : 1;
    constexpr int NW = kThreads / 32;
    constexpr int LP = psi_tma_pitch<T, MAXO>();
    const int NO = EXACT ? MAXO : NO_rt;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // tensor copies land on 128-byte boundaries
    unsigned char* base = smem_raw + ((128u - (psi_smem_u32(smem_raw) & 127u)) & 127u);
    const T* ring = reinterpret_cast<const T*>(base);
    const double* vring = reinterpret_cast<const double*>(base + S::stages * S::slot_psi);
    unsigned char* tail = base + S::stages * S::slot_psi + S::vstages * S::slot_v;
    T* Lw = reinterpret_cast<T*>(tail);  // -omega Lambda, row pitch LP, zero on and above the diagonal
    T* sg = Lw + MAXO * LP;              // sigma_in
    uint64_t* bars = reinterpret_cast<uint64_t*>(tail + psi_tma_coef_bytes<T, MAXO>());
    const uint32_t full0 = psi_smem_u32(bars), empty0 = full0 + 8 * S::stages;
    const uint32_t vfull0 = empty0 + 8 * S::stages, vempty0 = vfull0 + 8 * S::vstages;
    const uint32_t ring0 = psi_smem_u32(ring), vring0 = psi_smem_u32(vring);
    __shared__ int abort_flag;

    if (g.active && !g.active[blockIdx.y]) return;
    const int y = (int)blockIdx.y;
    const uint32_t N = g.N;
    const int ntx = (g.nx + kTX - 1) / kTX, nty = (g.ny + kTY - 1) / kTY;
    const int ntiles = ntx * nty * g.nz;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int units = my_tiles * NO;
    const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
    const bool with_w = NO > 1 && io.lambda_in != nullptr;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < S::stages; ++s) {
            psi_mbar_init(full0 + 8 * s, 1);
            psi_mbar_init(empty0 + 8 * s, NW);
        }
        for (int s = 0; s < S::vstages; ++s) {
            psi_mbar_init(vfull0 + 8 * s, 1);
            psi_mbar_init(vempty0 + 8 * s, NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_psi)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_v)) : "memory");
    }
    // read before this block arrives at the overlap counter: the last block
    // of a fused-overlap launch overwrites Lambda and sigma in place
    for (int i = (int)threadIdx.x; i < MAXO * LP; i += kThreads) {
        const int j = i / LP, k = i - j * LP;
        Lw[i] = (with_w && j < NO && k < j) ? (T)(-c.omega * io.lambda_in[(size_t)y * NO * NO + j * NO + k]) : T(0);
    }
    for (int j = (int)threadIdx.x; j < MAXO; j += kThreads) sg[j] = j < NO ? (T)io.sigma_in[(size_t)y * NO + j] : T(0);
    __syncthreads();

    // issue cursor (thread 0): next unit, its tile and orbital
    int iu = 0, itl = 0, ij = 0, ivt = 0;  // ivt: Vc boxes issued
    bool ok = true;
    // Issues units while iu < limit and their tile is below tile_cap; false on a
    // wait that gave up.
    auto produce = [&](int limit, int tile_cap) -> bool {
        for (; iu < limit && iu < units && itl < tile_cap; ++iu) {
            const int tile = (int)blockIdx.x + itl * (int)gridDim.x;
            const int bxi = tile % ntx, t2 = tile / ntx, byi = t2 % nty, z = t2 / nty;
            const int x0 = bxi * kTX - S::pad, y0 = byi * kTY - 1;
            if (ij == 0) {  // the tile's Vc box first
                const int vs = itl % S::vstages, vk = itl / S::vstages;
                if (vk > 0 && !psi_mbar_wait(vempty0 + 8 * vs, (uint32_t)(vk - 1) & 1u, &abort_flag)) return false;
                psi_mbar_expect(vfull0 + 8 * vs, (uint32_t)(S::box * 8));
                psi_tma_load(vring0 + vs * S::slot_v, &tm_v, x0, y0, z - 1, y, vfull0 + 8 * vs);
                ++ivt;
            }
            const int s = iu % S::stages, k = iu / S::stages;
            if (k > 0 && !psi_mbar_wait(empty0 + 8 * s, (uint32_t)(k - 1) & 1u, &abort_flag)) return false;
            psi_mbar_expect(full0 + 8 * s, (uint32_t)(S::box * sizeof(T)));
            psi_tma_load(ring0 + s * S::slot_psi, &tm_psi, x0, y0, z - 1, y * NO + ij, full0 + 8 * s);
            if (++ij == NO) {
                ij = 0;
                ++itl;
            }
        }
        return true;
    };
    if (threadIdx.x == 0) ok = produce(S::stages - 1, S::vstages);

    const T dt = (T)c.dt;
    const T xi0 = (T)c.xi[0], xi1 = (T)c.xi[1], xi2 = (T)c.xi[2];
    const T cv[3] = {dt * (T)c.chi[0], dt * (T)c.chi[1], dt * (T)c.chi[2]};
    const T xiv[3] = {xi0, xi1, xi2};
    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);
    T kx[MAXO];
#pragma unroll
    for (int k = 0; k < MAXO; ++k) kx[k] = T(0);
    T* __restrict__ pout = static_cast<T*>(io.f_out) + (size_t)y * NO * N;
    // the thread's site in a box: plane 1, row warp + 1, column lane + pad
    const int cb = (S::by + warp + 1) * S::bx + lane + S::pad;
    int u = 0;
    for (int tl = 0; tl < my_tiles && ok; ++tl) {
        const int tile = (int)blockIdx.x + tl * (int)gridDim.x;
        const int bxi = tile % ntx, t2 = tile / ntx, byi = t2 % nty, z = t2 / nty;
        const int gx = bxi * kTX + lane, gy = byi * kTY + warp;
        const bool live = gx < g.nx && gy < g.ny;
        const size_t site = ((size_t)z * g.ny + gy) * g.nx + gx;
        const int vs = tl % S::vstages;
        // (the tile's Vc box went out with its first unit, during the previous tile or the prologue)
        if (ok) ok = psi_mbar_wait(vfull0 + 8 * vs, (uint32_t)(tl / S::vstages) & 1u, &abort_flag);
        if (!ok) break;
        T a[19];
        {
            const double* vb = vring + (size_t)vs * (S::slot_v / 8) + cb;
#pragma unroll
            for (int p = 0; p < 19; ++p)
                a[p] = xiv[vclass(p)] -
                       cv[vclass(p)] * (T)vb[-(vel(p, 0) + vel(p, 1) * S::bx + vel(p, 2) * S::bx * S::by)];
        }
        __syncwarp();
        if (lane == 0) psi_mbar_arrive(vempty0 + 8 * vs);
        T psn[EXACT ? MAXO : 1];
#pragma unroll
        for (int j = 0; j < MAXO; ++j) {
            if (j >= NO) break;
            if (threadIdx.x == 0 && ok) ok = produce(u + S::stages - 1, tl + S::vstages);
            const int s = u % S::stages;
            if (ok) ok = psi_mbar_wait(full0 + 8 * s, (uint32_t)(u / S::stages) & 1u, &abort_flag);
            if (!ok) break;
            const T* pb = ring + (size_t)s * (S::slot_psi / sizeof(T)) + cb;
            const T v0 = pb[0];
            // independent partial sums: short dependency chains
            T pq[3] = {a[0] * v0, T(0), T(0)}, k1[2] = {T(0), T(0)}, k2[2] = {T(0), T(0)};
#pragma unroll
            for (int p = 1; p < 19; ++p) {
                const T w = pb[-(vel(p, 0) + vel(p, 1) * S::bx + vel(p, 2) * S::bx * S::by)];
                pq[p % 3] += a[p] * w;
                if (vclass(p) == 1) k1[p & 1] += w;
                else k2[p & 1] += w;
            }
            T ps = (pq[0] + pq[1]) + pq[2];
            __syncwarp();
            if (lane == 0) psi_mbar_arrive(empty0 + 8 * s);
            ++u;
            kx[j] = xi0 * v0 + xi1 * (k1[0] + k1[1]) + xi2 * (k2[0] + k2[1]);
            if (j > 0) {
                // -omega Lambda_j. by 16-byte broadcast loads, V independent partial sums
                constexpr int V = 16 / sizeof(T);
                const T* Lr = Lw + j * LP;
                T ws[V];
#pragma unroll
                for (int e = 0; e < V; ++e) ws[e] = T(0);
#pragma unroll
                for (int kb = 0; kb < j; kb += V) {
                    T l[V];
                    if constexpr (V == 4) {
                        const float4 q = *reinterpret_cast<const float4*>(Lr + kb);
                        l[0] = q.x;
                        l[1] = q.y;
                        l[2] = q.z;
                        l[3] = q.w;
                    } else {
                        const double2 q = *reinterpret_cast<const double2*>(Lr + kb);
                        l[0] = q.x;
                        l[1] = q.y;
                    }
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (kb + e < j) ws[e] += l[e] * kx[kb + e];
                }
                if constexpr (V == 4) ps += (ws[0] + ws[1]) + (ws[2 % V] + ws[3 % V]);
                else ps += ws[0] + ws[1];
            }
            ps = live ? ps * sg[j] : T(0);
            if (live) pout[(size_t)j * N + site] = ps;
            if constexpr (EXACT) psn[j] = ps;
        }
        if (!ok) {
            if (live)
                for (int j = 0; j < NO; ++j) pout[(size_t)j * N + site] = T(NAN);
            break;
        }
        if constexpr (EXACT) {
#pragma unroll
            for (int a2 = 0; a2 < MAXO; ++a2)
#pragma unroll
                for (int b2 = 0; b2 <= a2; ++b2) acc[tri(a2, b2)] += psn[a2] * psn[b2];
        }
    }
    if (!ok) abort_flag = 1;
    if (threadIdx.x == 0) {
        // every copy issued has landed before the block's shared memory goes away
        for (int w = iu > S::stages ? iu - S::stages : 0; w < iu; ++w)
            psi_mbar_wait(full0 + 8 * (w % S::stages), (uint32_t)(w / S::stages) & 1u, nullptr);
        for (int t = ivt > S::vstages ? ivt - S::vstages : 0; t < ivt; ++t)
            psi_mbar_wait(vfull0 + 8 * (t % S::vstages), (uint32_t)(t / S::vstages) & 1u, nullptr);
    }
    if constexpr (EXACT) {
        double v[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) v[k] = ok ? (double)acc[k] : (double)NAN;
        double* partial = sc.partial + (size_t)y * sc.max_blocks * sc.max_vals;
        block_sum_store<NP>(v, partial + (size_t)blockIdx.x * NP);
        __shared__ double tot[NP];
        if (grid_total<NP>(partial, sc.counter + y, tot) && threadIdx.x == 0)
            store_overlap(tot, NO, c.h, io.S_out + (size_t)y * NO * NO, io.lambda_out + (size_t)y * NO * NO,
                          io.sigma_out + (size_t)y * NO);
    }
}

template <typename T, int MAXO, bool EXACT>
cudaError_t launch_relax_psi_tma_k(int NO, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                   cudaStream_t st) {
    using S = PsiTmaShape<T>;
    auto kern = k_relax_psi_tma<T, MAXO, EXACT>;
    constexpr size_t smem = psi_tma_smem<T, MAXO>();
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    if (EXACT && (sc.max_vals < NO * (NO + 1) / 2 || sc.systems < B)) return cudaErrorInvalidValue;
    CUtensorMap tp, tv;
    cudaError_t e = encode_box_map(&tp, sizeof(T) == 8, io.f_in, g.nx, g.ny, g.nz, NO * B, S::bx, S::by, S::bz);
    if (e == cudaSuccess) e = encode_box_map(&tv, true, io.V, g.nx, g.ny, g.nz, B, S::bx, S::by, S::bz);
    if (e != cudaSuccess) return e;
    static const int nb = [&] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kThreads, smem) != cudaSuccess || n < 1) n = 1;
        return n;
    }();
    const size_t tiles = (size_t)((g.nx + kTX - 1) / kTX) * ((g.ny + kTY - 1) / kTY) * g.nz;
    size_t per = std::max<size_t>(1, (size_t)nb * num_sms() / std::max(B, 1));
    if (EXACT) per = std::min<size_t>(per, (size_t)sc.max_blocks);
    per = std::min(per, tiles);
    kern<<<dim3((unsigned)per, (unsigned)B), kThreads, smem, st>>>(tp, tv, g, c, io, sc, NO);
    count_launches(1);
    return cudaGetLastError();
}

// Orbital-storage step through the TMA kernel: up to kMaxOrb orbitals with
// the overlap fused, more in compile-time buckets of 16 (overlap after).
template <typename T>
cudaError_t launch_relax_psi_tma(int NO, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                 cudaStream_t st) {
    if (!psi_tma_applies(g.nx, io.f_in, io.V, sizeof(T))) return cudaErrorInvalidValue;
    switch (NO) {
#define LBKS_CASE(n) \
    case n: return launch_relax_psi_tma_k<T, n, true>(NO, g, c, io, sc, B, st);
        LBKS_CASE(1) LBKS_CASE(2) LBKS_CASE(3) LBKS_CASE(4) LBKS_CASE(5) LBKS_CASE(6) LBKS_CASE(7) LBKS_CASE(8)
#undef LBKS_CASE
        default: break;
    }
    if (NO <= 16) return launch_relax_psi_tma_k<T, 16, false>(NO, g, c, io, sc, B, st);
    if (NO <= 32) return launch_relax_psi_tma_k<T, 32, false>(NO, g, c, io, sc, B, st);
    if (NO <= 48) return launch_relax_psi_tma_k<T, 48, false>(NO, g, c, io, sc, B, st);
    if (NO <= kMaxOrbWide) return launch_relax_psi_tma_k<T, kMaxOrbWide, false>(NO, g, c, io, sc, B, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbks
