// Stream-collide at omega = 1 fed by the tensor memory accelerator: the
// pulled populations of each work unit arrive in shared memory by bulk
// copies, so the bytes in flight are bounded by a ring of shared-memory
// slots, not by registers.
//
// A work unit is one orbital j of a tile of kBulkTile consecutive sites
// [s0, s0 + Lt) of one system.  For velocity p the populations arriving at the
// tile come from the contiguous index range [s0 - off_p, s0 - off_p + Lt) of
// f_in[j][p], off_p = vx + vy nx + vz nx ny the linear offset of v_p.  One
// producer thread copies those 19 ranges (start rounded down, end rounded up
// to 16 bytes, clamped to the array) with cp.async.bulk into a slot of an
// S-deep ring; the slot's mbarrier counts the bytes in.  Sources that wrap
// across a row or plane, or lie outside the grid, are copied or not but never
// read: the site's has_source test decides.
//
// The pulled W source sum_p xi_p u_(j-1)(r - v_p) reads one array at 19
// offsets; velocities with the same (vy, vz) read the same row, so nine
// ranges [s0 - vy nx - vz nx ny - 1, ... + Lt + 1) cover them, copied into the
// same slot from the second orbital on.  The first orbital's slot also
// receives V of the tile.
//
// Eight consumer warps own one site of the tile each.  Per unit a thread sums
// its 19 arriving populations and the W source from the slot, scales by
// sigma_j and collides (Eq. KSLB at omega = 1, where every post-collision
// population is xi_p psi - dt chi_p V psi: three values per site), frees the
// slot (one arrival per warp) and writes the 19 populations and psi with
// streaming stores.
//
// The overlap S = h^3 Psi Psi^T of the step is fused: psi of every orbital of
// the tile is kept in shared memory, and at the end of the tile the consumer
// warps add the tile's pair products to per-block FP64 sums (FP32 products
// summed over the tile's sites, FP64 across tiles; exact: FP64 products and
// sums throughout).  The last block finishes the grid sum in a fixed order
// and writes S, Lambda and sigma.  No psi is read back from global memory.
//
// Every mbarrier wait is bounded.  A wait that gives up sets the block's abort
// flag: the producer stops issuing, consumers stop storing, the block's
// overlap partials become NaN (the solve then fails on the host), the
// producer waits (bounded) for every copy it issued and the block returns.
//
// Needs omega = 1, FP32 or bfloat16 populations with float orbitals, N a
// multiple of 16 / sizeof(population) and of 4, and 16-byte aligned arrays
// (bulk_applies in lbks_relax.cuh).  Included by lbks_relax_variants.cuh.
#pragma once

namespace lbks {

constexpr int kBulkTile = 256;                    // sites per work unit, one per consumer thread
constexpr int kBulkConsumers = kBulkTile;         // eight consumer warps
constexpr int kBulkThreads = kBulkConsumers + 32; // and one producer warp
constexpr int kBulkMaxStages = 16;
constexpr uint32_t kBulkWaitLimit = 1u << 22;

template <typename TS, typename T>
struct BulkShape {
    static constexpr int ce = 16 / (int)sizeof(TS);   // population elements per 16 bytes
    static constexpr int row = kBulkTile + 2 * ce;    // slot elements per population
    static constexpr int ceu = 16 / (int)sizeof(T);   // W-field elements per 16 bytes
    // slot elements per W-field row: a range of Lt + 2 sites (x halo of one)
    // rounded out to 16 bytes spans at most Lt + 2 ceu; the pitch is a whole
    // number of 16-byte units so that every row starts on a 16-byte boundary
    static constexpr int rowu = kBulkTile + 3 * ceu;
    static constexpr int pop_bytes = 19 * row * (int)sizeof(TS);
    static constexpr int u_bytes = 9 * rowu * (int)sizeof(T);
    static constexpr int slot_bytes = pop_bytes + u_bytes + kBulkTile * (int)sizeof(double);  // + V
    // every bulk copy's shared-memory destination must be 16-byte aligned
    static_assert(row * sizeof(TS) % 16 == 0 && rowu * sizeof(T) % 16 == 0, "row pitches of whole 16 bytes");
    static_assert(pop_bytes % 16 == 0 && u_bytes % 16 == 0 && slot_bytes % 16 == 0, "slot parts of whole 16 bytes");
    static_assert(rowu >= kBulkTile + 2 * ceu, "a W-field range fits its row");
};

// Row of the W-field ranges that velocity p reads: its (vy, vz) among
// (0,0), (1,0), (-1,0), (0,1), (0,-1), (1,1), (-1,-1), (1,-1), (-1,1).
__host__ __device__ constexpr int urow_of(int p) {
    constexpr int r[19] = {0, 0, 0, 1, 2, 3, 4, 1, 2, 2, 1, 3, 4, 4, 3, 5, 6, 7, 8};
    return r[p];
}
__host__ __device__ constexpr int urow_vy(int r) {
    constexpr int v[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    return v[r];
}
__host__ __device__ constexpr int urow_vz(int r) {
    constexpr int v[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    return v[r];
}

__device__ __forceinline__ uint32_t bulk_smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void bulk_mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bulk_mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_mbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Waits for the phase of the given parity; false after `limit` polls or, with
// a flag, once another thread of the block has aborted.
__device__ __forceinline__ bool bulk_mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit,
                                               const volatile int* abort_flag) {
    for (uint32_t i = 0; i < limit; ++i) {
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
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// global -> shared, completion counted on bar.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Named barrier of the consumer warps (id 1); the producer warp never joins it.
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kBulkConsumers) : "memory"); }
__device__ __forceinline__ int consumers_or(int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"(pred), "n"(kBulkConsumers)
        : "memory");
    return r;
}

// Floor of a / b for b > 0 (a may be negative).
__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

template <typename TS, typename T>
__global__ void __launch_bounds__(kBulkThreads, 1)
    k_stream_collide_bulk(Grid g, Coef c, RelaxIO io, Scratch sc, int NO, int S, int psi_bufs, int exact,
                          uint32_t wait_limit) {
    using Sh = BulkShape<TS, T>;
    constexpr int CE = Sh::ce, ROW = Sh::row, CEU = Sh::ceu, ROWU = Sh::rowu;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int NP = NO * (NO + 1) / 2;
    const int y = (int)blockIdx.y;
    if (g.active && !g.active[y]) return;
    const uint32_t N = g.N;
    const int tid = (int)threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // shared memory: slots, psi tiles, FP64 pair sums, barriers
    unsigned char* slots = smem_raw;
    T* psit = reinterpret_cast<T*>(slots + (size_t)S * Sh::slot_bytes);
    double* accs = reinterpret_cast<double*>(psit + (size_t)psi_bufs * NO * kBulkTile);
    uint64_t* bars = reinterpret_cast<uint64_t*>(accs + NP);
    const uint32_t full0 = bulk_smem_u32(bars), empty0 = full0 + 8 * S;
    __shared__ int abort_flag;

    const TS* __restrict__ fin = static_cast<const TS*>(io.f_in) + (size_t)y * NO * 19 * N;
    TS* __restrict__ fout = static_cast<TS*>(io.f_out) + (size_t)y * NO * 19 * N;
    T* __restrict__ psio = static_cast<T*>(io.psi_out) + (size_t)y * NO * N;
    const T* __restrict__ ubase =
        io.u_in ? static_cast<const T*>(io.u_in) + (size_t)y * (NO > 1 ? NO - 1 : 1) * N : nullptr;
    const double* __restrict__ V = io.V + (size_t)y * N;

    const int64_t nxy = (int64_t)g.nx * g.ny;
    const uint32_t ntiles = (N + kBulkTile - 1) / kBulkTile;
    const int my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const int units = my_tiles * NO;

    if (tid == 0) abort_flag = 0;
    for (int k = tid; k < NP; k += kBulkThreads) accs[k] = 0.0;
    if (tid == kBulkConsumers) {
        for (int s = 0; s < S; ++s) {
            bulk_mbar_init(full0 + 8 * s, 1);
            bulk_mbar_init(empty0 + 8 * s, kBulkConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    bool failed = false;
    if (warp == kBulkConsumers / 32) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int u = 0;
            for (; u < units; ++u) {
                const int stage = u % S, k = u / S;
                if (k > 0 && !bulk_mbar_wait(empty0 + 8 * stage, (uint32_t)(k - 1) & 1u, wait_limit, &abort_flag)) {
                    failed = true;
                    break;
                }
                if (abort_flag) break;
                const int tl = u / NO, j = u - tl * NO;
                const int64_t s0 = (int64_t)(blockIdx.x + (uint32_t)tl * gridDim.x) * kBulkTile;
                const int64_t lt = min64(kBulkTile, (int64_t)N - s0);
                const TS* fj = fin + (size_t)j * 19 * N;
                const uint32_t slot = bulk_smem_u32(slots + (size_t)stage * Sh::slot_bytes);
                const bool with_u = ubase != nullptr && j > 0;
                // a range [lo, hi) of the array, its 16-byte-rounded start a, clamped to the array
                auto pop_range = [&](int p, int64_t& a, int64_t& lo, int64_t& hi) {
                    const int64_t off = vel(p, 0) + vel(p, 1) * (int64_t)g.nx + vel(p, 2) * nxy;
                    a = floor_div(s0 - off, CE) * CE;
                    lo = max64(a, 0);
                    hi = min64(floor_div(s0 - off + lt + CE - 1, CE) * CE, (int64_t)N);
                };
                auto u_range = [&](int r, int64_t& a, int64_t& lo, int64_t& hi) {
                    const int64_t off = urow_vy(r) * (int64_t)g.nx + urow_vz(r) * nxy;
                    a = floor_div(s0 - off - 1, CEU) * CEU;
                    lo = max64(a, 0);
                    hi = min64(floor_div(s0 - off + lt + 1 + CEU - 1, CEU) * CEU, (int64_t)N);
                };
                uint32_t bytes = j == 0 ? (uint32_t)(lt * (int64_t)sizeof(double)) : 0u;
#pragma unroll
                for (int p = 0; p < 19; ++p) {
                    int64_t a, lo, hi;
                    pop_range(p, a, lo, hi);
                    if (hi > lo) bytes += (uint32_t)((hi - lo) * (int64_t)sizeof(TS));
                }
                if (with_u) {
#pragma unroll
                    for (int r = 0; r < 9; ++r) {
                        int64_t a, lo, hi;
                        u_range(r, a, lo, hi);
                        if (hi > lo) bytes += (uint32_t)((hi - lo) * (int64_t)sizeof(T));
                    }
                }
                bulk_mbar_expect(full0 + 8 * stage, bytes);
#pragma unroll
                for (int p = 0; p < 19; ++p) {
                    int64_t a, lo, hi;
                    pop_range(p, a, lo, hi);
                    if (hi > lo)
                        bulk_load(slot + (uint32_t)((p * ROW + (lo - a)) * (int64_t)sizeof(TS)), fj + (size_t)p * N + lo,
                                  (uint32_t)((hi - lo) * (int64_t)sizeof(TS)), full0 + 8 * stage);
                }
                if (with_u) {
                    const T* uj = ubase + (size_t)(j - 1) * N;
#pragma unroll
                    for (int r = 0; r < 9; ++r) {
                        int64_t a, lo, hi;
                        u_range(r, a, lo, hi);
                        if (hi > lo)
                            bulk_load(slot + (uint32_t)(Sh::pop_bytes + (r * ROWU + (lo - a)) * (int64_t)sizeof(T)),
                                      uj + lo, (uint32_t)((hi - lo) * (int64_t)sizeof(T)), full0 + 8 * stage);
                    }
                }
                if (j == 0)
                    bulk_load(slot + (uint32_t)(Sh::pop_bytes + Sh::u_bytes), V + s0, (uint32_t)(lt * sizeof(double)),
                              full0 + 8 * stage);
            }
            if (failed) abort_flag = 1;
            // every copy issued must have landed before the block's shared memory goes away
            for (int w = u > S ? u - S : 0; w < u; ++w)
                bulk_mbar_wait(full0 + 8 * (w % S), (uint32_t)(w / S) & 1u, kBulkWaitLimit, nullptr);
        }
    } else {
        // ----------------------------------------------------------- consumers
        const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
        const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
        const T dt = (T)c.dt;
        // Tile starts are multiples of kBulkTile, so the slot index of the source
        // r - v_p is tid + rem_p with rem_p = (-off_p) mod CE, and in the W-field
        // row of (vy, vz) it is tid + 1 - vx + ((-off_row - 1) mod CEU): per-velocity
        // constants of the grid, formed where they are used.
        const int nxm = g.nx & (CE - 1), nxym = (int)(nxy & (CE - 1));
        const int nxu = g.nx & (CEU - 1), nxyu = (int)(nxy & (CEU - 1));
        T vr = T(0);
        for (int tl = 0; tl < my_tiles; ++tl) {
            const int64_t s0 = (int64_t)(blockIdx.x + (uint32_t)tl * gridDim.x) * kBulkTile;
            const int64_t lt = min64(kBulkTile, (int64_t)N - s0);
            const bool live = tid < lt;
            const uint32_t s = (uint32_t)(s0 + (live ? tid : 0));
            const Site t = decode(g, s);
            uint32_t mask = 0;
#pragma unroll
            for (int p = 0; p < 19; ++p)
                if (live && has_source(t, p)) mask |= 1u << p;
            T* prow = psit + (size_t)(psi_bufs > 1 ? (tl & 1) : 0) * NO * kBulkTile;
            for (int j = 0; j < NO; ++j) {
                const int u = tl * NO + j, stage = u % S;
                bool ok = !failed && bulk_mbar_wait(full0 + 8 * stage, (uint32_t)(u / S) & 1u, wait_limit, &abort_flag);
                if (!ok) failed = true;
                T ps = T(0);
                if (ok) {
                    const unsigned char* slot = slots + (size_t)stage * Sh::slot_bytes;
                    const TS* sf = reinterpret_cast<const TS*>(slot);
#pragma unroll
                    for (int p = 0; p < 19; ++p) {
                        const int rem = (-vel(p, 0) - vel(p, 1) * nxm - vel(p, 2) * nxym) & (CE - 1);
                        if ((mask >> p) & 1u) ps += to_compute<T>(sf[p * ROW + tid + rem]);
                    }
                    if (ubase && j > 0) {
                        const T* su = reinterpret_cast<const T*>(slot + Sh::pop_bytes);
                        T w = T(0);
#pragma unroll
                        for (int p = 0; p < 19; ++p) {
                            const int r = urow_of(p);
                            const int rem = (-urow_vy(r) * nxu - urow_vz(r) * nxyu - 1) & (CEU - 1);
                            if ((mask >> p) & 1u) w += xi[vclass(p)] * su[r * ROWU + tid + 1 - vel(p, 0) + rem];
                        }
                        ps += w;
                    }
                    if (j == 0)
                        vr = live ? (T)reinterpret_cast<const double*>(slot + Sh::pop_bytes + Sh::u_bytes)[tid] : T(0);
                }
                __syncwarp();
                if (lane == 0 && ok) bulk_mbar_arrive(empty0 + 8 * stage);
                if (!ok) {
                    abort_flag = 1;
                    prow[(size_t)j * kBulkTile + tid] = T(0);
                    continue;
                }
                ps *= (T)__ldg(io.sigma_in + (size_t)y * NO + j);
                const T B = dt * vr * ps;
                const T e[3] = {xi[0] * ps - chi[0] * B, xi[1] * ps - chi[1] * B, xi[2] * ps - chi[2] * B};
                prow[(size_t)j * kBulkTile + tid] = live ? ps : T(0);
                if (live) {
                    TS* oj = fout + (size_t)j * 19 * N + s;
#pragma unroll
                    for (int p = 0; p < 19; ++p) st_stream(oj + (size_t)p * N, to_store<TS>(e[vclass(p)]));
                    psio[(size_t)j * N + s] = ps;
                }
            }
            // overlap of the tile: pair k to warp k % 8, sites strided over the lanes
            if (consumers_or(failed)) failed = true;
            if (!failed) {
                for (int k = warp; k < NP; k += kBulkConsumers / 32) {
                    int a, b;
                    tri_pair(k, a, b);
                    const T* ra = prow + (size_t)a * kBulkTile;
                    const T* rb = prow + (size_t)b * kBulkTile;
                    double v;
                    if (exact) {
                        double q = 0.0;
                        for (int l = lane; l < kBulkTile; l += 32) q += (double)ra[l] * (double)rb[l];
                        v = q;
                    } else {
                        T q = T(0);
                        for (int l = lane; l < kBulkTile; l += 32) q += ra[l] * rb[l];
                        v = (double)q;
                    }
                    v = warp_sum1(v);
                    if (lane == 0) accs[k] += v;
                }
            }
            if (psi_bufs == 1) consumers_sync();  // the tile's psi rows are read before the next tile writes them
        }
    }
    __syncthreads();
    if (abort_flag) failed = true;
    double* partial = sc.partial + (size_t)y * sc.max_blocks * sc.max_vals;
    for (int k = tid; k < NP; k += kBulkThreads)
        partial[(size_t)blockIdx.x * NP + k] = failed ? __longlong_as_double(0x7ff8000000000000ll) : accs[k];
    double* tot = reinterpret_cast<double*>(slots);  // the slots are free now
    if (grid_total_rt(partial, sc.counter + y, tot, NP))
        store_overlap_block(tot, NO, c.h, io.S_out + (size_t)y * NO * NO, io.lambda_out + (size_t)y * NO * NO,
                            io.sigma_out + (size_t)y * NO);
}

// Resident blocks: one per SM; slots as many as the shared memory holds
// (at most kBulkMaxStages) after the psi tiles and the pair sums.
template <typename TS, typename T>
cudaError_t launch_stream_collide_bulk(int NO, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc,
                                       int B, bool exact, uint32_t wait_limit, cudaStream_t st) {
    using Sh = BulkShape<TS, T>;
    auto kern = k_stream_collide_bulk<TS, T>;
    const int NP = NO * (NO + 1) / 2;
    if (sc.max_vals < NP || sc.systems < B || NO < 1 || NO > kMaxOrbWide) return cudaErrorInvalidValue;
    static const int smem_max = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        return v;
    }();
    const int psi_bufs = NO <= 16 ? 2 : 1;
    const size_t fixed = (size_t)psi_bufs * NO * kBulkTile * sizeof(T) + (size_t)NP * sizeof(double);
    const size_t room = (size_t)smem_max - 1024 - fixed;  // static shared memory and reserve
    int S = (int)std::min<size_t>(kBulkMaxStages, room / (Sh::slot_bytes + 16));
    if (S < 2) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)S * Sh::slot_bytes + fixed + 16 * (size_t)S;
    // the grid-total scratch reuses the slots: NP doubles must fit
    if ((size_t)S * Sh::slot_bytes < (size_t)NP * sizeof(double)) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const size_t tiles = (g.N + kBulkTile - 1) / kBulkTile;
    const int per = std::max(1, std::min(sc.max_blocks, num_sms() / std::max(B, 1)));
    const dim3 grid((unsigned)std::max<size_t>(1, std::min<size_t>(tiles, (size_t)per)), (unsigned)B);
    kern<<<grid, kBulkThreads, smem, st>>>(g, c, io, sc, NO, S, psi_bufs, exact ? 1 : 0, wait_limit);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lbks
