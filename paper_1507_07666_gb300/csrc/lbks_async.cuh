// Stream-collide with the pulled populations staged in shared memory by
// asynchronous copies (cp.async), several work units ahead.
//
// A work unit is one orbital of a tile of kTile consecutive sites.  For
// velocity p the populations arriving at the tile's sites come from the
// contiguous index range [s0 - off_p, s0 - off_p + kTile), off_p the linear
// offset of v_p: every thread copies its share of those ranges (16-byte pieces,
// the start rounded down to a 16-byte boundary) for the 19 populations and,
// from the second orbital on, the 19 shifted W-field ranges, into one slot of
// a kStages-deep ring.  Sources that wrap across a row or plane, or fall
// outside the grid, are loaded or not but never read: the site's has_source
// test decides.  The loads in flight are bounded by the ring, not by
// registers; the collision, the psi epilogue and the overlap partials are
// those of k_stream_collide.  Needs N % (16 / sizeof(TS)) == 0 and 16-byte
// aligned arrays (async_applies).  Included by lbks_relax_variants.cuh.
#pragma once

namespace lbks {

constexpr int kTile = kThreads;  // sites per work unit, one per thread

template <typename TS, typename T>
struct AsyncShape {
    static constexpr int ce_f = 16 / (int)sizeof(TS);  // elements per 16-byte piece
    static constexpr int ce_u = 16 / (int)sizeof(T);
    static constexpr int row_f = kTile + ce_f;          // staged elements per population
    static constexpr int row_u = kTile + ce_u;
    static constexpr int slot_bytes = 19 * (row_f * (int)sizeof(TS) + row_u * (int)sizeof(T));
    static constexpr int stages = sizeof(TS) == 8 ? 2 : sizeof(TS) == 4 ? 3 : 4;
    static constexpr int smem = stages * slot_bytes;
};

__device__ __forceinline__ void acp16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void acp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void acp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

// First staged element of velocity p's range for a tile starting at s0.
template <int CE>
__device__ __forceinline__ int64_t staged_start(int64_t s0, int off) {
    const int64_t a = s0 - off;
    return a <= 0 ? 0 : a - (a % CE);
}

template <typename TS, typename T, int NO, bool OM1, bool BATCHED>
__global__ void __launch_bounds__(kThreads, 1) k_stream_collide_async(Grid g, Coef c, RelaxIO io, Scratch sc) {
    using A = AsyncShape<TS, T>;
    constexpr int NP = NO * (NO + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (BATCHED && inactive(g)) return;
    const uint32_t N = g.N;
    const size_t y = BATCHED ? sys_id() : 0;
    const TS* __restrict__ fin = static_cast<const TS*>(io.f_in) + y * NO * 19 * N;
    const T* __restrict__ uin = static_cast<const T*>(io.u_in);
    const T* __restrict__ ubase = uin ? uin + y * (NO > 1 ? NO - 1 : 1) * N : nullptr;
    TS* __restrict__ fout = static_cast<TS*>(io.f_out) + y * NO * 19 * N;
    T* __restrict__ psio = static_cast<T*>(io.psi_out) + y * NO * N;
    const int off[19] = {
#define LBKS_OFF(p) vel(p, 0) + vel(p, 1) * g.nx + vel(p, 2) * g.nx * g.ny
        LBKS_OFF(0),  LBKS_OFF(1),  LBKS_OFF(2),  LBKS_OFF(3),  LBKS_OFF(4),  LBKS_OFF(5),  LBKS_OFF(6),
        LBKS_OFF(7),  LBKS_OFF(8),  LBKS_OFF(9),  LBKS_OFF(10), LBKS_OFF(11), LBKS_OFF(12), LBKS_OFF(13),
        LBKS_OFF(14), LBKS_OFF(15), LBKS_OFF(16), LBKS_OFF(17), LBKS_OFF(18)
#undef LBKS_OFF
    };
    T sig[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) sig[j] = (T)io.sigma_in[y * NO + j];
    const T om = (T)c.omega, dt = (T)c.dt, om1 = (T)(1.0 - c.omega);
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);

    const uint32_t ntiles = (N + kTile - 1) / kTile;
    const int my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const int units = my_tiles * NO;  // work units: (tile, orbital), orbital fastest
    const uint32_t ring = static_cast<uint32_t>(__cvta_generic_to_shared(smem_raw));

    // Copies of work unit `w` into its slot (every thread its pieces), one commit group.
    auto issue = [&](int w) {
        if (w < units) {
            const int64_t s0 = (int64_t)(blockIdx.x + (uint32_t)(w / NO) * gridDim.x) * kTile;
            const int j = w % NO;
            const uint32_t slot = ring + (uint32_t)((w % A::stages) * A::slot_bytes);
            const TS* fj = fin + (size_t)j * 19 * N;
            constexpr int pf = A::row_f / A::ce_f;  // pieces per population
            for (int k = threadIdx.x; k < 19 * pf; k += kThreads) {
                const int p = k / pf, q = k - p * pf;
                const int64_t cs = staged_start<A::ce_f>(s0, off[p]);
                const int64_t e = cs + (int64_t)q * A::ce_f;
                if (e < (int64_t)N) acp16(slot + (uint32_t)((p * A::row_f + q * A::ce_f) * sizeof(TS)), fj + (size_t)p * N + e);
            }
            if (j > 0 && ubase) {
                const T* uj = ubase + (size_t)(j - 1) * N;
                const uint32_t uslot = slot + (uint32_t)(19 * A::row_f * sizeof(TS));
                constexpr int pu = A::row_u / A::ce_u;
                for (int k = threadIdx.x; k < 19 * pu; k += kThreads) {
                    const int p = k / pu, q = k - p * pu;
                    const int64_t cs = staged_start<A::ce_u>(s0, off[p]);
                    const int64_t e = cs + (int64_t)q * A::ce_u;
                    if (e < (int64_t)N) acp16(uslot + (uint32_t)((p * A::row_u + q * A::ce_u) * sizeof(T)), uj + e);
                }
            }
        }
        acp_commit();
    };
#pragma unroll 1
    for (int w = 0; w < A::stages - 1; ++w) issue(w);

    // tiles outermost, orbitals unrolled inside (static indices into psi and sig)
    for (int tl = 0; tl < my_tiles; ++tl) {
        const int64_t s0 = (int64_t)(blockIdx.x + (uint32_t)tl * gridDim.x) * kTile;
        const uint32_t s = (uint32_t)s0 + threadIdx.x;
        T psi[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            const int w = tl * NO + j;
            acp_wait<A::stages - 2>();  // this thread's pieces of unit w have landed
            __syncthreads();            // everyone's; and the slot of unit w - 1 is free
            issue(w + A::stages - 1);
            const unsigned char* slot = smem_raw + (w % A::stages) * A::slot_bytes;
            const TS* sf = reinterpret_cast<const TS*>(slot);
            const T* su = reinterpret_cast<const T*>(slot + 19 * A::row_f * sizeof(TS));
            psi[j] = T(0);
            if (s < N) {
                const Site t = decode(g, s);
                T gp[19];
#pragma unroll
                for (int p = 0; p < 19; ++p) {
                    const int64_t src = (int64_t)s - off[p];
                    gp[p] = has_source(t, p)
                                ? to_compute<T>(sf[p * A::row_f + (int)(src - staged_start<A::ce_f>(s0, off[p]))])
                                : T(0);
                }
                if (j > 0 && ubase) {
#pragma unroll
                    for (int p = 0; p < 19; ++p) {
                        const int64_t src = (int64_t)s - off[p];
                        if (has_source(t, p))
                            gp[p] += xi[vclass(p)] * su[p * A::row_u + (int)(src - staged_start<A::ce_u>(s0, off[p]))];
                    }
                }
                const T vr = (T)__ldg(io.V + y * N + s);
                T ps = T(0);
#pragma unroll
                for (int p = 0; p < 19; ++p) ps += gp[p];
                ps *= sig[j];
                const T A_ = om * ps, B_ = dt * vr * ps;
                const T e[3] = {xi[0] * A_ - chi[0] * B_, xi[1] * A_ - chi[1] * B_, xi[2] * A_ - chi[2] * B_};
                const T c1 = om1 * sig[j];
                TS* oj = fout + (size_t)j * 19 * N;
#pragma unroll
                for (int p = 0; p < 19; ++p)
                    st_stream(oj + (size_t)p * N + s, to_store<TS>(OM1 ? e[vclass(p)] : c1 * gp[p] + e[vclass(p)]));
                psio[(size_t)j * N + s] = ps;
                psi[j] = ps;
            }
        }
#pragma unroll
        for (int a = 0; a < NO; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) acc[tri(a, b)] += psi[a] * psi[b];
    }
    acp_wait<0>();  // no copy may land after the block's shared memory is gone

    double v[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) v[k] = (double)acc[k];
    double* partial = sc.partial + y * sc.max_blocks * sc.max_vals;
    block_sum_store<NP>(v, partial + (size_t)blockIdx.x * NP);
    __shared__ double tot[NP];
    if (grid_total<NP>(partial, sc.counter + y, tot) && threadIdx.x == 0)
        store_overlap(tot, NO, c.h, io.S_out + y * NO * NO, io.lambda_out + y * NO * NO, io.sigma_out + y * NO);
}

template <typename TS, typename T, int NO, bool OM1, bool BATCHED>
cudaError_t launch_stream_collide_async(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                        cudaStream_t st) {
    using A = AsyncShape<TS, T>;
    auto kern = k_stream_collide_async<TS, T, NO, OM1, BATCHED>;
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, A::smem);
    if (attr != cudaSuccess) return attr;
    if (sc.max_vals < NO * (NO + 1) / 2 || sc.systems < B) return cudaErrorInvalidValue;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, A::smem) != cudaSuccess || nb < 1) nb = 1;
    kern<<<batch_grid(g.N, nb * num_sms(), B, sc.max_blocks), kThreads, A::smem, st>>>(g, c, io, sc);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lbks
