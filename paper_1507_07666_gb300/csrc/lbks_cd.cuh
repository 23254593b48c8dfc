// Concurrent dynamics (Eq. KSLBCD, Sec. 3 "Concurrent Dynamics"): the
// two-step, time-centred update of complex orbitals, templated on the compute
// type T (double or float) and the orbital count NO.  Included by
// lbks_cd_f64.cu and lbks_cd_f32.cu, each of which instantiates one T.
//
// At omega = 1 one ground-state step maps orbital j to
//   G_j(r) = sum_p [xi_p a_j - dt chi_p V phi_j](r - v_p),  zero outside the box,
//   a_j = phi_j - sum_{k<j} Lambda_jk phi_k,  Lambda_jk = <phi_k|phi_j> / <phi_k|phi_k>,
// i.e. phi_j + D_j with D_j = -dt H phi_j (+ the W source), H = (1 - K_xi)/dt + K_chi V.
// The paper's real-time scheme, read as the Wick rotation of that step with
// its own step tau, is
//   phi_j(t + tau) = phi_j(t - tau) + 2i (tau/dt) D_j(phi(t)) + 2 tau kappa E_j (K_q phi_j)(t),
// K_q the stencil of the U source's weights w_p q_p.  The kernel evaluates the
// general form
//   out_j = alpha prev_j + beta extra_j + c D_j(cur) + u_j (K_q cur_j)
// (c complex, u_j per orbital), which covers the step and the terms of the
// second-order start; one thread per site, the 18 neighbours of every orbital
// through L1, the overlap of `out` fused (the W source of the next step).
//
// Layout: a level holds [system][j][part][z][y][x], part 0 the real and 1 the
// imaginary values of orbital j, so its 2 NO planes read as real orbitals (the
// density and energy kernels take them as such).  Lambda and the overlap are
// [system][j][k][2] (real, imaginary) doubles.
#pragma once

#include "lbks_relax.cuh"

namespace lbks {

template <typename T, int NO>
__host__ __device__ constexpr int cd_min_blocks() {
    return sizeof(T) == 8 ? (NO <= 1 ? 3 : NO <= 4 ? 2 : 1) : (NO <= 2 ? 4 : NO <= 4 ? 3 : 2);
}

// Up to four orbitals the step accumulates the overlap of `out` itself; more
// would hold too many partial sums per thread, and a second kernel reads the
// level back.
template <int NO>
__host__ __device__ constexpr bool cd_fused_overlap() {
    return NO <= 4;
}

// Block and grid sums of the per-thread pair products acc (real and
// imaginary part of conj(out_i) out_j at 2 tri(j, i), i <= j); the last block
// writes S[i][j] = <out_i|out_j> and, with lam_out, Lambda_ji =
// <out_i|out_j> / <out_i|out_i> for i < j (zero elsewhere).  Every thread of
// the block must call it.
template <typename T, int NO>
__device__ __forceinline__ void finish_overlap(const T (&acc)[NO * (NO + 1)], double h, double* S_out,
                                               double* lam_out, const Scratch& sc) {
    constexpr int NP = NO * (NO + 1);
    const size_t y = sys_id();
    double v[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) v[k] = (double)acc[k];
    double* partial = sys_partial(sc);
    block_sum_store<NP>(v, partial + (size_t)blockIdx.x * NP);
    __shared__ double tot[NP];
    if (!grid_total<NP>(partial, sys_counter(sc), tot)) return;
    const double h3 = h * h * h;
    double* S = S_out + y * NO * NO * 2;
    double* L = lam_out ? lam_out + y * NO * NO * 2 : nullptr;
    for (int q = threadIdx.x; q < NO * NO; q += blockDim.x) {
        const int j = q / NO, i = q - j * NO;
        const int a = i <= j ? j : i, b = i <= j ? i : j;
        const double re = h3 * tot[2 * tri(a, b)];
        const double im = h3 * tot[2 * tri(a, b) + 1];
        S[(i * NO + j) * 2] = re;
        S[(i * NO + j) * 2 + 1] = i <= j ? im : -im;
        if (L) {
            const double nrm = h3 * tot[2 * tri(i, i)];
            L[(j * NO + i) * 2] = i < j ? re / nrm : 0.0;
            L[(j * NO + i) * 2 + 1] = i < j ? im / nrm : 0.0;
        }
    }
}

template <typename T, int NO, bool U>
__global__ void __launch_bounds__(kThreads, (cd_min_blocks<T, NO>())) k_cd_step(Grid g, CdCoef c, CdIO io, Scratch sc) {
    constexpr int NP = cd_fused_overlap<NO>() ? NO * (NO + 1) : 1;  // real and imaginary part of <out_i|out_j>, i <= j
    if (inactive(g)) return;
    const uint32_t N = g.N;
    const size_t y = sys_id();
    const size_t base = y * (size_t)NO * 2 * N;
    const T* __restrict__ cur = static_cast<const T*>(io.cur) + base;
    const T* __restrict__ prev = io.prev ? static_cast<const T*>(io.prev) + base : nullptr;
    const T* __restrict__ extra = io.extra ? static_cast<const T*>(io.extra) + base : nullptr;
    T* __restrict__ out = static_cast<T*>(io.out) + base;
    const double* __restrict__ Vs = io.V + y * N;
    const T dt = (T)c.dt;
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
    const T wq[3] = {(T)c.wq[0], (T)c.wq[1], (T)c.wq[2]};
    const T alpha = (T)io.alpha, beta = (T)io.beta, cr = (T)io.c_re, ci = (T)io.c_im;
    // -Lambda (strictly lower, complex), or no W source
    constexpr int NL = NO > 1 ? NO * (NO - 1) / 2 : 1;
    T lr[NL], li[NL];
    const bool with_w = NO > 1 && io.lam != nullptr;
#pragma unroll
    for (int j = 1; j < NO; ++j)
#pragma unroll
        for (int k = 0; k < j; ++k) {
            const double* l = io.lam + ((y * NO + j) * NO + k) * 2;
            lr[tri(j - 1, k)] = with_w ? (T)(-l[0]) : T(0);
            li[tri(j - 1, k)] = with_w ? (T)(-l[1]) : T(0);
        }
    T uc[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) uc[j] = U ? (T)io.ucoef[y * NO + j] : T(0);
    const bool with_s = cd_fused_overlap<NO>() && io.S_out != nullptr;
    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);

    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        const Site t = decode(g, s);
        // per orbital: ps = sum_p (xi_p - dt chi_p V) phi, kx = sum_p xi_p phi,
        // kq = sum_p w_p q_p phi, all over the pulled neighbours (real, imaginary)
        T psr[NO], psi[NO], kxr[NO], kxi[NO], kqr[NO], kqi[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) psr[j] = psi[j] = kxr[j] = kxi[j] = kqr[j] = kqi[j] = T(0);
#pragma unroll
        for (int p = 0; p < 19; ++p) {
            if (!has_source(t, p)) continue;
            const uint32_t src = source_index(g, s, p);
            const int k = vclass(p);
            const T a = xi[k] - dt * chi[k] * (T)__ldg(Vs + src);
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                const T vr = __ldg(cur + (size_t)(2 * j) * N + src);
                const T vi = __ldg(cur + (size_t)(2 * j + 1) * N + src);
                psr[j] += a * vr;
                psi[j] += a * vi;
                kxr[j] += xi[k] * vr;
                kxi[j] += xi[k] * vi;
                if (U && k != 1) {  // w_p q_p vanishes on the axis velocities
                    kqr[j] += wq[k] * vr;
                    kqi[j] += wq[k] * vi;
                }
            }
        }
        T o_re[NO], o_im[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            // G_j = ps_j - sum_{k<j} Lambda_jk kx_k; D_j = G_j - phi_j
            T gr = psr[j], gi = psi[j];
#pragma unroll
            for (int k = 0; k < j; ++k) {
                const T mr = lr[tri(j - 1, k)], mi = li[tri(j - 1, k)];
                gr += mr * kxr[k] - mi * kxi[k];
                gi += mr * kxi[k] + mi * kxr[k];
            }
            const T dr = gr - cur[(size_t)(2 * j) * N + s];
            const T di = gi - cur[(size_t)(2 * j + 1) * N + s];
            T vr = cr * dr - ci * di, vi = cr * di + ci * dr;
            if (prev) {
                vr += alpha * prev[(size_t)(2 * j) * N + s];
                vi += alpha * prev[(size_t)(2 * j + 1) * N + s];
            }
            if (extra) {
                vr += beta * extra[(size_t)(2 * j) * N + s];
                vi += beta * extra[(size_t)(2 * j + 1) * N + s];
            }
            if (U) {
                vr += uc[j] * kqr[j];
                vi += uc[j] * kqi[j];
            }
            out[(size_t)(2 * j) * N + s] = vr;
            out[(size_t)(2 * j + 1) * N + s] = vi;
            o_re[j] = vr;
            o_im[j] = vi;
        }
        if constexpr (cd_fused_overlap<NO>()) {
            if (with_s) {
                // conj(out_i) out_j = (a_i a_j + b_i b_j) + i (a_i b_j - b_i a_j)
#pragma unroll
                for (int j = 0; j < NO; ++j)
#pragma unroll
                    for (int i = 0; i <= j; ++i) {
                        acc[2 * tri(j, i)] += o_re[i] * o_re[j] + o_im[i] * o_im[j];
                        acc[2 * tri(j, i) + 1] += o_re[i] * o_im[j] - o_im[i] * o_re[j];
                    }
            }
        }
    }
    if constexpr (cd_fused_overlap<NO>()) {
        if (with_s) finish_overlap<T, NO>(acc, io.h, io.S_out, io.lam_out, sc);
    }
}

// The same step with its inputs staged in shared memory: a block takes a
// tile of kCdTX x kCdTY x TZ sites, loads the tile's box with a one-site halo
// of every orbital's real and imaginary plane and of V once (zero outside the
// grid, the empty-source rule), and sums the 19 neighbours from shared
// memory.  Each thread owns one (x, y) column and TZ sites along z.  Tiles are
// taken in a block-stride loop.  Dynamic shared memory: (2 NO + 1) box values.
constexpr int kCdTX = 32, kCdTY = 8;

template <int TZ>
__host__ __device__ constexpr int cd_box() {
    return (kCdTX + 2) * (kCdTY + 2) * (TZ + 2);
}

template <typename T, int NO, bool U, int TZ>
__global__ void __launch_bounds__(kThreads) k_cd_step_tile(Grid g, CdCoef c, CdIO io, Scratch sc) {
    constexpr int NP = cd_fused_overlap<NO>() ? NO * (NO + 1) : 1;
    constexpr int PX = kCdTX + 2, PY = kCdTY + 2, BOX = cd_box<TZ>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* box = reinterpret_cast<T*>(smem_raw);  // [2 NO + 1][BOX]: re/im of each orbital, then V
    if (inactive(g)) return;
    const uint32_t N = g.N;
    const size_t y = sys_id();
    const size_t base = y * (size_t)NO * 2 * N;
    const T* __restrict__ cur = static_cast<const T*>(io.cur) + base;
    const T* __restrict__ prev = io.prev ? static_cast<const T*>(io.prev) + base : nullptr;
    const T* __restrict__ extra = io.extra ? static_cast<const T*>(io.extra) + base : nullptr;
    T* __restrict__ out = static_cast<T*>(io.out) + base;
    const double* __restrict__ Vs = io.V + y * N;
    const T dt = (T)c.dt;
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
    const T wq[3] = {(T)c.wq[0], (T)c.wq[1], (T)c.wq[2]};
    const T alpha = (T)io.alpha, beta = (T)io.beta, cr = (T)io.c_re, ci = (T)io.c_im;
    constexpr int NL = NO > 1 ? NO * (NO - 1) / 2 : 1;
    T lr[NL], li[NL];
    const bool with_w = NO > 1 && io.lam != nullptr;
#pragma unroll
    for (int j = 1; j < NO; ++j)
#pragma unroll
        for (int k = 0; k < j; ++k) {
            const double* l = io.lam + ((y * NO + j) * NO + k) * 2;
            lr[tri(j - 1, k)] = with_w ? (T)(-l[0]) : T(0);
            li[tri(j - 1, k)] = with_w ? (T)(-l[1]) : T(0);
        }
    T uc[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) uc[j] = U ? (T)io.ucoef[y * NO + j] : T(0);
    const bool with_s = cd_fused_overlap<NO>() && io.S_out != nullptr;
    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);

    const int tx = threadIdx.x % kCdTX, ty = threadIdx.x / kCdTX;
    const int ntx = (g.nx + kCdTX - 1) / kCdTX, nty = (g.ny + kCdTY - 1) / kCdTY, ntz = (g.nz + TZ - 1) / TZ;
    const int ntiles = ntx * nty * ntz;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int bxi = tile % ntx, byi = (tile / ntx) % nty, bzi = tile / (ntx * nty);
        const int x0 = bxi * kCdTX - 1, y0 = byi * kCdTY - 1, z0 = bzi * TZ - 1;  // box origin
        __syncthreads();  // the previous tile's box is no longer read
        for (int i = threadIdx.x; i < BOX; i += kThreads) {
            const int bx = i % PX, by = (i / PX) % PY, bz = i / (PX * PY);
            const int gx = x0 + bx, gy = y0 + by, gz = z0 + bz;
            const bool in = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz;
            const size_t gs = in ? ((size_t)gz * g.ny + gy) * g.nx + gx : 0;
#pragma unroll
            for (int q = 0; q < 2 * NO; ++q) box[q * BOX + i] = in ? __ldg(cur + (size_t)q * N + gs) : T(0);
            box[2 * NO * BOX + i] = in ? (T)__ldg(Vs + gs) : T(0);
        }
        __syncthreads();
        const int gx = x0 + 1 + tx, gy = y0 + 1 + ty;
#pragma unroll 1
        for (int dz = 0; dz < TZ; ++dz) {
            const int gz = z0 + 1 + dz;
            const bool live = gx < g.nx && gy < g.ny && gz < g.nz;
            const int b = ((dz + 1) * PY + (ty + 1)) * PX + (tx + 1);  // the site in the box
            T psr[NO], psi[NO], kxr[NO], kxi[NO], kqr[NO], kqi[NO];
#pragma unroll
            for (int j = 0; j < NO; ++j) psr[j] = psi[j] = kxr[j] = kxi[j] = kqr[j] = kqi[j] = T(0);
#pragma unroll
            for (int p = 0; p < 19; ++p) {
                const int src = b - (vel(p, 0) + vel(p, 1) * PX + vel(p, 2) * PX * PY);
                const int k = vclass(p);
                const T a = xi[k] - dt * chi[k] * box[2 * NO * BOX + src];
#pragma unroll
                for (int j = 0; j < NO; ++j) {
                    const T vr = box[(2 * j) * BOX + src], vi = box[(2 * j + 1) * BOX + src];
                    psr[j] += a * vr;
                    psi[j] += a * vi;
                    kxr[j] += xi[k] * vr;
                    kxi[j] += xi[k] * vi;
                    if (U && k != 1) {
                        kqr[j] += wq[k] * vr;
                        kqi[j] += wq[k] * vi;
                    }
                }
            }
            if (!live) continue;
            const size_t s = ((size_t)gz * g.ny + gy) * g.nx + gx;
            T o_re[NO], o_im[NO];
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                T gr = psr[j], gi = psi[j];
#pragma unroll
                for (int k = 0; k < j; ++k) {
                    const T mr = lr[tri(j - 1, k)], mi = li[tri(j - 1, k)];
                    gr += mr * kxr[k] - mi * kxi[k];
                    gi += mr * kxi[k] + mi * kxr[k];
                }
                const T dr = gr - box[(2 * j) * BOX + b];
                const T di = gi - box[(2 * j + 1) * BOX + b];
                T vr = cr * dr - ci * di, vi = cr * di + ci * dr;
                if (prev) {
                    vr += alpha * prev[(size_t)(2 * j) * N + s];
                    vi += alpha * prev[(size_t)(2 * j + 1) * N + s];
                }
                if (extra) {
                    vr += beta * extra[(size_t)(2 * j) * N + s];
                    vi += beta * extra[(size_t)(2 * j + 1) * N + s];
                }
                if (U) {
                    vr += uc[j] * kqr[j];
                    vi += uc[j] * kqi[j];
                }
                out[(size_t)(2 * j) * N + s] = vr;
                out[(size_t)(2 * j + 1) * N + s] = vi;
                o_re[j] = vr;
                o_im[j] = vi;
            }
            if constexpr (cd_fused_overlap<NO>()) {
                if (with_s) {
#pragma unroll
                    for (int j = 0; j < NO; ++j)
#pragma unroll
                        for (int i = 0; i <= j; ++i) {
                            acc[2 * tri(j, i)] += o_re[i] * o_re[j] + o_im[i] * o_im[j];
                            acc[2 * tri(j, i) + 1] += o_re[i] * o_im[j] - o_im[i] * o_re[j];
                        }
                }
            }
        }
    }
    if constexpr (cd_fused_overlap<NO>()) {
        if (with_s) finish_overlap<T, NO>(acc, io.h, io.S_out, io.lam_out, sc);
    }
}

// Tile depth of the staged kernel, or 0 where its box would leave fewer than
// two blocks per SM (the one-site kernel runs there).
template <typename T, int NO>
__host__ __device__ constexpr int cd_tile_depth() {
    return (2 * NO + 1) * cd_box<4>() * (int)sizeof(T) <= 112 * 1024   ? 4
           : (2 * NO + 1) * cd_box<2>() * (int)sizeof(T) <= 112 * 1024 ? 2
                                                                       : 0;
}

// Overlap and Lambda of one level alone (the first level of a run).
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_cd_overlap(Grid g, const T* __restrict__ phi, double h, double* S_out,
                                                         double* lam_out, Scratch sc) {
    constexpr int NP = NO * (NO + 1);
    if (inactive(g)) return;
    const uint32_t N = g.N;
    const size_t y = sys_id();
    phi += y * (size_t)NO * 2 * N;
    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        T re[NO], im[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) {
            re[j] = phi[(size_t)(2 * j) * N + s];
            im[j] = phi[(size_t)(2 * j + 1) * N + s];
        }
#pragma unroll
        for (int j = 0; j < NO; ++j)
#pragma unroll
            for (int i = 0; i <= j; ++i) {
                acc[2 * tri(j, i)] += re[i] * re[j] + im[i] * im[j];
                acc[2 * tri(j, i) + 1] += re[i] * im[j] - im[i] * re[j];
            }
    }
    finish_overlap<T, NO>(acc, h, S_out, lam_out, sc);
}

// ----------------------------------------------------------------- launchers
template <typename T, int NO>
cudaError_t launch_cd_overlap_no(const Grid& g, const void* phi, double h, double* S, double* lam, const Scratch& sc,
                                 int B, cudaStream_t st) {
    auto kern = k_cd_overlap<T, NO>;
    static const int nb = blocks_per_sm(kern);
    if (sc.max_vals < NO * (NO + 1) || sc.systems < B) return cudaErrorInvalidValue;
    kern<<<batch_grid(g.N, nb * num_sms(), B, sc.max_blocks), kThreads, 0, st>>>(g, static_cast<const T*>(phi), h, S,
                                                                                   lam, sc);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, int NO, bool U>
cudaError_t launch_cd_step_no(const Grid& g, const CdCoef& c, const CdIO& io, const Scratch& sc, int B,
                              cudaStream_t st) {
    if (cd_fused_overlap<NO>() && io.S_out && (sc.max_vals < NO * (NO + 1) || sc.systems < B))
        return cudaErrorInvalidValue;
    constexpr int TZ = cd_tile_depth<T, NO>();
    bool staged = false;
    if constexpr (TZ > 0) {
        if (cd_kernel_mode() != 0) {
            auto kern = k_cd_step_tile<T, NO, U, TZ>;
            const size_t smem = (size_t)(2 * NO + 1) * cd_box<TZ>() * sizeof(T);
            static const cudaError_t attr =
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (attr != cudaSuccess) return attr;
            static const int nb = [&] {
                int v = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, kThreads, smem) != cudaSuccess || v < 1)
                    v = 1;
                return v;
            }();
            const size_t tiles =
                (size_t)((g.nx + kCdTX - 1) / kCdTX) * ((g.ny + kCdTY - 1) / kCdTY) * ((g.nz + TZ - 1) / TZ);
            const int per = std::max(1, std::min(nb * num_sms() / std::max(B, 1), sc.max_blocks));
            kern<<<dim3((unsigned)std::min<size_t>(tiles, (size_t)per), (unsigned)B), kThreads, smem, st>>>(g, c, io,
                                                                                                            sc);
            staged = true;
        }
    }
    if (!staged) {
        auto kern = k_cd_step<T, NO, U>;
        static const int nb = blocks_per_sm(kern);
        kern<<<batch_grid(g.N, nb * num_sms(), B, sc.max_blocks), kThreads, 0, st>>>(g, c, io, sc);
    }
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !cd_fused_overlap<NO>() && io.S_out)
        e = launch_cd_overlap_no<T, NO>(g, io.out, io.h, io.S_out, io.lam_out, sc, B, st);
    return e;
}

template <typename T>
cudaError_t launch_cd_step(int NO, const Grid& g, const CdCoef& c, const CdIO& io, const Scratch& sc, int B,
                           cudaStream_t st) {
    const bool u = io.ucoef != nullptr;
    switch (NO) {
#define LBKS_CD_CASE(n) \
    case n:             \
        return u ? launch_cd_step_no<T, n, true>(g, c, io, sc, B, st) : launch_cd_step_no<T, n, false>(g, c, io, sc, B, st);
        LBKS_CD_CASE(1)
        LBKS_CD_CASE(2)
        LBKS_CD_CASE(3)
        LBKS_CD_CASE(4)
        LBKS_CD_CASE(5)
        LBKS_CD_CASE(6)
        LBKS_CD_CASE(7)
        LBKS_CD_CASE(8)
#undef LBKS_CD_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_cd_overlap(int NO, const Grid& g, const void* phi, double h, double* S, double* lam,
                              const Scratch& sc, int B, cudaStream_t st) {
    switch (NO) {
#define LBKS_CD_CASE(n) \
    case n:             \
        return launch_cd_overlap_no<T, n>(g, phi, h, S, lam, sc, B, st);
        LBKS_CD_CASE(1)
        LBKS_CD_CASE(2)
        LBKS_CD_CASE(3)
        LBKS_CD_CASE(4)
        LBKS_CD_CASE(5)
        LBKS_CD_CASE(6)
        LBKS_CD_CASE(7)
        LBKS_CD_CASE(8)
#undef LBKS_CD_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace lbks
