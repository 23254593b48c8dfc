// Relaxation in orbital storage at omega = 1 (tau = 1 of the paper's runs).
//
// At omega = 1 the collision forgets the arriving populations: the
// post-collision state of Eq. KSLB is f*_p(r) = xi_p A(r) - chi_p B(r) +
// xi_p u(r), with A = psi (this step's normalised orbital), B = dt V psi and
// u the W field.  Every stored population is a fixed combination of three
// site fields, so the next step's pull-and-sum collapses to a 19-point
// stencil on psi:
//
//   psi'(r) = sigma * sum_p [ (xi_p - dt chi_p Vc(r - v_p)) psi(r - v_p) + xi_p u(r - v_p) ],
//
// zero outside the box, where Vc is the potential of the collision that
// produced psi (the previous step's; zero for the start f = xi psi).  The
// populations never exist in memory: a step reads psi, u and Vc and writes
// psi' -- about 12 bytes of HBM traffic per orbital-site instead of 152.
// The same normalisation, overlap, Lambda and W field follow as in the
// population kernels.  Included by the lbks_relax_<precision>_psi.cu units.
#pragma once

#include "lbks_relax.cuh"

namespace lbks {

// out_j = sum_p [ (xi_p - dt chi_p Vc(r - v_p)) psi_j(r - v_p) + xi_p u_j(r - v_p) ]
// for the J orbitals j0 .. j0 + J - 1 of one site (terms outside the box are
// zero).  Velocities outermost: one source index and one weight live at a
// time, the J orbital loads of a velocity are independent.
// psi: orbital j0's array, u: the W field of orbital j0 (or nullptr when j0 has
// none, i.e. j0 == 0 or no W field); orbitals are N apart in both.
template <typename T, int J>
__device__ __forceinline__ void psi_stencil(const Grid& g, const Site& t, uint32_t s, const double* __restrict__ Vc,
                                            const T* __restrict__ psi, const T* __restrict__ u0,
                                            const T* __restrict__ u1, size_t N, const T (&xi)[3],
                                            const T (&chi)[3], T dt, T (&out)[J]) {
#pragma unroll
    for (int j = 0; j < J; ++j) out[j] = T(0);
#pragma unroll
    for (int p = 0; p < 19; ++p) {
        if (!has_source(t, p)) continue;
        const uint32_t src = source_index(g, s, p);
        const T a = xi[vclass(p)] - dt * chi[vclass(p)] * (T)__ldg(Vc + src);
#pragma unroll
        for (int j = 0; j < J; ++j) out[j] += a * __ldg(psi + (size_t)j * N + src);
        // W field: orbital j0 takes u0 (may be null), orbitals j0 + 1 .. take u1 + (j - 1) N
        if (u0) out[0] += xi[vclass(p)] * __ldg(u0 + src);
        if (u1) {
#pragma unroll
            for (int j = 1; j < J; ++j) out[j] += xi[vclass(p)] * __ldg(u1 + (size_t)(j - 1) * N + src);
        }
    }
}

// Up to kMaxOrb orbitals: one site per thread, all orbitals, overlap partials
// fused (as k_stream_collide); the last block writes S, Lambda and sigma.
// io.f_in / io.f_out: psi in / out ([sys][j][z][y][x], T); io.V: Vc.
//
// The W source needs no field: a thread holds every orbital of its site, and
// sum_p xi_p u_j(r - v_p) = -omega sum_{k<j} Lambda_jk (K_xi psi_k)(r) with
// K_xi psi_k = sum_p xi_p psi_k(r - v_p), which the same loads give.  Lambda
// is read from io.lambda_in (the previous step's, written by that step's
// last block; null at a cycle's first step) before any block of this launch
// arrives at the counter, so the last block may overwrite it.
// Resident blocks per SM the register allocator must allow: the unrolled
// stencil keeps the loads of several velocities of every orbital in flight.
template <typename T, int NO>
constexpr int psi_min_blocks() {
    return NO <= 2 ? 4 : (NO <= 5 && sizeof(T) == 4) ? 3 : 2;
}

template <typename T, int NO, bool BATCHED>
__global__ void __launch_bounds__(kThreads, (psi_min_blocks<T, NO>())) k_relax_psi(Grid g, Coef c, RelaxIO io,
                                                                                    Scratch sc) {
    constexpr int NP = NO * (NO + 1) / 2;
    if (BATCHED && inactive(g)) return;
    const uint32_t N = g.N;
    const size_t y = BATCHED ? sys_id() : 0;
    const T* __restrict__ pin = static_cast<const T*>(io.f_in);
    const T* __restrict__ uin = static_cast<const T*>(io.u_in);
    T* __restrict__ pout = static_cast<T*>(io.f_out);
    T sig[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) sig[j] = (T)io.sigma_in[y * NO + j];
    const T dt = (T)c.dt;
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);

    // -omega Lambda (strictly lower), or no W source
    constexpr int NL = NO > 1 ? NO * (NO - 1) / 2 : 1;
    T wl[NL];
    const bool with_w = NO > 1 && io.lambda_in != nullptr;
#pragma unroll
    for (int j = 1; j < NO; ++j)
#pragma unroll
        for (int k = 0; k < j; ++k)
            wl[tri(j - 1, k)] = with_w ? (T)(-c.omega * io.lambda_in[y * NO * NO + j * NO + k]) : T(0);
    (void)uin;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < N; s += gridDim.x * kThreads) {
        const Site t = decode(g, s);
        T ps[NO], kx[NO];
#pragma unroll
        for (int j = 0; j < NO; ++j) ps[j] = kx[j] = T(0);
        const double* Vc = io.V + y * N;
        const T* pj = pin + y * NO * N;
#pragma unroll
        for (int p = 0; p < 19; ++p) {
            if (!has_source(t, p)) continue;
            const uint32_t src = source_index(g, s, p);
            const T a = xi[vclass(p)] - dt * chi[vclass(p)] * (T)__ldg(Vc + src);
#pragma unroll
            for (int j = 0; j < NO; ++j) {
                const T v = __ldg(pj + (size_t)j * N + src);
                ps[j] += a * v;
                kx[j] += xi[vclass(p)] * v;
            }
        }
#pragma unroll
        for (int j = 0; j < NO; ++j) {
#pragma unroll
            for (int k = 0; k < j; ++k) ps[j] += wl[tri(j - 1, k)] * kx[k];
            ps[j] *= sig[j];
            pout[(y * NO + j) * N + s] = ps[j];
        }
#pragma unroll
        for (int j = 0; j < NO; ++j)
#pragma unroll
            for (int i = 0; i <= j; ++i) acc[tri(j, i)] += ps[j] * ps[i];
    }
    double v[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) v[k] = (double)acc[k];
    double* partial = sc.partial + y * sc.max_blocks * sc.max_vals;
    block_sum_store<NP>(v, partial + (size_t)blockIdx.x * NP);
    __shared__ double tot[NP];
    if (grid_total<NP>(partial, sc.counter + y, tot) && threadIdx.x == 0)
        store_overlap(tot, NO, c.h, io.S_out + y * NO * NO, io.lambda_out + y * NO * NO, io.sigma_out + y * NO);
}

// More than kMaxOrb orbitals: one site and a group of up to kPsiGroup orbitals
// per thread (they share the source indices and the weights), blockIdx.y =
// system * groups + group; the overlap follows in its own kernel.
constexpr int kPsiGroup = 4;

template <typename T, int J>
__device__ __forceinline__ void psi_group(const Grid& g, const Coef& c, const RelaxIO& io, int NO, int y, int j0,
                                          uint32_t s) {
    const size_t N = g.N;
    const T dt = (T)c.dt;
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
    const Site t = decode(g, s);
    const T* uw = static_cast<const T*>(io.u_in);
    const T* ubase = uw ? uw + (size_t)y * (NO - 1) * N : nullptr;  // W field of orbital j is ubase + (j - 1) N
    const T* u0 = (ubase && j0 > 0) ? ubase + (size_t)(j0 - 1) * N : nullptr;
    const T* u1 = ubase ? ubase + (size_t)j0 * N : nullptr;
    const size_t o0 = (size_t)y * NO + j0;
    T ps[J];
    psi_stencil<T, J>(g, t, s, io.V + (size_t)y * N, static_cast<const T*>(io.f_in) + o0 * N, u0, u1, N, xi, chi, dt,
                      ps);
#pragma unroll
    for (int j = 0; j < J; ++j) static_cast<T*>(io.f_out)[(o0 + j) * N + s] = (T)io.sigma_in[o0 + j] * ps[j];
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 3) k_relax_psi_wide(Grid g, Coef c, RelaxIO io, int NO) {
    const int groups = (NO + kPsiGroup - 1) / kPsiGroup;
    const int y = (int)blockIdx.y / groups, jg = (int)blockIdx.y - y * groups;
    if (g.active && !g.active[y]) return;
    const uint32_t s = blockIdx.x * kThreads + threadIdx.x;
    if (s >= g.N) return;
    const int j0 = jg * kPsiGroup, J = min(kPsiGroup, NO - j0);  // block-uniform
    if (J == 4) psi_group<T, 4>(g, c, io, NO, y, j0, s);
    else if (J == 3) psi_group<T, 3>(g, c, io, NO, y, j0, s);
    else if (J == 2) psi_group<T, 2>(g, c, io, NO, y, j0, s);
    else psi_group<T, 1>(g, c, io, NO, y, j0, s);
}

// The same step with the stencil's inputs staged in shared memory: a block
// takes a tile of kTX x kTY x kTZ sites, loads the tile's box with a one-site
// halo of every orbital's psi and of Vc once (zero outside the grid, which is
// the empty-source rule), and sums the 19 neighbours from shared memory.
// Each thread owns one (x, y) column of the tile and kTZ sites along z.
// Tiles are taken in a block-stride loop (the grid stays within the overlap
// scratch's block count).  Dynamic shared memory: (NO + 1) box values of T.
constexpr int kTX = 32, kTY = 8, kTZ = 4;
constexpr int kBX = kTX + 2, kBY = kTY + 2, kBZ = kTZ + 2, kBox = kBX * kBY * kBZ;

// Box row layout.  Scalar staging: kBX values from x0 - 1.  Vector staging
// (VEC: nx a multiple of 16 / sizeof(T), 16-byte aligned psi and Vc): the
// tile's kTX values sit 16-byte aligned at column vpad<T>, the halo values
// beside them, rows of kTX + 2 vpad<T> values; interior pieces are copied with
// 16-byte loads and stores.
template <typename T>
__host__ __device__ constexpr int vpad() { return 16 / (int)sizeof(T); }
template <typename T, bool VEC>
__host__ __device__ constexpr int box_pitch() { return VEC ? kTX + 2 * vpad<T>() : kBX; }
template <typename T, bool VEC>
__host__ __device__ constexpr int box_size() { return box_pitch<T, VEC>() * kBY * kBZ; }

// Tile shapes of the staged stencil up to kMaxOrb orbitals: TX x (kThreads XW / TX) x TZ
// sites, each thread XW x-neighbouring (x, y) columns of TZ sites; the tuner picks one
// per grid shape.
template <int TX, int TZ, int XW = 1>
struct PsiTile {  // XW: x-neighbouring sites per thread (TX / XW thread columns)
    static constexpr int TY = kThreads * XW / TX, BY = TY + 2, BZ = TZ + 2;
    template <typename T, bool VEC>
    __host__ __device__ static constexpr int pitch() { return VEC ? TX + 2 * vpad<T>() : TX + 2; }
    template <typename T, bool VEC>
    __host__ __device__ static constexpr int size() { return pitch<T, VEC>() * BY * BZ; }
};
// The shapes (TX, TZ, XW) the tuner tries (kPsiTileTX, kPsiTileTZ, kPsiTileXW);
// shape 0 is the default.

// 16 bytes of T from global (read-only) to shared memory.
template <typename T>
__device__ __forceinline__ void copy16(T* dst, const T* src) {
    *reinterpret_cast<float4*>(dst) = __ldg(reinterpret_cast<const float4*>(src));
}
// 16 / sizeof(T) values of Vc (FP64) as T.
template <typename T>
__device__ __forceinline__ void copy16_v(T* dst, const double* src) {
    if constexpr (sizeof(T) == 8) {
        *reinterpret_cast<double2*>(dst) = __ldg(reinterpret_cast<const double2*>(src));
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2*>(src));
        const double2 b = __ldg(reinterpret_cast<const double2*>(src + 2));
        *reinterpret_cast<float4*>(dst) = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
}
template <typename T>
__device__ __forceinline__ void zero16(T* dst) { *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f); }

// Two sites per thread take twice the accumulators and their larger boxes
// leave at most two CTAs per SM anyway: at least two resident CTAs there.
template <typename T, int NO, int XW, bool PL = false>
constexpr int psi_tile_min_blocks() {
    return (XW == 2 || PL) && psi_min_blocks<T, NO>() > 2 ? 2 : psi_min_blocks<T, NO>();
}

template <typename T, int NO, bool BATCHED, bool VEC, int TX = kTX, int TZ = kTZ, int XW = 1, bool PL = false>
__global__ void __launch_bounds__(kThreads, (psi_tile_min_blocks<T, NO, XW, PL>()))
    k_relax_psi_tile(Grid g, Coef c, RelaxIO io, Scratch sc) {
    static_assert(XW == 1 || VEC, "two sites per thread read aligned pairs: vector staging only");
    static_assert(!PL || XW == 1, "plane sums: one site per thread");
    constexpr int NP = NO * (NO + 1) / 2;
    constexpr int NL = NO > 1 ? NO * (NO - 1) / 2 : 1;
    using TS_ = PsiTile<TX, TZ, XW>;
    constexpr int TY = TS_::TY, BY = TS_::BY, BZ = TS_::BZ;
    constexpr int PX = TS_::template pitch<T, VEC>(), BOX = TS_::template size<T, VEC>();
    constexpr int XO = VEC ? vpad<T>() : 1;  // column of the tile's first x
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* box = reinterpret_cast<T*>(smem_raw);  // [NO + 1][BOX]: psi_0 .. psi_{NO-1}, then Vc
    if (BATCHED && inactive(g)) return;
    const uint32_t N = g.N;
    const size_t y = BATCHED ? sys_id() : 0;
    const T* __restrict__ pin = static_cast<const T*>(io.f_in) + y * NO * N;
    T* __restrict__ pout = static_cast<T*>(io.f_out) + y * NO * N;
    const double* __restrict__ Vc = io.V + y * N;
    T sig[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) sig[j] = (T)io.sigma_in[y * NO + j];
    const T dt = (T)c.dt;
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
    T wl[NL];
    const bool with_w = NO > 1 && io.lambda_in != nullptr;
#pragma unroll
    for (int j = 1; j < NO; ++j)
#pragma unroll
        for (int k = 0; k < j; ++k)
            wl[tri(j - 1, k)] = with_w ? (T)(-c.omega * io.lambda_in[y * NO * NO + j * NO + k]) : T(0);
    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);

    constexpr int TC = TX / XW;  // thread columns of the tile
    const int tx = threadIdx.x % TC, ty = threadIdx.x / TC;
    const int ntx = (g.nx + TX - 1) / TX, nty = (g.ny + TY - 1) / TY, ntz = (g.nz + TZ - 1) / TZ;
    const int ntiles = ntx * nty * ntz;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int bxi = tile % ntx, byi = (tile / ntx) % nty, bzi = tile / (ntx * nty);
        const int xs = bxi * TX, y0 = byi * TY - 1, z0 = bzi * TZ - 1;  // tile x start; box y, z origin
        __syncthreads();  // the previous tile's box is no longer read
        if constexpr (VEC) {
            constexpr int E = vpad<T>(), CH = TX / E, ITEMS = CH + 2;  // 16-byte pieces and the two halo values
            for (int i = threadIdx.x; i < BY * BZ * ITEMS; i += kThreads) {
                const int row = i / ITEMS, k = i - row * ITEMS;
                const int by = row % BY, bz = row / BY;
                const int gy = y0 + by, gz = z0 + bz;
                const bool rin = gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz;
                T* r = box + row * PX;
                if (k < CH) {
                    const int gx = xs + k * E;  // a whole piece is in or out: nx is a multiple of E
                    const bool in = rin && gx < g.nx;
                    const size_t gs = in ? ((size_t)gz * g.ny + gy) * g.nx + gx : 0;
#pragma unroll
                    for (int j = 0; j < NO; ++j) {
                        if (in) copy16(r + j * BOX + XO + k * E, pin + (size_t)j * N + gs);
                        else zero16(r + j * BOX + XO + k * E);
                    }
                    if (in) copy16_v(r + NO * BOX + XO + k * E, Vc + gs);
                    else zero16(r + NO * BOX + XO + k * E);
                } else {
                    const int gx = k == CH ? xs - 1 : xs + TX;
                    const int col = k == CH ? XO - 1 : XO + TX;
                    const bool in = rin && gx >= 0 && gx < g.nx;
                    const size_t gs = in ? ((size_t)gz * g.ny + gy) * g.nx + gx : 0;
#pragma unroll
                    for (int j = 0; j < NO; ++j) r[j * BOX + col] = in ? __ldg(pin + (size_t)j * N + gs) : T(0);
                    r[NO * BOX + col] = in ? (T)__ldg(Vc + gs) : T(0);
                }
            }
        } else {
            for (int i = threadIdx.x; i < BOX; i += kThreads) {
                const int bx = i % PX, by = (i / PX) % BY, bz = i / (PX * BY);
                const int gx = xs - 1 + bx, gy = y0 + by, gz = z0 + bz;
                const bool in = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz;
                const size_t gs = in ? ((size_t)gz * g.ny + gy) * g.nx + gx : 0;
#pragma unroll
                for (int j = 0; j < NO; ++j) box[j * BOX + i] = in ? __ldg(pin + (size_t)j * N + gs) : T(0);
                box[NO * BOX + i] = in ? (T)__ldg(Vc + gs) : T(0);
            }
        }
        __syncthreads();
        if constexpr (XW == 2) {
            // two x-neighbouring sites (x even): the arriving values of velocity p
            // at both sites from aligned pairs of the box row -- x-component 0:
            // the pair at the source; +1: the pair's left neighbour and its first
            // element; -1: its second element and the right neighbour's first
            using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
            auto ld2 = [&](int i) { return *reinterpret_cast<const T2*>(box + i); };
            const int gx = xs + 2 * tx, gy = y0 + 1 + ty;
#pragma unroll 1
            for (int dz = 0; dz < TZ; ++dz) {
                const int gz = z0 + 1 + dz;
                const bool live = gx < g.nx && gy < g.ny && gz < g.nz;  // nx is even here: both sites or none
                const int b = ((dz + 1) * BY + (ty + 1)) * PX + (2 * tx + XO);  // the first site in the box (even)
                T ps0[NO], ps1[NO], kx0[NO], kx1[NO];
#pragma unroll
                for (int j = 0; j < NO; ++j) ps0[j] = ps1[j] = kx0[j] = kx1[j] = T(0);
#pragma unroll
                for (int p = 0; p < 19; ++p) {
                    const int r = b - (vel(p, 1) * PX + vel(p, 2) * PX * BY);  // the source row at x-shift 0
                    const int vx = vel(p, 0);
                    auto pair = [&](int f, T& a0, T& a1) {
                        if (vx == 0) {
                            const T2 q = ld2(f * BOX + r);
                            a0 = q.x;
                            a1 = q.y;
                        } else if (vx > 0) {
                            a0 = ld2(f * BOX + r - 2).y;
                            a1 = ld2(f * BOX + r).x;
                        } else {
                            a0 = ld2(f * BOX + r).y;
                            a1 = ld2(f * BOX + r + 2).x;
                        }
                    };
                    T v0, v1;
                    pair(NO, v0, v1);
                    const T a0 = xi[vclass(p)] - dt * chi[vclass(p)] * v0;
                    const T a1 = xi[vclass(p)] - dt * chi[vclass(p)] * v1;
#pragma unroll
                    for (int j = 0; j < NO; ++j) {
                        T u0, u1;
                        pair(j, u0, u1);
                        ps0[j] += a0 * u0;
                        ps1[j] += a1 * u1;
                        kx0[j] += xi[vclass(p)] * u0;
                        kx1[j] += xi[vclass(p)] * u1;
                    }
                }
#pragma unroll
                for (int j = 0; j < NO; ++j) {
#pragma unroll
                    for (int k = 0; k < j; ++k) {
                        ps0[j] += wl[tri(j - 1, k)] * kx0[k];
                        ps1[j] += wl[tri(j - 1, k)] * kx1[k];
                    }
                    ps0[j] = live ? ps0[j] * sig[j] : T(0);
                    ps1[j] = live ? ps1[j] * sig[j] : T(0);
                }
                if (live) {
                    const size_t s = ((size_t)gz * g.ny + gy) * g.nx + gx;
#pragma unroll
                    for (int j = 0; j < NO; ++j) {
                        T2 o;
                        o.x = ps0[j];
                        o.y = ps1[j];
                        *reinterpret_cast<T2*>(pout + (size_t)j * N + s) = o;
                    }
                }
#pragma unroll
                for (int j = 0; j < NO; ++j)
#pragma unroll
                    for (int i = 0; i <= j; ++i) acc[tri(j, i)] += ps0[j] * ps0[i] + ps1[j] * ps1[i];
            }
            continue;
        }
        if constexpr (PL) {
            // plane sums: the pulled sum of a field over a velocity class is
            // rest u(r), faces Pf(z) + u(z - 1) + u(z + 1) and edges
            // Pe(z) + Pf(z - 1) + Pf(z + 1), with Pf / Pe the sums over the
            // four in-plane face / diagonal neighbours of the column in plane
            // z.  Fields: psi_j and g_j = Vc psi_j; the value and Pf of planes
            // t - 2, t - 1, t ride in registers (slot t % 3) down the column.
            const int gx = xs + tx, gy = y0 + 1 + ty;
            const int c0 = (ty + 1) * PX + (tx + XO);  // the column in box plane 0
            const T* vb = box + NO * BOX;
            T u0[3][NO], uf[3][NO], g0[3][NO], gf[3][NO];
#pragma unroll
            for (int t = 0; t < TZ + 2; ++t) {
                const int k = t % 3, cp = t * BY * PX + c0;
                {
                    const T v0 = vb[cp], vw = vb[cp - 1], ve = vb[cp + 1], vs = vb[cp - PX], vn = vb[cp + PX];
#pragma unroll
                    for (int j = 0; j < NO; ++j) {
                        const T* f = box + j * BOX;
                        const T a0 = f[cp], aw = f[cp - 1], ae = f[cp + 1], as = f[cp - PX], an = f[cp + PX];
                        u0[k][j] = a0;
                        uf[k][j] = (aw + ae) + (as + an);
                        g0[k][j] = v0 * a0;
                        gf[k][j] = (vw * aw + ve * ae) + (vs * as + vn * an);
                    }
                }
                if (t < 2) continue;
                // output: box plane t - 1, grid plane z0 + t - 1
                const int km = (t - 2) % 3, kc = (t - 1) % 3, kp = k, cc = (t - 1) * BY * PX + c0;
                const int gz = z0 + t - 1;
                const bool live = gx < g.nx && gy < g.ny && gz < g.nz;
                const T dsw = vb[cc - 1 - PX], dse = vb[cc + 1 - PX], dnw = vb[cc - 1 + PX], dne = vb[cc + 1 + PX];
                T ps[NO], kx[NO];
#pragma unroll
                for (int j = 0; j < NO; ++j) {
                    const T* f = box + j * BOX;
                    const T bsw = f[cc - 1 - PX], bse = f[cc + 1 - PX], bnw = f[cc - 1 + PX], bne = f[cc + 1 + PX];
                    const T ue = (bsw + bse) + (bnw + bne);
                    const T ge = (dsw * bsw + dse * bse) + (dnw * bnw + dne * bne);
                    const T uF = uf[kc][j] + (u0[km][j] + u0[kp][j]);
                    const T uE = ue + (uf[km][j] + uf[kp][j]);
                    const T gF = gf[kc][j] + (g0[km][j] + g0[kp][j]);
                    const T gE = ge + (gf[km][j] + gf[kp][j]);
                    kx[j] = xi[0] * u0[kc][j] + xi[1] * uF + xi[2] * uE;
                    ps[j] = kx[j] - dt * (chi[0] * g0[kc][j] + chi[1] * gF + chi[2] * gE);
                }
#pragma unroll
                for (int j = 0; j < NO; ++j) {
#pragma unroll
                    for (int i = 0; i < j; ++i) ps[j] += wl[tri(j - 1, i)] * kx[i];
                    ps[j] = live ? ps[j] * sig[j] : T(0);
                }
                if (live) {
                    const size_t s = ((size_t)gz * g.ny + gy) * g.nx + gx;
#pragma unroll
                    for (int j = 0; j < NO; ++j) pout[(size_t)j * N + s] = ps[j];
                }
#pragma unroll
                for (int j = 0; j < NO; ++j)
#pragma unroll
                    for (int i = 0; i <= j; ++i) acc[tri(j, i)] += ps[j] * ps[i];
            }
            continue;
        }
        const int gx = xs + tx, gy = y0 + 1 + ty;
#pragma unroll 1
        for (int dz = 0; dz < TZ; ++dz) {
            const int gz = z0 + 1 + dz;
            const bool live = gx < g.nx && gy < g.ny && gz < g.nz;
            const int b = ((dz + 1) * BY + (ty + 1)) * PX + (tx + XO);  // the site in the box
            T ps[NO], kx[NO];
#pragma unroll
            for (int j = 0; j < NO; ++j) ps[j] = kx[j] = T(0);
#pragma unroll
            for (int p = 0; p < 19; ++p) {
                const int src = b - (vel(p, 0) + vel(p, 1) * PX + vel(p, 2) * PX * BY);
                const T a = xi[vclass(p)] - dt * chi[vclass(p)] * box[NO * BOX + src];
#pragma unroll
                for (int j = 0; j < NO; ++j) {
                    const T v = box[j * BOX + src];
                    ps[j] += a * v;
                    kx[j] += xi[vclass(p)] * v;
                }
            }
#pragma unroll
            for (int j = 0; j < NO; ++j) {
#pragma unroll
                for (int k = 0; k < j; ++k) ps[j] += wl[tri(j - 1, k)] * kx[k];
                ps[j] = live ? ps[j] * sig[j] : T(0);
            }
            if (live) {
                const size_t s = ((size_t)gz * g.ny + gy) * g.nx + gx;
#pragma unroll
                for (int j = 0; j < NO; ++j) pout[(size_t)j * N + s] = ps[j];
            }
#pragma unroll
            for (int j = 0; j < NO; ++j)
#pragma unroll
                for (int i = 0; i <= j; ++i) acc[tri(j, i)] += ps[j] * ps[i];
        }
    }
    double v[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) v[k] = (double)acc[k];
    double* partial = sc.partial + y * sc.max_blocks * sc.max_vals;
    block_sum_store<NP>(v, partial + (size_t)blockIdx.x * NP);
    __shared__ double tot[NP];
    if (grid_total<NP>(partial, sc.counter + y, tot) && threadIdx.x == 0)
        store_overlap(tot, NO, c.h, io.S_out + y * NO * NO, io.lambda_out + y * NO * NO, io.sigma_out + y * NO);
}

template <typename T, int NO, bool BATCHED, bool VEC, int TX, int TZ, int XW = 1, bool PL = false>
cudaError_t launch_relax_psi_tile_v(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                    cudaStream_t st) {
    auto kern = k_relax_psi_tile<T, NO, BATCHED, VEC, TX, TZ, XW, PL>;
    using TS_ = PsiTile<TX, TZ, XW>;
    const size_t smem = (size_t)(NO + 1) * TS_::template size<T, VEC>() * sizeof(T);
    // opted in whatever the size: static and dynamic shared memory together may exceed 48 KB
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, smem) != cudaSuccess || nb < 1) nb = 1;
    if (sc.max_vals < NO * (NO + 1) / 2 || sc.systems < B) return cudaErrorInvalidValue;
    const size_t tiles =
        (size_t)((g.nx + TX - 1) / TX) * ((g.ny + TS_::TY - 1) / TS_::TY) * ((g.nz + TZ - 1) / TZ);
    const int per = std::max(1, std::min(sc.max_blocks, nb * num_sms() / std::max(B, 1)));
    kern<<<dim3((unsigned)std::min<size_t>(tiles, (size_t)per), (unsigned)B), kThreads, smem, st>>>(g, c, io, sc);
    count_launches(1);
    return cudaGetLastError();
}

// Vector staging where rows are whole 16-byte pieces and the arrays (psi in
// and out, Vc) 16-byte aligned.
// Shapes other than the default run with vector staging only; where it does
// not apply (rows not of whole 16-byte pieces, unaligned arrays) the default
// shape's scalar staging runs, and so does the default shape where another's
// box would not fit in a block's shared memory (FP64, many orbitals) or whose
// two sites per thread would not fit the registers (psi_tile_runs).
template <typename T, int NO, bool BATCHED, int K>
cudaError_t launch_relax_psi_tile_k(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                    cudaStream_t st) {
    if constexpr (K > 0 && psi_tile_runs((int)sizeof(T), NO, K))
        return launch_relax_psi_tile_v<T, NO, BATCHED, true, kPsiTileTX[K], kPsiTileTZ[K], kPsiTileXW[K],
                                       kPsiTilePL[K]>(g, c, io, sc, B, st);
    else
        return launch_relax_psi_tile_v<T, NO, BATCHED, true, kPsiTileTX[0], kPsiTileTZ[0]>(g, c, io, sc, B, st);
}
template <typename T, int NO, bool BATCHED>
cudaError_t launch_relax_psi_tile(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                  int shape, cudaStream_t st) {
    auto al = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    // the output too: the two-site shapes store pairs of values
    if (!(g.nx % vpad<T>() == 0 && al(io.f_in) && al(io.V) && al(io.f_out)))
        return launch_relax_psi_tile_v<T, NO, BATCHED, false, kPsiTileTX[0], kPsiTileTZ[0]>(g, c, io, sc, B, st);
    switch (shape) {
        case 1: return launch_relax_psi_tile_k<T, NO, BATCHED, 1>(g, c, io, sc, B, st);
        case 2: return launch_relax_psi_tile_k<T, NO, BATCHED, 2>(g, c, io, sc, B, st);
        case 3: return launch_relax_psi_tile_k<T, NO, BATCHED, 3>(g, c, io, sc, B, st);
        case 4: return launch_relax_psi_tile_k<T, NO, BATCHED, 4>(g, c, io, sc, B, st);
        case 5: return launch_relax_psi_tile_k<T, NO, BATCHED, 5>(g, c, io, sc, B, st);
        case 6: return launch_relax_psi_tile_k<T, NO, BATCHED, 6>(g, c, io, sc, B, st);
        case 7: return launch_relax_psi_tile_k<T, NO, BATCHED, 7>(g, c, io, sc, B, st);
        default: return launch_relax_psi_tile_k<T, NO, BATCHED, 0>(g, c, io, sc, B, st);
    }
}

// Explicit instantiations of the staged kernels' launchers for one value
// type (PREFIX extern: declared only, so that a unit that dispatches to them
// leaves their compilation to the unit that instantiates them).
#define LBKS_PSI_TILE_INST(PREFIX, T)                                                                            \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 1, false>(const Grid&, const Coef&, const RelaxIO&,    \
                                                                   const Scratch&, int, int, cudaStream_t);      \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 2, false>(const Grid&, const Coef&, const RelaxIO&,    \
                                                                   const Scratch&, int, int, cudaStream_t);      \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 3, false>(const Grid&, const Coef&, const RelaxIO&,    \
                                                                   const Scratch&, int, int, cudaStream_t);      \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 4, false>(const Grid&, const Coef&, const RelaxIO&,    \
                                                                   const Scratch&, int, int, cudaStream_t);      \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 5, false>(const Grid&, const Coef&, const RelaxIO&,    \
                                                                   const Scratch&, int, int, cudaStream_t);      \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 6, false>(const Grid&, const Coef&, const RelaxIO&,    \
                                                                   const Scratch&, int, int, cudaStream_t);      \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 7, false>(const Grid&, const Coef&, const RelaxIO&,    \
                                                                   const Scratch&, int, int, cudaStream_t);      \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 8, false>(const Grid&, const Coef&, const RelaxIO&,    \
                                                                   const Scratch&, int, int, cudaStream_t);      \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 1, true>(const Grid&, const Coef&, const RelaxIO&,     \
                                                                  const Scratch&, int, int, cudaStream_t);       \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 2, true>(const Grid&, const Coef&, const RelaxIO&,     \
                                                                  const Scratch&, int, int, cudaStream_t);       \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 3, true>(const Grid&, const Coef&, const RelaxIO&,     \
                                                                  const Scratch&, int, int, cudaStream_t);       \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 4, true>(const Grid&, const Coef&, const RelaxIO&,     \
                                                                  const Scratch&, int, int, cudaStream_t);       \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 5, true>(const Grid&, const Coef&, const RelaxIO&,     \
                                                                  const Scratch&, int, int, cudaStream_t);       \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 6, true>(const Grid&, const Coef&, const RelaxIO&,     \
                                                                  const Scratch&, int, int, cudaStream_t);       \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 7, true>(const Grid&, const Coef&, const RelaxIO&,     \
                                                                  const Scratch&, int, int, cudaStream_t);       \
    PREFIX template cudaError_t launch_relax_psi_tile<T, 8, true>(const Grid&, const Coef&, const RelaxIO&,     \
                                                                  const Scratch&, int, int, cudaStream_t);

// More than kMaxOrb orbitals, staged in shared memory: a block takes one
// tile and one group of up to kPsiGroup orbitals of one system (blockIdx.y =
// system * groups + group), stages the group's psi and W field and Vc with a
// one-site halo, and writes psi'; the overlap follows in its own kernel.
// Dynamic shared memory: (2 kPsiGroup + 1) box values of T.
template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads, 3) k_relax_psi_wide_tile(Grid g, Coef c, RelaxIO io, int NO) {
    constexpr int PX = box_pitch<T, VEC>(), BOX = box_size<T, VEC>();
    constexpr int XO = VEC ? vpad<T>() : 1;  // column of the tile's first x
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* box = reinterpret_cast<T*>(smem_raw);  // [kPsiGroup psi][kPsiGroup u][Vc], BOX each
    const int groups = (NO + kPsiGroup - 1) / kPsiGroup;
    const int y = (int)blockIdx.y / groups, jg = (int)blockIdx.y - y * groups;
    if (g.active && !g.active[y]) return;
    const size_t N = g.N;
    const int j0 = jg * kPsiGroup, J = min(kPsiGroup, NO - j0);
    const T* __restrict__ pin = static_cast<const T*>(io.f_in) + ((size_t)y * NO + j0) * N;
    const T* uw = static_cast<const T*>(io.u_in);
    // W field of orbital j (j >= 1): u + (y (NO - 1) + j - 1) N
    const T* ubase = uw ? uw + (size_t)y * (NO - 1) * N : nullptr;
    const double* __restrict__ Vc = io.V + (size_t)y * N;
    const T dt = (T)c.dt;
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    const int ntx = (g.nx + kTX - 1) / kTX, nty = (g.ny + kTY - 1) / kTY;
    const int tile = blockIdx.x;
    const int bxi = tile % ntx, byi = (tile / ntx) % nty, bzi = tile / (ntx * nty);
    const int xs = bxi * kTX, y0 = byi * kTY - 1, z0 = bzi * kTZ - 1;
    // the array staged in box slot a (0 .. 2 kPsiGroup - 1), or null for zeros
    auto source = [&](int a) -> const T* {
        if (a < kPsiGroup) return a < J ? pin + (size_t)a * N : nullptr;
        const int j = a - kPsiGroup, jj = j0 + j;  // the W field exists for orbitals >= 1
        return (j < J && ubase && jj > 0) ? ubase + (size_t)(jj - 1) * N : nullptr;
    };
    if constexpr (VEC) {
        constexpr int E = vpad<T>(), CH = kTX / E, ITEMS = CH + 2;  // 16-byte pieces and the two halo values
        for (int i = threadIdx.x; i < kBY * kBZ * ITEMS; i += kThreads) {
            const int row = i / ITEMS, k = i - row * ITEMS;
            const int by = row % kBY, bz = row / kBY;
            const int gy = y0 + by, gz = z0 + bz;
            const bool rin = gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz;
            T* r = box + row * PX;
            if (k < CH) {
                const int gx = xs + k * E;  // a whole piece is in or out: nx is a multiple of E
                const bool in = rin && gx < g.nx;
                const size_t gs = in ? ((size_t)gz * g.ny + gy) * g.nx + gx : 0;
#pragma unroll
                for (int a = 0; a < 2 * kPsiGroup; ++a) {
                    const T* src = source(a);
                    if (in && src) copy16(r + a * BOX + XO + k * E, src + gs);
                    else zero16(r + a * BOX + XO + k * E);
                }
                if (in) copy16_v(r + 2 * kPsiGroup * BOX + XO + k * E, Vc + gs);
                else zero16(r + 2 * kPsiGroup * BOX + XO + k * E);
            } else {
                const int gx = k == CH ? xs - 1 : xs + kTX;
                const int col = k == CH ? XO - 1 : XO + kTX;
                const bool in = rin && gx >= 0 && gx < g.nx;
                const size_t gs = in ? ((size_t)gz * g.ny + gy) * g.nx + gx : 0;
#pragma unroll
                for (int a = 0; a < 2 * kPsiGroup; ++a) {
                    const T* src = source(a);
                    r[a * BOX + col] = (in && src) ? __ldg(src + gs) : T(0);
                }
                r[2 * kPsiGroup * BOX + col] = in ? (T)__ldg(Vc + gs) : T(0);
            }
        }
    } else {
        for (int i = threadIdx.x; i < BOX; i += kThreads) {
            const int bx = i % PX, by = (i / PX) % kBY, bz = i / (PX * kBY);
            const int gx = xs - 1 + bx, gy = y0 + by, gz = z0 + bz;
            const bool in = gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz;
            const size_t gs = in ? ((size_t)gz * g.ny + gy) * g.nx + gx : 0;
#pragma unroll
            for (int a = 0; a < 2 * kPsiGroup; ++a) {
                const T* src = source(a);
                box[a * BOX + i] = (in && src) ? __ldg(src + gs) : T(0);
            }
            box[2 * kPsiGroup * BOX + i] = in ? (T)__ldg(Vc + gs) : T(0);
        }
    }
    __syncthreads();
    const int gx = xs + tx, gy = y0 + 1 + ty;
#pragma unroll 1
    for (int dz = 0; dz < kTZ; ++dz) {
        const int gz = z0 + 1 + dz;
        if (gx >= g.nx || gy >= g.ny || gz >= g.nz) continue;
        const int b = ((dz + 1) * kBY + (ty + 1)) * PX + (tx + XO);
        T ps[kPsiGroup];
#pragma unroll
        for (int j = 0; j < kPsiGroup; ++j) ps[j] = T(0);
#pragma unroll
        for (int p = 0; p < 19; ++p) {
            const int src = b - (vel(p, 0) + vel(p, 1) * PX + vel(p, 2) * PX * kBY);
            const T a = xi[vclass(p)] - dt * chi[vclass(p)] * box[2 * kPsiGroup * BOX + src];
#pragma unroll
            for (int j = 0; j < kPsiGroup; ++j)
                ps[j] += a * box[j * BOX + src] + xi[vclass(p)] * box[(kPsiGroup + j) * BOX + src];
        }
        const size_t s = ((size_t)gz * g.ny + gy) * g.nx + gx;
        const size_t o0 = (size_t)y * NO + j0;
#pragma unroll
        for (int j = 0; j < kPsiGroup; ++j)
            if (j < J) static_cast<T*>(io.f_out)[(o0 + j) * N + s] = (T)io.sigma_in[o0 + j] * ps[j];
    }
}

// The same step marching along z: a block owns a 32 x 8 column of sites and
// a run of zc planes, and keeps the planes z - 1, z, z + 1 of every orbital's
// psi and of Vc (one-site x and y halo, zero outside the grid) in a ring of
// four shared-memory planes.  While it sums the stencil of plane z it has
// the loads of plane z + 2 in flight in registers, and stores them into the
// ring slot that plane z - 2 held; one barrier per plane.  Every plane is
// loaded once per run (zc + 2 planes for zc outputs) instead of three times
// per 4-plane tile, and no thread waits for a whole box before it computes.
// Up to kMaxOrb orbitals; W source, overlap partials, Lambda and sigma as in
// k_relax_psi_tile.  Dynamic shared memory: 4 (NO + 1) 34 x 10 values of T.
constexpr int kZmW = kTX + 2, kZmH = kTY + 2, kZmPlane = kZmW * kZmH;

template <typename T, int NO, bool BATCHED>
__global__ void __launch_bounds__(kThreads, (psi_min_blocks<T, NO>())) k_relax_psi_zm(Grid g, Coef c, RelaxIO io,
                                                                                       Scratch sc, int zc) {
    constexpr int NP = NO * (NO + 1) / 2;
    constexpr int NL = NO > 1 ? NO * (NO - 1) / 2 : 1;
    constexpr int PT = (NO + 1) * kZmPlane;         // values of one plane of the ring (psi_0 .. psi_{NO-1}, Vc)
    constexpr int K = (PT + kThreads - 1) / kThreads;  // of them loaded by each thread
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ring = reinterpret_cast<T*>(smem_raw);  // [4][PT]
    if (BATCHED && inactive(g)) return;
    const uint32_t N = g.N;
    const size_t y = BATCHED ? sys_id() : 0;
    const T* __restrict__ pin = static_cast<const T*>(io.f_in) + y * NO * N;
    T* __restrict__ pout = static_cast<T*>(io.f_out) + y * NO * N;
    const double* __restrict__ Vc = io.V + y * N;
    T sig[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) sig[j] = (T)io.sigma_in[y * NO + j];
    const T dt = (T)c.dt;
    const T xi[3] = {(T)c.xi[0], (T)c.xi[1], (T)c.xi[2]};
    const T chi[3] = {(T)c.chi[0], (T)c.chi[1], (T)c.chi[2]};
    T wl[NL];
    const bool with_w = NO > 1 && io.lambda_in != nullptr;
#pragma unroll
    for (int j = 1; j < NO; ++j)
#pragma unroll
        for (int k = 0; k < j; ++k)
            wl[tri(j - 1, k)] = with_w ? (T)(-c.omega * io.lambda_in[y * NO * NO + j * NO + k]) : T(0);
    T acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = T(0);

    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    const int ntx = (g.nx + kTX - 1) / kTX, nty = (g.ny + kTY - 1) / kTY, nzc = (g.nz + zc - 1) / zc;
    const int items = ntx * nty * nzc;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int bxi = item % ntx, byi = (item / ntx) % nty, bzi = item / (ntx * nty);
        const int x0 = bxi * kTX, y0 = byi * kTY, zs = bzi * zc, ze = min(zs + zc, g.nz);
        // value i of plane z of the ring (zero outside the grid)
        auto fetch = [&](int z, int i) -> T {
            const int a = i / kZmPlane, e = i - a * kZmPlane;
            const int gx = x0 - 1 + e % kZmW, gy = y0 - 1 + e / kZmW;
            if (z < 0 || z >= g.nz || gx < 0 || gx >= g.nx || gy < 0 || gy >= g.ny) return T(0);
            const size_t gs = ((size_t)z * g.ny + gy) * g.nx + gx;
            return a < NO ? __ldg(pin + (size_t)a * N + gs) : (T)__ldg(Vc + gs);
        };
        auto slot = [&](int z) { return ring + (size_t)((z - zs + 1) & 3) * PT; };
        __syncthreads();  // the previous run's ring is no longer read
        for (int z = zs - 1; z <= zs + 1; ++z) {
            T* r = slot(z);
            for (int i = threadIdx.x; i < PT; i += kThreads) r[i] = fetch(z, i);
        }
        __syncthreads();
        const int gx = x0 + tx, gy = y0 + ty;
        const bool col = gx < g.nx && gy < g.ny;
        const int b = (ty + 1) * kZmW + (tx + 1);  // the site in a plane
#pragma unroll 1
        for (int z = zs; z < ze; ++z) {
            // plane z + 2 (needed while z + 1 < ze) in flight during this plane's sums
            T pre[K];
            const bool next = z + 2 <= ze;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int i = (int)threadIdx.x + k * kThreads;
                pre[k] = (next && i < PT) ? fetch(z + 2, i) : T(0);
            }
            const T* pm = slot(z - 1);
            const T* p0 = slot(z);
            const T* pp = slot(z + 1);
            T ps[NO], kx[NO];
#pragma unroll
            for (int j = 0; j < NO; ++j) ps[j] = kx[j] = T(0);
#pragma unroll
            for (int p = 0; p < 19; ++p) {
                const T* pl = vel(p, 2) > 0 ? pm : vel(p, 2) < 0 ? pp : p0;  // source plane z - vz
                const int src = b - (vel(p, 0) + vel(p, 1) * kZmW);
                const T a = xi[vclass(p)] - dt * chi[vclass(p)] * pl[NO * kZmPlane + src];
#pragma unroll
                for (int j = 0; j < NO; ++j) {
                    const T v = pl[j * kZmPlane + src];
                    ps[j] += a * v;
                    kx[j] += xi[vclass(p)] * v;
                }
            }
#pragma unroll
            for (int j = 0; j < NO; ++j) {
#pragma unroll
                for (int k = 0; k < j; ++k) ps[j] += wl[tri(j - 1, k)] * kx[k];
                ps[j] = col ? ps[j] * sig[j] : T(0);
            }
            if (col) {
                const size_t s = ((size_t)z * g.ny + gy) * g.nx + gx;
#pragma unroll
                for (int j = 0; j < NO; ++j) pout[(size_t)j * N + s] = ps[j];
            }
#pragma unroll
            for (int j = 0; j < NO; ++j)
#pragma unroll
                for (int i = 0; i <= j; ++i) acc[tri(j, i)] += ps[j] * ps[i];
            if (next) {
                T* r = slot(z + 2);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int i = (int)threadIdx.x + k * kThreads;
                    if (i < PT) r[i] = pre[k];
                }
            }
            __syncthreads();
        }
    }
    double v[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) v[k] = (double)acc[k];
    double* partial = sc.partial + y * sc.max_blocks * sc.max_vals;
    block_sum_store<NP>(v, partial + (size_t)blockIdx.x * NP);
    __shared__ double tot[NP];
    if (grid_total<NP>(partial, sc.counter + y, tot) && threadIdx.x == 0)
        store_overlap(tot, NO, c.h, io.S_out + y * NO * NO, io.lambda_out + y * NO * NO, io.sigma_out + y * NO);
}

// One run per block where the overlap scratch allows (the hardware balances
// the blocks): runs of at least 8 planes, as many runs as the scratch's
// blocks per system hold.
template <typename T, int NO, bool BATCHED>
cudaError_t launch_relax_psi_zm(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                                cudaStream_t st) {
    auto kern = k_relax_psi_zm<T, NO, BATCHED>;
    const size_t smem = (size_t)4 * (NO + 1) * kZmPlane * sizeof(T);
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return attr;
    if (sc.max_vals < NO * (NO + 1) / 2 || sc.systems < B) return cudaErrorInvalidValue;
    const int columns = ((g.nx + kTX - 1) / kTX) * ((g.ny + kTY - 1) / kTY);
    const int runs = std::max(1, sc.max_blocks / columns);  // runs along z the scratch allows per column
    const int zc = std::max(8, (g.nz + runs - 1) / runs);
    const size_t items = (size_t)columns * ((g.nz + zc - 1) / zc);
    kern<<<dim3((unsigned)std::min<size_t>(items, (size_t)sc.max_blocks), (unsigned)B), kThreads, smem, st>>>(g, c, io,
                                                                                                          sc, zc);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, int NO, bool BATCHED>
cudaError_t launch_relax_psi_n(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                               cudaStream_t st) {
    auto kern = k_relax_psi<T, NO, BATCHED>;
    static const int nb = blocks_per_sm(kern);
    if (sc.max_vals < NO * (NO + 1) / 2 || sc.systems < B) return cudaErrorInvalidValue;
    kern<<<batch_grid(g.N, nb * num_sms(), B, sc.max_blocks), kThreads, 0, st>>>(g, c, io, sc);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace lbks

#include "lbks_psi_tma.cuh"

namespace lbks {

template <typename T>
cudaError_t launch_relax_psi(int NO, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                             int kernel, cudaStream_t st) {
    const int shape = (kernel >> kPsiShapeShift) & 0xff;  // the staged kernel's tile shape
    kernel &= (1 << kPsiShapeShift) - 1;
    if (kernel == kPsiKernelTma) return launch_relax_psi_tma<T>(NO, g, c, io, sc, B, st);
    const bool tiled = kernel == kPsiKernelTiled || (kernel == kPsiKernelZ && NO > kMaxOrb);
    const bool zmarch = kernel == kPsiKernelZ && NO <= kMaxOrb;
    if (NO > kMaxOrb) {
        const size_t groups = (NO + kPsiGroup - 1) / kPsiGroup;
        if (groups * B > 65535) return cudaErrorInvalidConfiguration;
        if (tiled) {
            // scalar staging: the 16-byte layout's padded rows (9 x 9.6 KB of FP32 boxes)
            // leave two blocks per SM instead of three, which measured slower
            auto kern = k_relax_psi_wide_tile<T, false>;
            const size_t smem = (size_t)(2 * kPsiGroup + 1) * box_size<T, false>() * sizeof(T);
            static const cudaError_t attr_s =
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (attr_s != cudaSuccess) return attr_s;
            const size_t tiles =
                (size_t)((g.nx + kTX - 1) / kTX) * ((g.ny + kTY - 1) / kTY) * ((g.nz + kTZ - 1) / kTZ);
            kern<<<dim3((unsigned)tiles, (unsigned)(groups * B)), kThreads, smem, st>>>(g, c, io, NO);
            count_launches(1);
            return cudaGetLastError();
        }
        k_relax_psi_wide<T><<<dim3((g.N + kThreads - 1) / kThreads, (unsigned)(groups * B)), kThreads, 0, st>>>(
            g, c, io, NO);
        count_launches(1);
        return cudaGetLastError();
    }
    const bool b = B > 1;
    switch (NO) {
#define LBKS_CASE(n)                                                                                  \
    case n:                                                                                           \
        if (zmarch)                                                                                   \
            return b ? launch_relax_psi_zm<T, n, true>(g, c, io, sc, B, st)                           \
                     : launch_relax_psi_zm<T, n, false>(g, c, io, sc, B, st);                         \
        if (tiled)                                                                                    \
            return b ? launch_relax_psi_tile<T, n, true>(g, c, io, sc, B, shape, st)                  \
                     : launch_relax_psi_tile<T, n, false>(g, c, io, sc, B, shape, st);                \
        return b ? launch_relax_psi_n<T, n, true>(g, c, io, sc, B, st) : launch_relax_psi_n<T, n, false>(g, c, io, sc, B, st);
        LBKS_CASE(1) LBKS_CASE(2) LBKS_CASE(3) LBKS_CASE(4) LBKS_CASE(5) LBKS_CASE(6) LBKS_CASE(7) LBKS_CASE(8)
#undef LBKS_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbks
