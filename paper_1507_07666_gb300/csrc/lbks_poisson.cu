// Hartree potential: the 7-point lattice Poisson problem
//   (A v)(r) = 6 v(r) - sum of the six face neighbours = 4 pi h^2 rho(r) + ghost values
// solved by conjugate gradients in FP64 preconditioned with one geometric
// multigrid V-cycle in FP32 (scalars resident on the device).  GB300 issues
// FP64 at a small fraction of its FP32 rate, and the smoothing sweeps are
// ALU-bound in FP64; the preconditioner needs no more than single precision,
// since the FP64 iteration computes the residual and the solution.  Its
// rounding makes the preconditioner vary slightly between applications, so
// the direction update takes the flexible (Polak-Ribiere) form
// beta = <z_new, r_new - r_old> / <z_old, r_old> = -alpha <z_new, A p_old> / <z_old, r_old>.
//
// Multigrid hierarchy: coarse point I of a level sits on fine index 2I+1 of
// the level above (m = n/2 points per axis); coarsening stops when an axis
// would drop below 2 points.  Prolongation P is trilinear interpolation with
// zero ghosts, restriction is P^T, and the operator of level l is the
// rediscretised 2^l (6 - sum of neighbours), the Galerkin product's
// long-wavelength limit.  Smoothing is red-black Gauss-Seidel, red then
// black before the coarse correction and black then red after it, with the
// coarsest level solved by a fixed number of such sweeps: in exact
// arithmetic the V-cycle is a fixed symmetric positive definite operator.
#include "lbks_internal.cuh"
#include "lbks_reduce.cuh"

#include <algorithm>

namespace lbks {

namespace {

// Tuning knobs (set by measurement): red-black sweeps before the coarse
// correction (and after it), and the largest level the one-CTA tail takes.
#ifndef LBKS_MG_PRE
#define LBKS_MG_PRE 2
#endif
#ifndef LBKS_MG_TAIL_SITES
#define LBKS_MG_TAIL_SITES 4096
#endif
constexpr int kPre = LBKS_MG_PRE;
constexpr int kCoarse = 4;    // sweeps each way on the coarsest level (the flexible CG takes an inexact solve)
constexpr uint32_t kCoarseSites = 4096;  // coarsest levels up to this size are solved by one CTA

int grid_for(size_t n, int cap_blocks) {
    const size_t need = (n + kThreads - 1) / kThreads;
    return (int)std::max<size_t>(1, std::min<size_t>(need, (size_t)cap_blocks));
}

// Blocks per system of a reduction kernel over B systems.
int red_cap(const Scratch& sc, int vals, int B) {
    if (sc.max_vals < vals || sc.systems < B) return 0;
    return std::max(1, std::min(sc.max_blocks, num_sms() * 4 / std::max(B, 1)));
}

__device__ __forceinline__ void decode3(const Grid& g, uint32_t s, int& x, int& y, int& z) {
    const uint32_t q = g.divx.div(s);
    x = (int)(s - q * (uint32_t)g.nx);
    const uint32_t zz = g.divy.div(q);
    y = (int)(q - zz * (uint32_t)g.ny);
    z = (int)zz;
}

// 6 v(s) - sum of in-grid face neighbours
template <typename V>
__device__ __forceinline__ V stencil(const Grid& g, const V* __restrict__ v, uint32_t s, int x, int y, int z,
                                     V self) {
    const int sy = g.nx, sz = g.nx * g.ny;
    V t = V(6) * self;
    if (x > 0) t -= v[s - 1];
    if (x < g.nx - 1) t -= v[s + 1];
    if (y > 0) t -= v[s - sy];
    if (y < g.ny - 1) t -= v[s + sy];
    if (z > 0) t -= v[s - sz];
    if (z < g.nz - 1) t -= v[s + sz];
    return t;
}

// Sum of the in-grid face neighbours of site s (the site's own value is not
// read: a red-black half-sweep may find it stale).
__device__ __forceinline__ float nb_sum(const Grid& g, const float* __restrict__ v, uint32_t s, int x, int y, int z) {
    const int sy = g.nx, sz = g.nx * g.ny;
    float t = 0.0f;
    if (x > 0) t += v[s - 1];
    if (x < g.nx - 1) t += v[s + 1];
    if (y > 0) t += v[s - sy];
    if (y < g.ny - 1) t += v[s + sy];
    if (z > 0) t += v[s - sz];
    if (z < g.nz - 1) t += v[s + sz];
    return t;
}

// The system's slice of the PCG vectors and scalars.
__device__ __forceinline__ PoissonBufs at_sys(PoissonBufs pb, size_t N) {
    const size_t o = (size_t)blockIdx.y * N;
    pb.b += o; pb.r += o; pb.p += o; pb.ap += o; pb.z += o; pb.tmp += o;
    if (pb.r32) pb.r32 += o;
    if (pb.x32) pb.x32 += o;
    pb.cg += blockIdx.y;
    pb.mp += (size_t)blockIdx.y * kMpStride;
    return pb;
}

__device__ __forceinline__ double multipole_value(const double* mp, double X, double Y, double Z) {
    const double r2 = X * X + Y * Y + Z * Z;
    const double r = sqrt(r2);
    double v = mp[0] / r;
    v += (mp[1] * X + mp[2] * Y + mp[3] * Z) / (r2 * r);
    const double quad = mp[4] * X * X + mp[5] * Y * Y + mp[6] * Z * Z +
                        2.0 * (mp[7] * X * Y + mp[8] * X * Z + mp[9] * Y * Z);
    return v + 0.5 * quad / (r2 * r2 * r);
}

// ------------------------------------------------------------ multigrid kernels
// One colour of red-black Gauss-Seidel on A_l = scale (6 - sum nb):
// x = (b + scale * sum nb x) / (6 scale) at sites with (x+y+z) % 2 == colour.
// Slot k of a launch addresses the colour's site x = 2m + ((colour + y + z) & 1)
// of row (y, z), m = k mod hx, hx = ceil(nx / 2) slots per row (divh divides by hx).
// The update reads only the other colour; from_zero: the level starts at x = 0,
// so the sweep is x = b / (6 scale) and no neighbour is read.
__device__ __forceinline__ bool colour_site(const Grid& g, const FastDiv& divh, uint32_t k, int colour, int& ix,
                                            int& iy, int& iz, uint32_t& s) {
    const uint32_t q = divh.div(k);
    const int m = (int)(k - q * divh.d);
    const uint32_t zz = g.divy.div(q);
    iy = (int)(q - zz * (uint32_t)g.ny);
    iz = (int)zz;
    ix = 2 * m + ((colour + iy + iz) & 1);
    if (ix >= g.nx) return false;
    s = ((uint32_t)iz * (uint32_t)g.ny + (uint32_t)iy) * (uint32_t)g.nx + (uint32_t)ix;
    return true;
}

__global__ void __launch_bounds__(kThreads) k_mg_smooth(Grid g, FastDiv divh, float scale, int colour, int from_zero,
                                                        float* __restrict__ x, const float* __restrict__ b,
                                                        const CGState* cg) {
    if (inactive(g) || cg[blockIdx.y].done) return;
    x += (size_t)blockIdx.y * g.N;
    b += (size_t)blockIdx.y * g.N;
    const float inv = 1.0f / (6.0f * scale);
    const uint32_t slots = divh.d * (uint32_t)g.ny * (uint32_t)g.nz;
    for (uint32_t k = blockIdx.x * kThreads + threadIdx.x; k < slots; k += gridDim.x * kThreads) {
        int ix, iy, iz;
        uint32_t s;
        if (!colour_site(g, divh, k, colour, ix, iy, iz, s)) continue;
        if (from_zero) {
            x[s] = b[s] * inv;
            continue;
        }
        const float nb = nb_sum(g, x, s, ix, iy, iz);
        x[s] = (b[s] + scale * nb) * inv;
    }
}
// r = b - A_l x
__global__ void __launch_bounds__(kThreads) k_mg_residual(Grid g, float scale, const float* __restrict__ x,
                                                          const float* __restrict__ b, float* __restrict__ r,
                                                          const CGState* cg) {
    if (inactive(g) || cg[blockIdx.y].done) return;
    x += (size_t)blockIdx.y * g.N;
    b += (size_t)blockIdx.y * g.N;
    r += (size_t)blockIdx.y * g.N;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads) {
        int ix, iy, iz;
        decode3(g, s, ix, iy, iz);
        r[s] = b[s] - scale * stencil(g, x, s, ix, iy, iz, x[s]);
    }
}

// b_c(I) = sum over the 27 fine neighbours of fine point 2I+1 with weights
// prod_axis (1 at the centre, 1/2 beside it)  (= P^T r)
__global__ void __launch_bounds__(kThreads) k_mg_restrict(Grid gf, Grid gc, const float* __restrict__ rf,
                                                          float* __restrict__ bc, const CGState* cg) {
    if (inactive(gf) || cg[blockIdx.y].done) return;
    rf += (size_t)blockIdx.y * gf.N;
    bc += (size_t)blockIdx.y * gc.N;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < gc.N; s += gridDim.x * kThreads) {
        int I, J, K;
        decode3(gc, s, I, J, K);
        const int fx = 2 * I + 1, fy = 2 * J + 1, fz = 2 * K + 1;
        float acc = 0.0f;
        for (int dz = -1; dz <= 1; ++dz) {
            const int z = fz + dz;
            if (z < 0 || z >= gf.nz) continue;
            const float wz = dz ? 0.5f : 1.0f;
            for (int dy = -1; dy <= 1; ++dy) {
                const int y = fy + dy;
                if (y < 0 || y >= gf.ny) continue;
                const float wy = dy ? 0.5f : 1.0f;
                const size_t row = ((size_t)z * gf.ny + y) * gf.nx;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int x = fx + dx;
                    if (x < 0 || x >= gf.nx) continue;
                    acc += wz * wy * (dx ? 0.5f : 1.0f) * rf[row + x];
                }
            }
        }
        bc[s] = acc;
    }
}

// Coarse indices and weights of fine index i along an axis of m coarse points.
__device__ __forceinline__ int interp_axis(int i, int m, int* c, float* w) {
    if (i & 1) {
        c[0] = (i - 1) >> 1;
        w[0] = 1.0f;
        return c[0] < m ? 1 : 0;
    }
    int k = 0;
    const int lo = (i >> 1) - 1, hi = i >> 1;
    if (lo >= 0 && lo < m) { c[k] = lo; w[k] = 0.5f; ++k; }
    if (hi >= 0 && hi < m) { c[k] = hi; w[k] = 0.5f; ++k; }
    return k;
}


// x_f += P x_c (trilinear, zero ghosts).  (Fusing it into the first
// post-smoothing half-sweep, each site taking its neighbours' prolongated
// corrections, measured slower: six interpolations per site instead of one.)
__global__ void __launch_bounds__(kThreads) k_mg_prolong(Grid gf, Grid gc, const float* __restrict__ xc,
                                                         float* __restrict__ xf, const CGState* cg) {
    if (inactive(gf) || cg[blockIdx.y].done) return;
    xc += (size_t)blockIdx.y * gc.N;
    xf += (size_t)blockIdx.y * gf.N;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < gf.N; s += gridDim.x * kThreads) {
        int x, y, z;
        decode3(gf, s, x, y, z);
        int cx[2], cy[2], cz[2];
        float wx[2], wy[2], wz[2];
        const int nxw = interp_axis(x, gc.nx, cx, wx), nyw = interp_axis(y, gc.ny, cy, wy),
                  nzw = interp_axis(z, gc.nz, cz, wz);
        float acc = 0.0f;
        for (int a = 0; a < nzw; ++a)
            for (int b = 0; b < nyw; ++b) {
                const size_t row = ((size_t)cz[a] * gc.ny + cy[b]) * gc.nx;
                for (int c = 0; c < nxw; ++c) acc += wz[a] * wy[b] * wx[c] * xc[row + cx[c]];
            }
        xf[s] += acc;
    }
}

// Coarsest level in one CTA: x = 0, then kCoarse red/black sweeps and
// kCoarse black/red sweeps, a barrier between colours.
__global__ void __launch_bounds__(kThreads) k_mg_coarse_solve(Grid g, float scale, float* __restrict__ x,
                                                              const float* __restrict__ b, const CGState* cg) {
    if (inactive(g) || cg[blockIdx.y].done) return;
    x += (size_t)blockIdx.y * g.N;
    b += (size_t)blockIdx.y * g.N;
    const float inv = 1.0f / (6.0f * scale);
    for (uint32_t s = threadIdx.x; s < g.N; s += blockDim.x) x[s] = 0.0f;
    __syncthreads();
    for (int half = 0; half < 4 * kCoarse; ++half) {
        const int k = half >> 1;  // sweep number
        const int first = k < kCoarse ? 0 : 1;
        const int colour = (half & 1) ? 1 - first : first;
        for (uint32_t s = threadIdx.x; s < g.N; s += blockDim.x) {
            int ix, iy, iz;
            decode3(g, s, ix, iy, iz);
            if (((ix + iy + iz) & 1) != colour) continue;
            const float nb = nb_sum(g, x, s, ix, iy, iz);
            x[s] = (b[s] + scale * nb) * inv;
        }
        __syncthreads();
    }
}

// ----------------------------------------------- coarse levels inside one CTA
// Levels of at most kTailSites sites (and all coarser ones) run their part of
// the V-cycle -- zero, pre-smoothing, residual, restriction down to the
// coarsest solve, then prolongation and post-smoothing back up -- in one CTA
// per system, a barrier between passes, on copies in shared memory (x, b and
// r of every such level: at most 3 x 4 x 4689 bytes, since each level has at
// most an eighth of the sites of the one above).  The first of them takes
// its right-hand side from global memory and returns its correction there.
// The passes are those of the one-level kernels above, site by site in the
// same arithmetic; red-black Gauss-Seidel updates of one colour read only the
// other colour, so the results do not depend on how sites map to threads.
constexpr int kTailThreads = 512;
// 16^3: the single-precision passes of one CTA over a 16^3 level and the
// coarser ones take less than the launches they replace
constexpr uint32_t kTailSites = LBKS_MG_TAIL_SITES;
// shared-memory values of the tail at most: x, b, r of a level of kTailSites
// sites and of every coarser one (each at most an eighth of the one above)
constexpr size_t kTailValuesMax = 3 * (kTailSites + kTailSites / 7 + 8);

__device__ __forceinline__ void cta_smooth(const Grid& g, float scale, int colour, float* __restrict__ x,
                                           const float* __restrict__ b) {
    const float inv = 1.0f / (6.0f * scale);
    const uint32_t hx = (uint32_t)(g.nx + 1) / 2, slots = hx * (uint32_t)g.ny * (uint32_t)g.nz;
    for (uint32_t k = threadIdx.x; k < slots; k += blockDim.x) {  // the colour's sites only
        const uint32_t q = k / hx;
        const uint32_t zz = g.divy.div(q);
        const int iy = (int)(q - zz * (uint32_t)g.ny), iz = (int)zz;
        const int ix = 2 * (int)(k - q * hx) + ((colour + iy + iz) & 1);
        if (ix >= g.nx) continue;
        const uint32_t s = (zz * (uint32_t)g.ny + (uint32_t)iy) * (uint32_t)g.nx + (uint32_t)ix;
        const float nb = nb_sum(g, x, s, ix, iy, iz);
        x[s] = (b[s] + scale * nb) * inv;
    }
    __syncthreads();
}

// Shared-memory values the tail needs from level lc down.
size_t tail_values(const MGHierarchy& H, int lc) {
    size_t n = 0;
    for (int l = lc; l < H.nlev; ++l) n += 3 * (size_t)H.lev[l].g.N;
    return n;
}

__global__ void __launch_bounds__(kTailThreads) k_mg_tail(MGHierarchy H, int lc, float* __restrict__ xg,
                                                          const float* __restrict__ bg, const CGState* cg) {
    if (inactive(H.lev[0].g) || cg[blockIdx.y].done) return;
    extern __shared__ __align__(16) float tsh[];
    const int L = H.nlev;
    const size_t y = blockIdx.y;
    // level l's x, b and r in shared memory, levels lc .. L - 1 one after the other
    float* xs[kMaxLevels];
    float* bs[kMaxLevels];
    float* rs[kMaxLevels];
    {
        float* q = tsh;
        for (int l = lc; l < L; ++l) {
            const uint32_t n = H.lev[l].g.N;
            xs[l] = q;
            bs[l] = q + n;
            rs[l] = q + 2 * n;
            q += 3 * (size_t)n;
        }
    }
    {
        const uint32_t n = H.lev[lc].g.N;
        const float* b = bg + y * n;
        for (uint32_t s = threadIdx.x; s < n; s += blockDim.x) bs[lc][s] = b[s];
    }
    for (int l = lc; l < L; ++l) {
        const Grid& g = H.lev[l].g;
        const float sc = (float)(1 << l);
        float* x = xs[l];
        const float* b = bs[l];
        for (uint32_t s = threadIdx.x; s < g.N; s += blockDim.x) x[s] = 0.0f;
        __syncthreads();
        if (l == L - 1) {  // coarsest: kCoarse red/black sweeps, then kCoarse black/red
            for (int k = 0; k < kCoarse; ++k) {
                cta_smooth(g, sc, 0, x, b);
                cta_smooth(g, sc, 1, x, b);
            }
            for (int k = 0; k < kCoarse; ++k) {
                cta_smooth(g, sc, 1, x, b);
                cta_smooth(g, sc, 0, x, b);
            }
            break;
        }
        for (int k = 0; k < kPre; ++k) {
            cta_smooth(g, sc, 0, x, b);
            cta_smooth(g, sc, 1, x, b);
        }
        float* r = rs[l];
        for (uint32_t s = threadIdx.x; s < g.N; s += blockDim.x) {
            int ix, iy, iz;
            decode3(g, s, ix, iy, iz);
            r[s] = b[s] - sc * stencil(g, x, s, ix, iy, iz, x[s]);
        }
        __syncthreads();
        const Grid& gc = H.lev[l + 1].g;
        float* bc = bs[l + 1];
        for (uint32_t s = threadIdx.x; s < gc.N; s += blockDim.x) {
            int I, J, K;
            decode3(gc, s, I, J, K);
            const int fx = 2 * I + 1, fy = 2 * J + 1, fz = 2 * K + 1;
            float acc = 0.0f;
            for (int dz = -1; dz <= 1; ++dz) {
                const int z = fz + dz;
                if (z < 0 || z >= g.nz) continue;
                const float wz = dz ? 0.5f : 1.0f;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int yy = fy + dy;
                    if (yy < 0 || yy >= g.ny) continue;
                    const float wy = dy ? 0.5f : 1.0f;
                    const size_t row = ((size_t)z * g.ny + yy) * g.nx;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int xx = fx + dx;
                        if (xx < 0 || xx >= g.nx) continue;
                        acc += wz * wy * (dx ? 0.5f : 1.0f) * r[row + xx];
                    }
                }
            }
            bc[s] = acc;
        }
        __syncthreads();
    }
    for (int l = L - 2; l >= lc; --l) {
        const Grid& g = H.lev[l].g;
        const Grid& gc = H.lev[l + 1].g;
        const float sc = (float)(1 << l);
        float* x = xs[l];
        const float* xc = xs[l + 1];
        for (uint32_t s = threadIdx.x; s < g.N; s += blockDim.x) {
            int ix, iy, iz;
            decode3(g, s, ix, iy, iz);
            int cx[2], cy[2], cz[2];
            float wx[2], wy[2], wz[2];
            const int nxw = interp_axis(ix, gc.nx, cx, wx), nyw = interp_axis(iy, gc.ny, cy, wy),
                      nzw = interp_axis(iz, gc.nz, cz, wz);
            float acc = 0.0f;
            for (int a = 0; a < nzw; ++a)
                for (int bb = 0; bb < nyw; ++bb) {
                    const size_t row = ((size_t)cz[a] * gc.ny + cy[bb]) * gc.nx;
                    for (int cc = 0; cc < nxw; ++cc) acc += wz[a] * wy[bb] * wx[cc] * xc[row + cx[cc]];
                }
            x[s] += acc;
        }
        __syncthreads();
        for (int k = 0; k < kPre; ++k) {
            cta_smooth(g, sc, 1, x, bs[l]);
            cta_smooth(g, sc, 0, x, bs[l]);
        }
    }
    {
        const uint32_t n = H.lev[lc].g.N;
        float* x = xg + y * n;
        for (uint32_t s = threadIdx.x; s < n; s += blockDim.x) x[s] = xs[lc][s];
    }
}



// --------------------------------------------------------------------- PCG kernels
// b = 4 pi h^2 rho + ghost values; r = b - A x; |b|^2, |r|^2.
__global__ void __launch_bounds__(kThreads) k_pcg_start(Grid g, double h, const double* __restrict__ rho,
                                                        const double* __restrict__ x, double rtol, PoissonBufs pb,
                                                        Scratch sc) {
    if (inactive(g)) return;
    pb = at_sys(pb, g.N);
    rho += (size_t)blockIdx.y * g.N;
    x += (size_t)blockIdx.y * g.N;
    const double kPi = 3.141592653589793238462643383279502884;
    double acc[2] = {0.0, 0.0};
    const double* mp = pb.mp;
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads) {
        int ix, iy, iz;
        decode3(g, s, ix, iy, iz);
        const double rx = (ix - 0.5 * (g.nx - 1)) * h, ry = (iy - 0.5 * (g.ny - 1)) * h,
                     rz = (iz - 0.5 * (g.nz - 1)) * h;
        double b = 4.0 * kPi * h * h * rho[s];
        if (ix == 0) b += multipole_value(mp, rx - h, ry, rz);
        if (ix == g.nx - 1) b += multipole_value(mp, rx + h, ry, rz);
        if (iy == 0) b += multipole_value(mp, rx, ry - h, rz);
        if (iy == g.ny - 1) b += multipole_value(mp, rx, ry + h, rz);
        if (iz == 0) b += multipole_value(mp, rx, ry, rz - h);
        if (iz == g.nz - 1) b += multipole_value(mp, rx, ry, rz + h);
        pb.b[s] = b;
        const double r = b - stencil(g, x, s, ix, iy, iz, x[s]);
        pb.r[s] = r;
        pb.r32[s] = (float)r;
        acc[0] += b * b;
        acc[1] += r * r;
    }
    double* partial = sys_partial(sc);
    block_sum_store<2>(acc, partial + (size_t)blockIdx.x * 2);
    __shared__ double tot[2];
    if (grid_total<2>(partial, sys_counter(sc), tot) && threadIdx.x == 0) {
        CGState* cg = pb.cg;
        cg->bb = tot[0];
        cg->rr = tot[1];
        cg->rz = 0.0;
        cg->rtol = rtol;
        cg->iters = 0;
        cg->relres = tot[0] > 0.0 ? sqrt(tot[1] / tot[0]) : 0.0;
        cg->done = (tot[0] == 0.0 || sqrt(tot[1]) <= rtol * sqrt(tot[0])) ? 1 : 0;
    }
}

// z = (double) x32 (the V-cycle's result); rz = r . z; beta = -alpha
// (A p_old . z) / rz_old (the flexible form; 0 on the first iteration, where ap
// is not read)
__global__ void __launch_bounds__(kThreads) k_pcg_rz(Grid g, PoissonBufs pb, Scratch sc) {
    if (inactive(g)) return;
    pb = at_sys(pb, g.N);
    if (pb.cg->done) return;
    const bool first = pb.cg->iters == 0;
    double acc[2] = {0.0, 0.0};
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads) {
        const double z = (double)pb.x32[s];  // the preconditioner's single-precision result, widened
        pb.z[s] = z;
        acc[0] += pb.r[s] * z;
        if (!first) acc[1] += pb.ap[s] * z;
    }
    double* partial = sys_partial(sc);
    block_sum_store<2>(acc, partial + (size_t)blockIdx.x * 2);
    __shared__ double tot[2];
    if (grid_total<2>(partial, sys_counter(sc), tot) && threadIdx.x == 0) {
        CGState* cg = pb.cg;
        cg->beta = (!first && cg->rz > 0.0) ? -cg->alpha * tot[1] / cg->rz : 0.0;
        cg->rz = tot[0];
    }
}

// p = z + beta p; p = z on the first iteration of a solve (p is not read
// then: it holds whatever the memory held, and 0 * NaN is NaN).  (Forming p
// inside the A p kernel at the site and its six neighbours costs seven times
// the FP64 arithmetic, which GB300 issues at a small fraction of its FP32
// rate: measured slower than this separate pass.)
__global__ void __launch_bounds__(kThreads) k_pcg_dir(Grid g, PoissonBufs pb) {
    if (inactive(g)) return;
    pb = at_sys(pb, g.N);
    if (pb.cg->done) return;
    const double beta = pb.cg->beta;
    if (pb.cg->iters == 0) {
        for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads) pb.p[s] = pb.z[s];
        return;
    }
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads)
        pb.p[s] = pb.z[s] + beta * pb.p[s];
}

// ap = A p; alpha = rz / (p . ap)
__global__ void __launch_bounds__(kThreads) k_pcg_ap(Grid g, PoissonBufs pb, Scratch sc) {
    if (inactive(g)) return;
    pb = at_sys(pb, g.N);
    if (pb.cg->done) return;
    double acc[1] = {0.0};
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads) {
        int ix, iy, iz;
        decode3(g, s, ix, iy, iz);
        const double a = stencil(g, pb.p, s, ix, iy, iz, pb.p[s]);
        pb.ap[s] = a;
        acc[0] += pb.p[s] * a;
    }
    double* partial = sys_partial(sc);
    block_sum_store<1>(acc, partial + (size_t)blockIdx.x);
    __shared__ double tot[1];
    if (grid_total<1>(partial, sys_counter(sc), tot) && threadIdx.x == 0) {
        pb.cg->pap = tot[0];
        pb.cg->alpha = pb.cg->rz / tot[0];
    }
}

// x += alpha p; r -= alpha ap (and its single-precision copy); convergence
// test on |r| / |b|
__global__ void __launch_bounds__(kThreads) k_pcg_update(Grid g, double* __restrict__ x, PoissonBufs pb, Scratch sc) {
    if (inactive(g)) return;
    pb = at_sys(pb, g.N);
    if (pb.cg->done) return;
    x += (size_t)blockIdx.y * g.N;
    const double alpha = pb.cg->alpha;
    const double* __restrict__ p = pb.p;
    double acc[1] = {0.0};
    for (uint32_t s = blockIdx.x * kThreads + threadIdx.x; s < g.N; s += gridDim.x * kThreads) {
        x[s] += alpha * p[s];
        const double r = pb.r[s] - alpha * pb.ap[s];
        pb.r[s] = r;
        pb.r32[s] = (float)r;  // the next V-cycle's right-hand side
        acc[0] += r * r;
    }
    double* partial = sys_partial(sc);
    block_sum_store<1>(acc, partial + (size_t)blockIdx.x);
    __shared__ double tot[1];
    if (grid_total<1>(partial, sys_counter(sc), tot) && threadIdx.x == 0) {
        CGState* cg = pb.cg;
        cg->rr = tot[0];
        cg->iters += 1;
        cg->relres = sqrt(tot[0] / cg->bb);
        cg->done = (sqrt(tot[0]) <= cg->rtol * sqrt(cg->bb)) ? 1 : 0;
    }
}

// One V-cycle on every system's level arrays: the finest level's b is the
// single-precision residual (written by the CG kernels) and its x the result.
cudaError_t vcycle(const MGHierarchy& H, const CGState* cg, int ge, int Bs, cudaStream_t st, uint64_t* nl) {
    auto X = [&](int l) { return H.lev[l].x; };
    auto B = [&](int l) -> const float* { return H.lev[l].b; };
    auto R = [&](int l) { return H.lev[l].r; };
    auto grid = [&](size_t n) { return dim3(grid_for(n, std::max(1, ge / Bs)), Bs); };
    const int L = H.nlev;
    // first level small enough for the one-CTA tail (levels below it run there)
    int lc = L;
    for (int l = 0; l < L; ++l)
        if (H.lev[l].g.N <= kTailSites) {
            lc = l;
            break;
        }
    auto half = [&](int l) {  // one colour's sites: ceil(nx / 2) slots per row
        const Grid& g = H.lev[l].g;
        const uint32_t hx = (uint32_t)(g.nx + 1) / 2;
        return std::make_pair(FastDiv(hx), (size_t)hx * g.ny * g.nz);
    };
    for (int l = 0; l < L; ++l) {
        const Grid& g = H.lev[l].g;
        const float sc = (float)(1 << l);
        const dim3 gl = grid(g.N);
        if (l == lc) {
            const size_t smem = sizeof(float) * tail_values(H, lc);
            static const cudaError_t attr = cudaFuncSetAttribute(
                k_mg_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float) * kTailValuesMax));
            if (attr != cudaSuccess) return attr;
            if (smem > sizeof(float) * kTailValuesMax) return cudaErrorInvalidValue;
            k_mg_tail<<<dim3(1, Bs), kTailThreads, smem, st>>>(H, lc, X(l), B(l), cg);
            ++*nl;
            break;
        }
        if (l == L - 1 && g.N <= kCoarseSites) {
            k_mg_coarse_solve<<<dim3(1, Bs), kThreads, 0, st>>>(g, sc, X(l), B(l), cg);
            ++*nl;
            break;
        }
        const auto hd = half(l);
        const dim3 gh = grid(hd.second);
        if (l == L - 1) {  // a coarsest level too large for one CTA: sweeps from zero
            k_mg_smooth<<<gh, kThreads, 0, st>>>(g, hd.first, sc, 0, 1, X(l), B(l), cg);
            k_mg_smooth<<<gh, kThreads, 0, st>>>(g, hd.first, sc, 1, 0, X(l), B(l), cg);
            for (int k = 1; k < kCoarse; ++k) {
                k_mg_smooth<<<gh, kThreads, 0, st>>>(g, hd.first, sc, 0, 0, X(l), B(l), cg);
                k_mg_smooth<<<gh, kThreads, 0, st>>>(g, hd.first, sc, 1, 0, X(l), B(l), cg);
            }
            for (int k = 0; k < kCoarse; ++k) {
                k_mg_smooth<<<gh, kThreads, 0, st>>>(g, hd.first, sc, 1, 0, X(l), B(l), cg);
                k_mg_smooth<<<gh, kThreads, 0, st>>>(g, hd.first, sc, 0, 0, X(l), B(l), cg);
            }
            *nl += 4 * kCoarse;
            break;
        }
        // pre-smoothing from x = 0: the first red half-sweep reads no neighbour
        for (int k = 0; k < kPre; ++k) {
            k_mg_smooth<<<gh, kThreads, 0, st>>>(g, hd.first, sc, 0, k == 0 ? 1 : 0, X(l), B(l), cg);
            k_mg_smooth<<<gh, kThreads, 0, st>>>(g, hd.first, sc, 1, 0, X(l), B(l), cg);
        }
        k_mg_residual<<<gl, kThreads, 0, st>>>(g, sc, X(l), B(l), R(l), cg);
        const Grid& gc = H.lev[l + 1].g;
        k_mg_restrict<<<grid(gc.N), kThreads, 0, st>>>(g, gc, R(l), H.lev[l + 1].b, cg);
        *nl += 2 * kPre + 2;
    }
    for (int l = std::min(L, lc) - 1; l >= 0; --l) {
        if (l == L - 1) continue;  // coarsest level: nothing to prolong from
        const Grid& g = H.lev[l].g;
        const float sc = (float)(1 << l);
        const auto hd = half(l);
        const dim3 gh = grid(hd.second);
        // correction, then post-smoothing black then red
        k_mg_prolong<<<grid(g.N), kThreads, 0, st>>>(g, H.lev[l + 1].g, X(l + 1), X(l), cg);
        for (int k = 0; k < kPre; ++k) {
            k_mg_smooth<<<gh, kThreads, 0, st>>>(g, hd.first, sc, 1, 0, X(l), B(l), cg);
            k_mg_smooth<<<gh, kThreads, 0, st>>>(g, hd.first, sc, 0, 0, X(l), B(l), cg);
        }
        *nl += 1 + 2 * kPre;
    }
    return cudaGetLastError();
}

}  // namespace

int mg_levels(int nx, int ny, int nz) {
    int l = 1;
    while (l < kMaxLevels && nx / 2 >= 2 && ny / 2 >= 2 && nz / 2 >= 2) {
        nx /= 2;
        ny /= 2;
        nz /= 2;
        ++l;
    }
    return l;
}

// Floats of x, b, r of every level (the finest included), padded per level to
// four floats (16-byte aligned arrays), as doubles.
size_t mg_coarse_doubles(int nx, int ny, int nz) {
    size_t floats = 0;
    const int L = mg_levels(nx, ny, nz);
    for (int l = 0; l < L; ++l) {
        floats += 3 * (((size_t)nx * ny * nz + 3) & ~(size_t)3);
        nx /= 2;
        ny /= 2;
        nz /= 2;
    }
    return (floats + 1) / 2;
}

MGHierarchy make_hierarchy(const Grid& fine, double* coarse, int B) {
    MGHierarchy H;
    H.nlev = mg_levels(fine.nx, fine.ny, fine.nz);
    float* q = reinterpret_cast<float*>(coarse);
    int nx = fine.nx, ny = fine.ny, nz = fine.nz;
    for (int l = 0; l < H.nlev; ++l) {
        if (l > 0) {
            nx /= 2;
            ny /= 2;
            nz /= 2;
        }
        H.lev[l].g = l == 0 ? fine : make_grid(nx, ny, nz);
        H.lev[l].g.active = fine.active;
        const size_t n = (((size_t)nx * ny * nz + 3) & ~(size_t)3) * B;
        H.lev[l].x = q;
        H.lev[l].b = q + n;
        H.lev[l].r = q + 2 * n;
        q += 3 * n;
    }
    return H;
}

cudaError_t launch_poisson_start(const Grid& g, double h, const double* rho, double* x, double rtol,
                                 const PoissonBufs& pb, const Scratch& sc, int B, cudaStream_t st) {
    const int cap = red_cap(sc, 2, B);
    if (cap < 1) return cudaErrorInvalidValue;
    k_pcg_start<<<dim3(grid_for(g.N, cap), B), kThreads, 0, st>>>(g, h, rho, x, rtol, pb, sc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_poisson_iterate(const Grid& g, double* x, double rtol, int iters, const PoissonBufs& pb,
                                   const MGHierarchy& H, const Scratch& sc, int B, cudaStream_t st) {
    (void)rtol;  // the start kernel's tolerance, device-resident
    const int cap = red_cap(sc, 1, B);
    if (cap < 1) return cudaErrorInvalidValue;
    const dim3 gr(grid_for(g.N, cap), B);
    const int ge = num_sms() * 8;
    const dim3 gel(grid_for(g.N, std::max(1, ge / B)), B);
    uint64_t nl = 0;
    for (int i = 0; i < iters; ++i) {
        cudaError_t e = vcycle(H, pb.cg, ge, B, st, &nl);
        if (e != cudaSuccess) return e;
        k_pcg_rz<<<gr, kThreads, 0, st>>>(g, pb, sc);
        k_pcg_dir<<<gel, kThreads, 0, st>>>(g, pb);
        k_pcg_ap<<<gr, kThreads, 0, st>>>(g, pb, sc);
        k_pcg_update<<<gr, kThreads, 0, st>>>(g, x, pb, sc);
        nl += 4;
    }
    count_launches(nl);
    return cudaGetLastError();
}

}  // namespace lbks
