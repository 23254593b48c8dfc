// C ABI of liblbks (include/lbks.h): system handles, the self-consistent
// driver (CUDA graph per relaxation cycle), step-level entry points.
#include "lbks.h"
#include "lbks_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

namespace lbks {

namespace {
thread_local std::string g_err;
thread_local bool g_capturing = false;
std::atomic<uint64_t> g_launches{0};

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? LBKS_ENOMEM : LBKS_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}
}  // namespace

int set_last_error(int code, const char* msg) {
    g_err = msg ? msg : "";
    return code;
}

void count_launches(uint64_t n) {
    if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}

int num_sms() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

Coef make_coef(double omega, double theta, double dt, double h) {
    Coef c;
    c.omega = omega;
    c.dt = dt;
    c.theta = theta;
    c.h = h;
    const double cs2 = 1.0 / 3.0;
    const double w[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    for (int k = 0; k < 3; ++k) {
        const double v2 = (double)k;
        const double q = (v2 - 3.0 * cs2) / (2.0 * cs2 * cs2);  // second-order Hermite polynomial
        c.xi[k] = w[k] * (1.0 + (theta - cs2) * q);
        c.chi[k] = w[k] * (1.0 - (v2 - 3.0 * cs2) / (2.0 * cs2));
    }
    return c;
}

Grid make_grid(int nx, int ny, int nz) {
    Grid g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.N = (uint32_t)((size_t)nx * ny * nz);
    g.divx = FastDiv((uint32_t)nx);
    g.divy = FastDiv((uint32_t)ny);
    return g;
}

namespace {

const PrecisionOps* ops_for(int precision) {
    if (precision == LBKS_FP64) return &ops_f64();
    if (precision == LBKS_FP32) return &ops_f32();
    if (precision == LBKS_BF16) return &ops_bf16();
    return nullptr;
}

constexpr int kScratchVals = kMaxOrb * kMaxOrb + kMaxOrb;  // largest reduction width up to kMaxOrb orbitals
// Largest reduction width of a handle with n_orb orbitals.
int scratch_vals(int n_orb) { return n_orb <= kMaxOrb ? kScratchVals : n_orb * (n_orb + 1) / 2 + n_orb; }
// Doubles of the energy-matrix output per system.
int emat_stride(int n_orb) { return n_orb <= kMaxOrb ? kEmatStride : kEmatWideStride; }

// The counter is zeroed on `st`, the stream the scratch is then used on: a
// legacy-stream cudaMemset is not ordered before work on non-blocking streams.
cudaError_t alloc_scratch(Scratch& sc, cudaStream_t st) {
    sc.max_blocks = num_sms() * 8;
    sc.max_vals = scratch_vals(kMaxOrbWide);
    sc.systems = 1;
    cudaError_t e = cudaMalloc(&sc.partial, sizeof(double) * (size_t)sc.max_blocks * sc.max_vals);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&sc.counter, sizeof(unsigned) * 4);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(sc.counter, 0, sizeof(unsigned) * 4, st);
}

// Library-managed workspace of the step-level entry points, one per
// (device, stream): reduction scratch and Poisson vectors grown on demand.
struct Workspace {
    Scratch sc;
    double* pvec = nullptr;  // n_pvec doubles: b, r, p, ap, z, tmp and the coarse levels
    size_t n_pvec = 0;
    CGState* cg = nullptr;
    double* mp = nullptr;
};
std::mutex g_ws_mu;
std::map<std::pair<int, void*>, Workspace*> g_ws;

int workspace(void* stream, size_t n_pvec, Workspace** out) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_ws_mu);
    Workspace*& w = g_ws[{dev, stream}];
    if (!w) {
        w = new Workspace();
        cudaError_t e = alloc_scratch(w->sc, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaMalloc(&w->cg, sizeof(CGState));
        if (e == cudaSuccess) e = cudaMalloc(&w->mp, sizeof(double) * 16);
        if (e != cudaSuccess) {
            delete w;
            w = nullptr;
            return cuda_fail(e, "workspace allocation");
        }
    }
    if (n_pvec > w->n_pvec) {
        if (w->pvec) cudaFree(w->pvec);
        w->pvec = nullptr;
        w->n_pvec = 0;
        cudaError_t e = cudaMalloc(&w->pvec, sizeof(double) * n_pvec);
        if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
        w->n_pvec = n_pvec;
    }
    *out = w;
    return LBKS_OK;
}

// Symmetric eigenvalues by cyclic Jacobi rotations (n <= 64), ascending.
void jacobi_eigenvalues(int n, std::vector<double> a, double* out) {
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
            }
    }
    for (int i = 0; i < n; ++i) out[i] = a[i * n + i];
    std::sort(out, out + n);
}

bool valid_params(const lbks_params* p) {
    return p && p->omega > 0.0 && p->omega < 2.0 && p->theta > 0.0 && p->n_inner >= 2 && p->mix > 0.0 &&
           p->mix <= 1.0 && p->e_tol > 0.0 && p->max_cycles >= 1 && ops_for(p->precision) &&
           p->poisson_rtol > 0.0 && p->poisson_max_iter >= 1 && !std::isnan(p->eig_tol) &&
           p->poisson_adapt >= 0.0 && std::isfinite(p->poisson_adapt) &&
           !std::isnan(p->rho_tol) &&
           (p->storage == LBKS_STORE_POPULATIONS ||
            (p->storage == LBKS_STORE_PSI && p->omega == 1.0 && p->precision != LBKS_BF16));
}

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): advances the state, returns the next output.
uint64_t splitmix64(uint64_t& state) {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Offsets (bohr) of the Gaussian start centres from their nuclei, n_orb x 3.
// seed 0: 0.25 (sin(1 + 2.1 j), sin(2 + 3.3 j), sin(3 + 4.7 j)); otherwise
// 0.25 (2u - 1) per component, u the top 53 bits of successive SplitMix64
// outputs from state = seed, drawn x, y, z for j = 0, 1, ...
std::vector<double> start_offsets(int n_orb, uint64_t seed) {
    std::vector<double> off(3 * (size_t)n_orb);
    if (seed == 0) {
        for (int j = 0; j < n_orb; ++j) {
            off[3 * j] = 0.25 * std::sin(1.0 + 2.1 * j);
            off[3 * j + 1] = 0.25 * std::sin(2.0 + 3.3 * j);
            off[3 * j + 2] = 0.25 * std::sin(3.0 + 4.7 * j);
        }
        return off;
    }
    uint64_t state = seed;
    for (size_t k = 0; k < off.size(); ++k) {
        const double u = (double)(splitmix64(state) >> 11) * 0x1.0p-53;
        off[k] = 0.25 * (2.0 * u - 1.0);
    }
    return off;
}

// Stop rule (include/lbks.h): the changes of one watched quantity over the
// last three blocks of kStopBlock cycles, newest first.  A change below
// kFloorUlps u s (u the unit roundoff of the orbital values, s the quantity's
// scale) is rounding noise.
constexpr int kStopBlock = 4;
constexpr double kTailCap = 0.92;  // per block: a contraction of 0.98 per cycle
constexpr double kFloorUlps = 8.0;
struct Changes {
    double d[3] = {INFINITY, INFINITY, INFINITY};
    int n = 0;
    void push(double v) {
        d[2] = d[1];
        d[1] = d[0];
        d[0] = v;
        ++n;
    }
    // d0 q / (1 - q), q the larger of d0/d1 and d1/d2 capped at kTailCap
    double tail() const {
        if (n < 3) return INFINITY;
        auto ratio = [](double a, double b) { return b > 0.0 ? a / b : (a > 0.0 ? INFINITY : 0.0); };
        const double q = std::min(std::max(ratio(d[0], d[1]), ratio(d[1], d[2])), kTailCap);
        return d[0] * q / (1.0 - q);
    }
    bool settled(double tol, double floor) const {
        if (!(tol > 0.0)) return true;
        if (n < 3) return false;
        return d[0] <= floor || (d[0] <= tol && tail() <= tol);
    }
};

}  // namespace
}  // namespace lbks

using namespace lbks;

// One handle holds B >= 1 systems of the same shape and parameters; each
// system's arrays sit consecutively (see PrecisionOps).  Single-system calls
// address system 0.
struct lbks_system {
    lbks_params prm;
    int nx, ny, nz, n_orb, B;
    double h, dt, a;
    Grid g;
    Coef c;
    const PrecisionOps* ops;
    size_t N;
    int dev;
    void* f[2] = {nullptr, nullptr};       // populations; orbital storage: psi ping-pong (psi aliases f[cur])
    void* f_wide[2] = {nullptr, nullptr};  // FP32 populations of the BF16 polish phase
    bool psi_storage = false;              // lbks_params.storage == LBKS_STORE_PSI
    double* vprev = nullptr;               // orbital storage: potential of the last collision
    bool polished = false;
    int cur = 0;
    void* u = nullptr;
    void* psi = nullptr;
    double *vin = nullptr, *vout = nullptr, *vext = nullptr, *vh = nullptr, *rho = nullptr;
    double* rho_ref = nullptr;  // density at the end of the last block of the stop rule
    double* pvec = nullptr;  // b, r, p, ap, z, tmp (B*N each), then the multigrid levels
    CGState* cg = nullptr;
    MGHierarchy mg;
    cudaGraphExec_t poisson_graph = nullptr;  // kPoissonChunk preconditioned CG iterations
    uint64_t poisson_nodes = 0;
    double* small = nullptr;
    double *S, *lam, *sigma, *Linv, *e4, *emat, *mp, *atoms, *forces;
    int* ints = nullptr;  // status[B], active[B], atom counts[B]
    int *status, *active, *counts;
    OrbitalStart* starts = nullptr;  // [B][n_orb]
    Scratch sc;
    double* host = nullptr;  // pinned readback area
    cudaStream_t st = nullptr;   // internal stream for synchronous calls
    cudaStream_t cap = nullptr;  // capture stream
    int variant = kRelaxSites;   // stream-collide variant (tuned per shape)
    double tune_ms[kRelaxVariants] = {-1.0, -1.0, -1.0, -1.0};
    double tune_shape_ms[kPsiShapes] = {-1.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0};  // orbital storage: the staged kernel per tile shape
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    uint64_t graph_nodes[2] = {0, 0};
    std::vector<std::vector<double>> xyz, Z;  // per system
    std::vector<int> has_atoms;
    bool ready = false;  // orbitals and energies initialised
    std::vector<lbks_energy_terms> terms;
    std::vector<double> drho;  // ||rho - rho_prev|| / ||rho|| of the last evaluation, per system
    int poisson_iters = 0;
    double poisson_ms = 0.0;                   // device time of the Hartree solves (CUDA events)
    cudaEvent_t pev[2] = {nullptr, nullptr};
    // concurrent dynamics (lbks_cd_start / lbks_cd_run): three complex levels
    // [j][part][N] of the compute type, rotated step by step
    void* cd_lev[3] = {nullptr, nullptr, nullptr};
    int cd_prev = 0, cd_cur = 1;
    double* cd_small = nullptr;  // Lambda x 2, S, U coefficients x 2, energy matrix of 2 n_orb rows
    int cd_lam = 0;              // which Lambda buffer belongs to the current level
    Scratch cd_sc;               // reductions of up to 2 n_orb rows
    bool cd_ready = false, cd_u = false;
    double cd_tau = 0.0, cd_time = 0.0;
    int cd_npot = 10;
    int64_t cd_steps = 0;
    std::vector<double> cd_F;  // forces at the current level (host, 3 n_atoms)
};

namespace {

// Doubles per system of the small device arrays (S, Lambda, L^-1, sigma,
// energy integrals, energy matrix, multipoles).
size_t small_per_sys(int no) { return 3 * (size_t)no * no + no + kE4Stride + emat_stride(no) + kMpStride; }
constexpr int kPoissonChunk = 2;  // PCG iterations per graph launch between convergence checks
// Doubles per system of the pinned readback area: energy integrals, energy
// matrix, the density change (two sums) and spare room.
size_t host_per_sys(int no) { return kE4Stride + emat_stride(no) + 4; }

PoissonBufs poisson_bufs(double* v, size_t n, CGState* cg, double* mp, const MGHierarchy& H) {
    return PoissonBufs{v, v + n, v + 2 * n, v + 3 * n, v + 4 * n, v + 5 * n, cg, mp, H.lev[0].b, H.lev[0].x};
}

double* host_e4(lbks_system* s, int i) { return s->host + (size_t)i * host_per_sys(s->n_orb); }
double* host_emat(lbks_system* s, int i) { return host_e4(s, i) + kE4Stride; }
// h^3 sum (rho - rho_prev)^2 and h^3 sum rho^2 of the last density (mp[10], mp[11])
double* host_drho(lbks_system* s, int i) { return host_emat(s, i) + emat_stride(s->n_orb); }
int* host_status(lbks_system* s) { return reinterpret_cast<int*>(s->host + (size_t)s->B * host_per_sys(s->n_orb)); }
int* host_active(lbks_system* s) { return host_status(s) + s->B; }
CGState* host_cg(lbks_system* s) {
    return reinterpret_cast<CGState*>(s->host + (size_t)s->B * host_per_sys(s->n_orb) + s->B + 1);
}

int poisson_graph(lbks_system* s) {
    if (s->poisson_graph) return LBKS_OK;
    const PoissonBufs pb = poisson_bufs(s->pvec, s->N * s->B, s->cg, s->mp, s->mg);
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    g_capturing = true;
    cudaError_t ee =
        launch_poisson_iterate(s->g, s->vh, s->prm.poisson_rtol, kPoissonChunk, pb, s->mg, s->sc, s->B, s->cap);
    g_capturing = false;
    e = cudaStreamEndCapture(s->cap, &gr);
    if (ee != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return cuda_fail(ee, "capture Poisson iterations");
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    size_t nodes = 0;
    cudaGraphGetNodes(gr, nullptr, &nodes);
    e = cudaGraphInstantiate(&s->poisson_graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate Poisson graph");
    s->poisson_nodes = nodes;
    return LBKS_OK;
}

// The cycle's Hartree tolerance: poisson_rtol, or with poisson_adapt > 0 the
// inexact-solve bound of include/lbks.h from the previous evaluation's density
// change (the largest over the running systems); `adapt` false: poisson_rtol.
double hartree_rtol(const lbks_system* s, bool adapt) {
    const double base = s->prm.poisson_rtol;
    if (!adapt || s->prm.poisson_adapt <= 0.0) return base;
    double d = 0.0;
    for (int i = 0; i < s->B; ++i)
        if (host_active(const_cast<lbks_system*>(s))[i]) d = std::max(d, s->drho[i]);
    return std::max(base, std::min(1e-4, s->prm.poisson_adapt * d));
}

int hartree_solve(lbks_system* s, cudaStream_t st, bool adapt = false) {
    const PoissonBufs pb = poisson_bufs(s->pvec, s->N * s->B, s->cg, s->mp, s->mg);
    int rc = poisson_graph(s);
    if (rc != LBKS_OK) return rc;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        if (!s->pev[k]) e = cudaEventCreate(&s->pev[k]);
    if (e == cudaSuccess) e = cudaEventRecord(s->pev[0], st);
    if (e == cudaSuccess)
        e = launch_poisson_start(s->g, s->h, s->rho, s->vh, hartree_rtol(s, adapt), pb, s->sc, s->B, st);
    if (e != cudaSuccess) return cuda_fail(e, "poisson start");
    CGState* hcg = host_cg(s);
    const int* act = host_active(s);
    int done_iters = 0;
    while (true) {
        e = cudaMemcpyAsync(hcg, s->cg, sizeof(CGState) * s->B, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "poisson readback");
        int pending = -1;
        for (int i = 0; i < s->B; ++i)
            if (act[i] && !hcg[i].done) pending = i;
        if (pending < 0) break;
        if (done_iters >= s->prm.poisson_max_iter)
            return fail(LBKS_ENOTCONV, "Hartree PCG (system %d): relative residual %.3e after %d iterations",
                        pending, hcg[pending].relres, hcg[pending].iters);
        e = cudaGraphLaunch(s->poisson_graph, st);
        if (e != cudaSuccess) return cuda_fail(e, "poisson iterate");
        count_launches(s->poisson_nodes);
        done_iters += kPoissonChunk;
    }
    int most = 0;
    for (int i = 0; i < s->B; ++i)
        if (act[i]) most = std::max(most, hcg[i].iters);
    s->poisson_iters += most;
    // the loop above ended on a synchronised readback: the events are complete
    float ms = 0.0f;
    e = cudaEventRecord(s->pev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(s->pev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, s->pev[0], s->pev[1]);
    if (e != cudaSuccess) return cuda_fail(e, "poisson timing");
    s->poisson_ms += ms;
    return LBKS_OK;
}

// Density, Hartree, xc, potential (mixed unless first), energies of the
// current orthonormal orbitals of every active system.
int evaluate(lbks_system* s, cudaStream_t st, int first) {
    const int B = s->B;
    cudaError_t e = s->ops->density(s->n_orb, s->g, s->h, s->psi, s->rho, s->rho_ref, s->mp, s->sc, B, st);
    if (e != cudaSuccess) return cuda_fail(e, "density");
    int rc = hartree_solve(s, st, true);
    if (rc != LBKS_OK) return rc;
    e = launch_potential(s->g, s->h, s->rho, s->vext, s->vh, s->vout, s->vin, first, s->prm.mix, s->e4, s->sc, B, st);
    if (e != cudaSuccess) return cuda_fail(e, "potential");
    e = s->ops->energy_matrix(s->n_orb, s->g, s->c, s->psi, s->vout, s->emat, s->sc, B, st);
    if (e != cudaSuccess) return cuda_fail(e, "energy matrix");
    const int no = s->n_orb;
    for (int i = 0; i < B && e == cudaSuccess; ++i) {
        e = cudaMemcpyAsync(host_e4(s, i), s->e4 + (size_t)i * kE4Stride, sizeof(double) * kE4Stride,
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_emat(s, i), s->emat + (size_t)i * emat_stride(no), sizeof(double) * (no * no + no),
                                cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_drho(s, i), s->mp + (size_t)i * kMpStride + 10, sizeof(double) * 2,
                                cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_status(s), s->status, sizeof(int) * B, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "energy readback");
    const int* act = host_active(s);
    for (int i = 0; i < B; ++i) {
        if (!act[i]) continue;
        if (host_status(s)[i] != 0)
            return fail(LBKS_ENOTCONV, "system %d: overlap matrix not positive definite at orbital %d", i,
                        host_status(s)[i] - 1);
        const double* h4 = host_e4(s, i);
        const double* hm = host_emat(s, i);
        lbks_energy_terms& t = s->terms[i];
        memset(&t, 0, sizeof t);
        double ts = 0.0;
        for (int j = 0; j < no; ++j) ts += hm[no * no + j];
        t.T_s = 2.0 * ts;
        t.E_ext = h4[0];
        t.E_H = 0.5 * h4[1];
        t.E_xc = h4[2];
        t.n_electrons = h4[3];
        double enn = 0.0;
        const std::vector<double>& xyz = s->xyz[i];
        const std::vector<double>& Z = s->Z[i];
        const int na = (int)Z.size();
        for (int a = 0; a < na; ++a)
            for (int b = 0; b < a; ++b) {
                const double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1],
                             dz = xyz[3 * a + 2] - xyz[3 * b + 2];
                enn += Z[a] * Z[b] / std::sqrt(dx * dx + dy * dy + dz * dz);
            }
        t.E_nn = enn;
        t.E_total = t.T_s + t.E_ext + t.E_H + t.E_xc + t.E_nn;
        std::vector<double> H(no * no);
        for (int j = 0; j < no; ++j) {
            t.orbital_energies[j] = hm[j * no + j];
            for (int k = 0; k < no; ++k) H[j * no + k] = 0.5 * (hm[j * no + k] + hm[k * no + j]);
        }
        jacobi_eigenvalues(no, H, t.eigenvalues);
        const double* dr = host_drho(s, i);
        s->drho[i] = dr[1] > 0.0 ? std::sqrt(std::max(dr[0], 0.0) / dr[1]) : INFINITY;
    }
    return LBKS_OK;
}

// The same cycle in orbital storage (omega = 1): f[] hold psi; the first step
// pulls with the previous cycle's collision potential (vprev), later steps
// with this cycle's (vin); the cycle ends by keeping vin as vprev.
cudaError_t enqueue_cycle_psi(lbks_system* s, cudaStream_t st, int start) {
    int cur = start;
    const int n = s->prm.n_inner, B = s->B;
    // up to kMaxOrb orbitals, and at any count with the TMA kernel, the step
    // forms the W source from Lambda itself; otherwise it pulls the W field u
    const bool fused_w = s->n_orb <= kMaxOrb || (s->variant & kRelaxVariantMask) == kPsiKernelTma;
    for (int t = 0; t < n; ++t) {
        RelaxIO io{s->f[cur], (t == 0 || fused_w) ? nullptr : s->u, t == 0 ? s->vprev : s->vin, s->sigma,
                   s->f[1 - cur], s->f[1 - cur], s->S, s->lam, s->sigma, (t == 0 || !fused_w) ? nullptr : s->lam};
        const int v = s->variant | (t == n - 1 ? kRelaxExactOverlap : 0);  // the last overlap feeds the Cholesky
        cudaError_t e = s->ops->relax_psi(s->n_orb, s->g, s->c, io, s->sc, B, v, st);
        if (e != cudaSuccess) return e;
        cur ^= 1;
        if (t < n - 1 && !fused_w) {
            e = s->ops->w_field(s->n_orb, s->g, s->prm.omega, s->f[cur], s->lam, s->u, B, st);
            if (e != cudaSuccess) return e;
        }
    }
    cudaError_t e = launch_cholesky(s->n_orb, s->S, s->Linv, s->status, s->active, B, st);
    if (e == cudaSuccess) e = s->ops->orth_apply(s->n_orb, s->g, s->Linv, nullptr, s->f[cur], B, st);
    if (e == cudaSuccess) e = launch_fill(s->sigma, (size_t)s->n_orb * B, 1.0, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->vprev, s->vin, sizeof(double) * s->N * B, cudaMemcpyDeviceToDevice, st);
    return e;
}

// n_inner - 1 steps of Eq. KSLB and one orthonormalising step, starting from f[start].
cudaError_t enqueue_cycle(lbks_system* s, cudaStream_t st, int start) {
    if (s->psi_storage) return enqueue_cycle_psi(s, st, start);
    int cur = start;
    const int n = s->prm.n_inner, B = s->B;
    for (int t = 0; t < n; ++t) {
        RelaxIO io{s->f[cur], t == 0 ? nullptr : s->u, s->vin, s->sigma, s->f[1 - cur], s->psi, s->S, s->lam, s->sigma};
        const int v = s->variant | (t == n - 1 ? kRelaxExactOverlap : 0);  // the last overlap feeds the Cholesky
        cudaError_t e = s->ops->relax(s->n_orb, s->g, s->c, io, s->sc, B, v, st);
        if (e != cudaSuccess) return e;
        cur ^= 1;
        if (t < n - 1) {
            e = s->ops->w_field(s->n_orb, s->g, s->prm.omega, s->psi, s->lam, s->u, B, st);
            if (e != cudaSuccess) return e;
        }
    }
    cudaError_t e = launch_cholesky(s->n_orb, s->S, s->Linv, s->status, s->active, B, st);
    if (e == cudaSuccess) e = s->ops->orth_apply(s->n_orb, s->g, s->Linv, s->f[cur], s->psi, B, st);
    if (e == cudaSuccess) e = launch_fill(s->sigma, (size_t)s->n_orb * B, 1.0, st);
    return e;
}

int cycle_graph(lbks_system* s, int start) {
    if (s->graph[start]) return LBKS_OK;
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    g_capturing = true;
    cudaError_t ee = enqueue_cycle(s, s->cap, start);
    g_capturing = false;
    e = cudaStreamEndCapture(s->cap, &gr);
    if (ee != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return cuda_fail(ee, "capture relaxation cycle");
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    size_t nodes = 0;
    cudaGraphGetNodes(gr, nullptr, &nodes);
    e = cudaGraphInstantiate(&s->graph[start], gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate graph");
    s->graph_nodes[start] = nodes;
    return LBKS_OK;
}

int upload_active(lbks_system* s, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(s->active, host_active(s), sizeof(int) * s->B, cudaMemcpyHostToDevice, st);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "upload active flags");
}

// BF16 -> FP32 switch: widen the current populations, continue with FP32
// kernels (orbitals, W field and scalars are float already).
int polish(lbks_system* s, cudaStream_t st) {
    cudaError_t e = launch_bf16_to_f32(s->f[s->cur], s->f_wide[s->cur], s->N * s->B * 19 * s->n_orb, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "polish switch");
    for (int k = 0; k < 2; ++k) {
        if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
        s->graph[k] = nullptr;
        std::swap(s->f[k], s->f_wide[k]);
    }
    s->ops = &ops_f32();
    s->polished = true;
    return LBKS_OK;
}

// Keeps the current density as the reference of the stop rule's next block
// (the density kernel measures the change against it).
int mark_block(lbks_system* s, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(s->rho_ref, s->rho, sizeof(double) * s->N * s->B, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "reference density");
}

// Relaxation cycles of all systems in lock step; a system stops (drops out
// of every launch) once the stop rule holds for it (include/lbks.h), unless
// `fixed` (exactly n cycles).
int run_cycles(lbks_system* s, int fixed, int n, cudaStream_t st, lbks_result* out) {
    if (!s->ready) return fail(LBKS_EINVAL, "geometry has not been set");
    const int B = s->B, no = s->n_orb;
    const auto t0 = std::chrono::steady_clock::now();
    // per cycle: the energy (BF16 polish switch, lbks_result.dE); per block of
    // kStopBlock cycles: energy, eigenvalues and density (the stop rule)
    std::vector<double> prev(B), ref_E(B), ref_eig((size_t)B * no), de1(B, INFINITY), de2(B, INFINITY);
    std::vector<Changes> dE(B), dEig(B), dRho(B);
    std::vector<int> cycles(B, 0), converged(B, 0);
    int* act = host_active(s);
    for (int i = 0; i < B; ++i) {
        prev[i] = ref_E[i] = s->terms[i].E_total;
        for (int j = 0; j < no; ++j) ref_eig[(size_t)i * no + j] = s->terms[i].eigenvalues[j];
        act[i] = 1;
    }
    int rc = upload_active(s, st);
    if (rc == LBKS_OK) rc = mark_block(s, st);  // the current density starts the first block
    if (rc != LBKS_OK) return rc;
    const int limit = fixed ? n : s->prm.max_cycles;
    const int start_iters = s->poisson_iters;
    const double start_poisson_ms = s->poisson_ms;
    int cycles_polished = 0;
    for (int c = 0; c < limit; ++c) {
        rc = cycle_graph(s, s->cur);
        if (rc != LBKS_OK) return rc;
        cudaError_t e = cudaGraphLaunch(s->graph[s->cur], st);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        count_launches(s->graph_nodes[s->cur]);
        s->cur ^= (s->prm.n_inner & 1);
        if (s->psi_storage) s->psi = s->f[s->cur];
        rc = evaluate(s, st, 0);
        if (rc != LBKS_OK) return rc;
        // A BF16 handle with a polish phase converges only in FP32, and only
        // after two FP32 cycles have washed the bfloat16 rounding out of the
        // orbitals (the energy is second order in it, eigenvalues first order).
        const bool wait_polish = s->f_wide[0] && !fixed && (!s->polished || cycles_polished < 2);
        int remaining = 0;
        bool ready = true;
        const bool block_end = (c + 1) % kStopBlock == 0;
        for (int i = 0; i < B; ++i) {
            if (!act[i]) continue;
            ++cycles[i];
            const lbks_energy_terms& t = s->terms[i];
            if (!std::isfinite(t.E_total)) return fail(LBKS_ENOTCONV, "system %d: energy not finite", i);
            // per cycle: ready for FP32 storage below polish_tol, or stalled at
            // the bfloat16 noise floor (|dE| no longer halving over two cycles)
            de2[i] = de1[i];
            de1[i] = std::fabs(t.E_total - prev[i]);
            prev[i] = t.E_total;
            const bool stalled = de1[i] < 100.0 * s->prm.polish_tol && de1[i] > 0.5 * de2[i];
            if (!(de1[i] < s->prm.polish_tol || stalled)) ready = false;
            if (!block_end) {
                ++remaining;
                continue;
            }
            double de_eig = 0.0;
            for (int j = 0; j < no; ++j) {
                de_eig = std::max(de_eig, std::fabs(t.eigenvalues[j] - ref_eig[(size_t)i * no + j]));
                ref_eig[(size_t)i * no + j] = t.eigenvalues[j];
            }
            dE[i].push(std::fabs(t.E_total - ref_E[i]));
            dEig[i].push(de_eig);
            dRho[i].push(s->drho[i]);
            ref_E[i] = t.E_total;
            // rounding floors: FP64 orbitals 2^-53, FP32 (and the BF16 handle's
            // FP32 polish) 2^-24, scaled by |E|, max |eps_j| and 1
            const double u = s->ops->psi_elem == sizeof(double) ? 0x1.0p-53 : 0x1.0p-24;
            double eig_scale = 0.0;
            for (int j = 0; j < no; ++j) eig_scale = std::max(eig_scale, std::fabs(t.eigenvalues[j]));
            if (!fixed && !wait_polish && dE[i].settled(s->prm.e_tol, kFloorUlps * u * std::fabs(t.E_total)) &&
                dEig[i].settled(s->prm.eig_tol, kFloorUlps * u * eig_scale) &&
                dRho[i].settled(s->prm.rho_tol, kFloorUlps * u)) {
                converged[i] = 1;
                act[i] = 0;
            } else {
                ++remaining;
            }
        }
        if (block_end) {
            rc = mark_block(s, st);
            if (rc != LBKS_OK) return rc;
        }
        if (s->polished) ++cycles_polished;
        if (!remaining) break;
        if (!s->polished && s->f_wide[0] && !fixed && ready) {
            rc = polish(s, st);
            if (rc != LBKS_OK) return rc;
        }
        if (!fixed) {
            rc = upload_active(s, st);
            if (rc != LBKS_OK) return rc;
        }
    }
    const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int all = 1;
    for (int i = 0; i < B; ++i) {
        all &= converged[i] || fixed;
        if (!out) continue;
        lbks_result& r = out[i];
        memset(&r, 0, sizeof r);
        r.E_total = s->terms[i].E_total;
        r.dE = de1[i];
        for (int j = 0; j < no; ++j) r.eigenvalues[j] = s->terms[i].eigenvalues[j];
        r.n_electrons = s->terms[i].n_electrons;
        r.cycles = cycles[i];
        r.steps = cycles[i] * s->prm.n_inner;
        r.converged = converged[i];
        r.poisson_iters = s->poisson_iters - start_iters;
        r.wall_s = wall;
        r.poisson_s = 1e-3 * (s->poisson_ms - start_poisson_ms);
        r.d_eig = dEig[i].d[0];
        r.d_rho = dRho[i].d[0];
        r.err_E = dE[i].tail();
        r.err_eig = dEig[i].tail();
        r.err_rho = dRho[i].tail();
    }
    if (!all) return fail(LBKS_ENOTCONV, "not every system converged within %d cycles", limit);
    return LBKS_OK;
}

// ---------------------------------------------------------- kernel tuner
// The stream-collide variant (one site per thread, two x-neighbouring sites
// per thread, one site with the next orbital prefetched) is chosen per shape
// by timing all on the first handle of that shape, process-wide: key
// (precision, orbitals, omega == 1, nx, ny, nz, systems).  Up to kMaxOrb
// orbitals only; wider sets have one kernel.
using TuneKey = std::tuple<int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;
std::atomic<int> g_variant_mode{0};  // 0 tuned, else 1 + the forced variant
// Orbital storage, up to kMaxOrb orbitals: the staged kernel's tile shape,
// -1 tuned per grid shape (step-level calls: the default shape), else forced.
std::atomic<int> g_psi_shape{-1};

TuneKey tune_key(int precision, int n_orb, double omega, int nx, int ny, int nz, int B) {
    return TuneKey(precision, n_orb, omega == 1.0 ? 1 : 0, nx, ny, nz, B);
}

// Variant for a launch outside a handle (lbks_relax_step): forced, tuned for
// the shape, else one site per thread.
int variant_for(int precision, int n_orb, double omega, int nx, int ny, int nz) {
    const int mode = g_variant_mode.load();
    // more than kMaxOrb orbitals: one orbital per thread at one or two sites, or the bulk-copy kernel
    auto wide_ok = [&](int v) { return n_orb <= kMaxOrb || v == kRelaxBulk || v == kRelaxPairs ? v : kRelaxSites; };
    if (mode > 0) return wide_ok(mode - 1);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(tune_key(precision, n_orb, omega, nx, ny, nz, 1));
    if (it == g_tuned.end()) return kRelaxSites;
    return wide_ok(it->second);
}

// Times both variants on the handle's own buffers before they hold state
// (called at the start of initialise: populations, orbitals, S, Lambda and
// sigma are all rewritten afterwards).  A few launches, once per shape.
int tune_relax(lbks_system* s) {
    const int mode = g_variant_mode.load();
    // orbital storage: the TMA kernel where its tensor maps apply
    const bool tma_ok = s->psi_storage && psi_tma_applies(s->nx, s->f[0], s->vin, s->ops->psi_elem) &&
                        psi_tma_applies(s->nx, s->f[1], s->vprev, s->ops->psi_elem);
    const int forced_shape = g_psi_shape.load();
    const bool shaped = s->psi_storage && s->n_orb <= kMaxOrb;  // the staged kernel takes a tile shape
    if (mode > 0) {
        s->variant = mode - 1;
        if (s->psi_storage && ((s->variant == kPsiKernelZ && s->n_orb > kMaxOrb) ||
                               (s->variant == kPsiKernelTma && !tma_ok)))
            s->variant = kPsiKernelTiled;
        if (!s->psi_storage && s->n_orb > kMaxOrb && s->variant != kRelaxBulk && s->variant != kRelaxPairs)
            s->variant = kRelaxSites;
        if (shaped && forced_shape > 0) s->variant |= forced_shape << kPsiShapeShift;
        return LBKS_OK;
    }
    // the bulk-copy kernel: omega = 1, FP32 or bfloat16 populations, N a multiple of 8
    // (the launch checks alignment too and falls back to the one-site kernel)
    const bool bulk_may = !s->psi_storage && s->prm.omega == 1.0 && s->prm.precision != LBKS_FP64 && s->N % 8 == 0;
    // more than kMaxOrb orbitals: the one-orbital-per-thread population kernel
    // at one and at two sites per thread against the bulk-copy kernel; in
    // orbital storage the tiled step with its W-field pass against the TMA step
    const bool wide = s->n_orb > kMaxOrb;
    if (wide && (s->psi_storage ? !tma_ok : (!bulk_may && s->nx % 2 != 0))) {
        s->variant = kRelaxSites;
        return LBKS_OK;
    }
    // orbital storage has its own kernels (0: tiled in shared memory, 1: one site per thread, 2: TMA)
    const TuneKey key = tune_key(s->prm.precision + (s->psi_storage ? 16 : 0) + (forced_shape >= 0 ? 32 * (1 + forced_shape) : 0),
                                 s->n_orb, s->prm.omega, s->nx, s->ny, s->nz, s->B);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            s->variant = it->second;
            return LBKS_OK;
        }
    }
    cudaStream_t st = s->st;
    const size_t NB = s->N * s->B;
    cudaError_t e = cudaMemsetAsync(
        s->f[0], 0, s->psi_storage ? s->ops->psi_elem * NB * s->n_orb : s->ops->elem * NB * 19 * s->n_orb, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->vin, 0, sizeof(double) * NB, st);
    if (e == cudaSuccess) e = launch_fill(s->sigma, (size_t)s->n_orb * s->B, 1.0, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->lam, 0, sizeof(double) * s->n_orb * s->n_orb * s->B, st);
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
    const RelaxIO io = s->psi_storage
                           ? RelaxIO{s->f[0], nullptr, s->vin, s->sigma, s->f[1], s->f[1], s->S, s->lam, s->sigma,
                                     nullptr}
                           : RelaxIO{s->f[0], s->n_orb > 1 ? s->u : nullptr, s->vin, s->sigma, s->f[1], s->psi, s->S,
                                     s->lam, s->sigma};
    auto relax = s->psi_storage ? s->ops->relax_psi : s->ops->relax;
    // one step of variant v; wide orbital storage: with the W source as the
    // cycle forms it (the W-field kernel before the tiled step, Lambda inside the TMA step)
    auto step = [&](int v) -> cudaError_t {
        RelaxIO sio = io;
        if (wide && v == kPsiKernelTma) sio.lambda_in = s->lam;
        if (wide && v != kPsiKernelTma) {
            sio.u_in = s->u;
            cudaError_t we = s->ops->w_field(s->n_orb, s->g, s->prm.omega, s->f[0], s->lam, s->u, s->B, st);
            if (we != cudaSuccess) return we;
        }
        return relax(s->n_orb, s->g, s->c, sio, s->sc, s->B, v, st);
    };
    constexpr int kReps = 3;
    auto timed = [&](int v, float* out) -> cudaError_t {
        cudaError_t te = step(v);  // warm-up
        if (te == cudaSuccess) te = cudaEventRecord(ev[0], st);
        for (int r = 0; r < kReps && te == cudaSuccess; ++r) te = step(v);
        if (te == cudaSuccess) te = cudaEventRecord(ev[1], st);
        if (te == cudaSuccess) te = cudaEventSynchronize(ev[1]);
        if (te == cudaSuccess) te = cudaEventElapsedTime(out, ev[0], ev[1]);
        return te;
    };
    // orbital storage: the staged kernel's tile shape first (forced, or the fastest)
    int shape = forced_shape >= 0 ? forced_shape : 0;
    if (shaped && forced_shape < 0) {
        float best = 0.f;
        for (int k = 0; k < kPsiShapes && e == cudaSuccess; ++k) {
            if (!psi_tile_runs((int)s->ops->psi_elem, s->n_orb, k)) continue;  // would run shape 0
            float t = 0.f;
            e = timed(kPsiKernelTiled | (k << kPsiShapeShift), &t);
            s->tune_shape_ms[k] = t / kReps;
            if (k == 0 || t < best) {
                best = t;
                shape = k;
            }
        }
    }
    const int tiled_v = shaped ? (kPsiKernelTiled | (shape << kPsiShapeShift)) : kPsiKernelTiled;
    float ms[kRelaxVariants] = {0.f, 0.f, 0.f, 0.f};
    // variants that differ from the first kernel on this shape
    bool tried[kRelaxVariants] = {true, s->psi_storage ? !wide : s->nx % 2 == 0,
                                  s->psi_storage ? tma_ok : (!wide && s->n_orb > 1),
                                  s->psi_storage ? !wide : bulk_may};
    for (int v = 0; v < kRelaxVariants && e == cudaSuccess; ++v) {
        if (!tried[v]) continue;
        e = timed(v == kPsiKernelTiled && s->psi_storage ? tiled_v : v, &ms[v]);
    }
    for (int k = 0; k < 3; ++k)
        if (ev[k]) cudaEventDestroy(ev[k]);
    if (e != cudaSuccess) return cuda_fail(e, "stream-collide tuning");
    int best = kRelaxSites;
    for (int v = 0; v < kRelaxVariants; ++v) {
        s->tune_ms[v] = tried[v] ? ms[v] / kReps : -1.0;
        if (tried[v] && ms[v] < ms[best]) best = v;
    }
    // the tuned shape rides along whichever kernel wins (the others ignore it)
    s->variant = best | (shaped ? shape << kPsiShapeShift : 0);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.emplace(key, s->variant);
    return LBKS_OK;
}

// Device layout of the nuclei: atoms[B][kMaxAtoms][4] = (x, y, z, Z), counts[B].
void pack_atoms(const lbks_system* s, std::vector<double>& atoms, std::vector<int>& counts) {
    atoms.assign((size_t)s->B * kMaxAtoms * 4, 0.0);
    counts.assign(s->B, 0);
    for (int i = 0; i < s->B; ++i) {
        const std::vector<double>& xyz = s->xyz[i];
        const std::vector<double>& Z = s->Z[i];
        const int na = (int)Z.size();
        counts[i] = na;
        for (int a = 0; a < na; ++a) {
            double* d = &atoms[((size_t)i * kMaxAtoms + a) * 4];
            d[0] = xyz[3 * a];
            d[1] = xyz[3 * a + 1];
            d[2] = xyz[3 * a + 2];
            d[3] = Z[a];
        }
    }
}

// Gaussian starts, orthonormalisation, equilibrium populations and the first
// evaluation for every system of the handle (all must have atoms).
int initialise(lbks_system* s) {
    const int B = s->B;
    if (s->polished) {  // start again in bfloat16
        for (int k = 0; k < 2; ++k) {
            if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
            s->graph[k] = nullptr;
            std::swap(s->f[k], s->f_wide[k]);
        }
        s->ops = ops_for(s->prm.precision);
        s->polished = false;
    }
    for (int i = 0; i < B; ++i)
        if (!s->has_atoms[i]) return fail(LBKS_EINVAL, "system %d has no geometry", i);
    cudaStream_t st = s->st;
    std::vector<double> atoms;
    std::vector<int> counts;
    pack_atoms(s, atoms, counts);
    std::vector<OrbitalStart> starts((size_t)B * s->n_orb);
    for (int i = 0; i < B; ++i) {
        const std::vector<double>& xyz = s->xyz[i];
        const std::vector<double>& Z = s->Z[i];
        const int na = (int)Z.size();
        std::vector<int> order(na);
        for (int a = 0; a < na; ++a) order[a] = a;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return Z[a] > Z[b]; });
        const std::vector<double> off = start_offsets(s->n_orb, s->prm.seed);
        for (int j = 0; j < s->n_orb; ++j) {
            const int I = order[j % na], m = j / na;
            OrbitalStart& o = starts[(size_t)i * s->n_orb + j];
            o.cx = xyz[3 * I] + off[3 * j];
            o.cy = xyz[3 * I + 1] + off[3 * j + 1];
            o.cz = xyz[3 * I + 2] + off[3 * j + 2];
            o.width = 1.2 * (1.0 + 0.35 * m);
        }
    }
    int* act = host_active(s);
    for (int i = 0; i < B; ++i) act[i] = 1;
    cudaError_t e = cudaMemcpyAsync(s->atoms, atoms.data(), sizeof(double) * atoms.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->counts, counts.data(), sizeof(int) * B, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->starts, starts.data(), sizeof(OrbitalStart) * starts.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->active, act, sizeof(int) * B, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "initialise orbitals");
    int trc = tune_relax(s);
    if (trc != LBKS_OK) return trc;
    if (e == cudaSuccess) e = launch_vext(s->g, s->h, s->counts, s->atoms, s->a, s->vext, B, st);
    if (s->psi_storage) {  // orbitals in f[0]; the start f = xi psi has no potential term: vprev = 0
        s->psi = s->f[0];
        if (e == cudaSuccess) e = cudaMemsetAsync(s->vprev, 0, sizeof(double) * s->N * B, st);
    }
    if (e == cudaSuccess) e = s->ops->init_orbitals(s->n_orb, s->g, s->h, s->starts, s->psi, B, st);
    if (e == cudaSuccess) e = s->ops->gram(s->n_orb, s->g, s->h, s->psi, s->S, s->sc, B, st);
    if (e == cudaSuccess) e = launch_cholesky(s->n_orb, s->S, s->Linv, s->status, s->active, B, st);
    if (e == cudaSuccess) e = s->ops->orth_apply(s->n_orb, s->g, s->Linv, nullptr, s->psi, B, st);
    if (e == cudaSuccess && !s->psi_storage) e = s->ops->equilibrium(s->n_orb, s->g, s->c, s->psi, s->f[0], B, st);
    if (e == cudaSuccess) e = launch_fill(s->sigma, (size_t)s->n_orb * B, 1.0, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->vh, 0, sizeof(double) * s->N * B, st);
    if (e != cudaSuccess) return cuda_fail(e, "initialise orbitals");
    s->cur = 0;
    s->poisson_iters = 0;
    s->ready = true;
    int rc = evaluate(s, st, 1);
    if (rc != LBKS_OK) {
        s->ready = false;
        return rc;
    }
    return mark_block(s, st);
}

int check_atoms(const lbks_system* s, int n_atoms, const double* xyz, const double* Z) {
    if (!xyz || !Z) return fail(LBKS_EINVAL, "null argument");
    if (n_atoms < 1 || n_atoms > kMaxAtoms) return fail(LBKS_EINVAL, "n_atoms must be in [1, %d]", kMaxAtoms);
    double zsum = 0.0;
    const double hx = 0.5 * (s->nx - 1) * s->h, hy = 0.5 * (s->ny - 1) * s->h, hz = 0.5 * (s->nz - 1) * s->h;
    for (int i = 0; i < n_atoms; ++i) {
        if (!(std::fabs(xyz[3 * i]) <= hx && std::fabs(xyz[3 * i + 1]) <= hy && std::fabs(xyz[3 * i + 2]) <= hz))
            return fail(LBKS_EINVAL, "atom %d lies outside the box", i);
        if (!(Z[i] > 0.0)) return fail(LBKS_EINVAL, "atom %d has non-positive charge", i);
        zsum += Z[i];
    }
    if (std::fabs(zsum - 2.0 * s->n_orb) > 1e-9)
        return fail(LBKS_EINVAL, "sum of Z (%g) must equal 2 n_orb (%d): closed-shell neutral systems only", zsum,
                    2 * s->n_orb);
    return LBKS_OK;
}

void free_system(lbks_system* s) {
    for (int k = 0; k < 2; ++k) {
        if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
        if (s->f[k]) cudaFree(s->f[k]);
        if (s->f_wide[k]) cudaFree(s->f_wide[k]);
    }
    if (s->poisson_graph) cudaGraphExecDestroy(s->poisson_graph);
    if (s->psi_storage) s->psi = nullptr;  // an alias of f[cur]
    void* ptrs[] = {s->u,   s->psi,   s->vin,    s->vout,          s->vext,          s->vh, s->rho, s->pvec,
                    s->cg,  s->small, s->ints,   s->starts,        s->sc.partial,    s->sc.counter, s->vprev,
                    s->rho_ref};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (void* p : s->cd_lev)
        if (p) cudaFree(p);
    void* cdp[] = {s->cd_small, s->cd_sc.partial, s->cd_sc.counter};
    for (void* p : cdp)
        if (p) cudaFree(p);
    for (cudaEvent_t ev : s->pev)
        if (ev) cudaEventDestroy(ev);
    if (s->host) cudaFreeHost(s->host);
    if (s->st) cudaStreamDestroy(s->st);
    if (s->cap) cudaStreamDestroy(s->cap);
    delete s;
}

size_t bytes_of(const lbks_params* p, int nx, int ny, int nz, int n_orb, int B) {
    const size_t N = (size_t)nx * ny * nz;
    const size_t e = ops_for(p->precision)->elem, ep = ops_for(p->precision)->psi_elem;
    const bool psi = p->storage == LBKS_STORE_PSI;  // f[] hold psi, no separate psi array, one more field
    const size_t per = (psi ? ep * N * (size_t)n_orb * 2 : e * N * (size_t)n_orb * 19 * 2) +
                       ep * N * ((size_t)std::max(1, n_orb - 1) + (psi ? 0 : n_orb)) +
                       sizeof(double) * N * (psi ? 13 : 12) + sizeof(double) * mg_coarse_doubles(nx, ny, nz) +
                       sizeof(double) * ((size_t)num_sms() * 8 * scratch_vals(n_orb) + small_per_sys(n_orb) +
                                         7 * kMaxAtoms) +
                       ((p->precision == LBKS_BF16 && p->polish_tol > 0.0) ? sizeof(float) * N * n_orb * 19 * 2 : 0);
    return per * B;
}

int create(const lbks_params* p, int nx, int ny, int nz, double h, int n_orb, int B, lbks_system** out) {
    if (!out) return fail(LBKS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!valid_params(p)) return fail(LBKS_EINVAL, "invalid lbks_params");
    if (nx < 2 || ny < 2 || nz < 2) return fail(LBKS_EINVAL, "grid must be at least 2 sites per axis");
    if (!(h > 0.0)) return fail(LBKS_EINVAL, "h must be positive");
    if (n_orb < 1 || n_orb > kMaxOrbWide) return fail(LBKS_EINVAL, "n_orb must be in [1, %d]", kMaxOrbWide);
    if (B < 1 || B > 4096) return fail(LBKS_EINVAL, "n_systems must be in [1, 4096]");
    if ((size_t)nx * ny * nz >= (1ull << 31)) return fail(LBKS_EINVAL, "grid has 2^31 sites or more");
    lbks_system* s = new lbks_system();
    s->prm = *p;
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->n_orb = n_orb;
    s->B = B;
    s->h = h;
    s->dt = p->theta * h * h * (2.0 - p->omega) / p->omega;
    s->a = p->softening > 0.0 ? p->softening : h;
    s->g = make_grid(nx, ny, nz);
    s->c = make_coef(p->omega, p->theta, s->dt, h);
    s->ops = ops_for(p->precision);
    s->N = (size_t)nx * ny * nz;
    cudaGetDevice(&s->dev);
    s->terms.assign(B, lbks_energy_terms{});
    s->drho.assign(B, INFINITY);
    s->xyz.assign(B, {});
    s->Z.assign(B, {});
    s->has_atoms.assign(B, 0);
    const size_t e = s->ops->elem, ep = s->ops->psi_elem, N = s->N, NB = N * B;
    cudaError_t err = cudaSuccess;
    auto A = [&](void** ptr, size_t bytes) {
        if (err == cudaSuccess) err = cudaMalloc(ptr, bytes);
    };
    s->psi_storage = p->storage == LBKS_STORE_PSI;
    const size_t fbytes = s->psi_storage ? ep * NB * n_orb : e * NB * 19 * n_orb;
    A(&s->f[0], fbytes);
    A(&s->f[1], fbytes);
    if (s->psi_storage) A((void**)&s->vprev, 8 * NB);
    if (p->precision == LBKS_BF16 && p->polish_tol > 0.0) {
        A(&s->f_wide[0], sizeof(float) * NB * 19 * n_orb);
        A(&s->f_wide[1], sizeof(float) * NB * 19 * n_orb);
    }
    A(&s->u, ep * NB * std::max(1, n_orb - 1));
    if (!s->psi_storage) A(&s->psi, ep * NB * n_orb);
    A((void**)&s->vin, 8 * NB);
    A((void**)&s->vout, 8 * NB);
    A((void**)&s->vext, 8 * NB);
    A((void**)&s->vh, 8 * NB);
    A((void**)&s->rho, 8 * NB);
    A((void**)&s->rho_ref, 8 * NB);
    A((void**)&s->pvec, 8 * (6 * NB + B * mg_coarse_doubles(nx, ny, nz)));
    A((void**)&s->cg, sizeof(CGState) * B);
    A((void**)&s->small, sizeof(double) * (small_per_sys(n_orb) + 7 * kMaxAtoms) * B);
    A((void**)&s->ints, sizeof(int) * 3 * B);
    A((void**)&s->starts, sizeof(OrbitalStart) * n_orb * B);
    if (err == cudaSuccess) {
        s->sc.max_blocks = num_sms() * 8;
        s->sc.max_vals = scratch_vals(n_orb);
        s->sc.systems = B;
        err = cudaMalloc(&s->sc.partial, sizeof(double) * (size_t)s->sc.max_blocks * s->sc.max_vals * B);
    }
    A((void**)&s->sc.counter, sizeof(unsigned) * B);
    if (err == cudaSuccess)
        err = cudaMallocHost((void**)&s->host, sizeof(double) * (host_per_sys(n_orb) * B + B + 1) +
                                                   sizeof(CGState) * B + sizeof(int) * 2 * B + 64);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    // Zeroed on the handle's own stream and waited for: a legacy-stream
    // cudaMemset returns before it runs and is not ordered before work on
    // non-blocking streams (the caller's, or a server slot's), which could
    // then see the arrival counters or the active flags reset mid-solve.
    if (err == cudaSuccess) err = cudaMemsetAsync(s->sc.counter, 0, sizeof(unsigned) * B, s->st);
    if (err == cudaSuccess) err = cudaMemsetAsync(s->vh, 0, 8 * NB, s->st);
    if (err == cudaSuccess) err = cudaMemsetAsync(s->rho, 0, 8 * NB, s->st);
    if (err == cudaSuccess) err = cudaMemsetAsync(s->rho_ref, 0, 8 * NB, s->st);
    if (err == cudaSuccess) err = cudaMemsetAsync(s->u, 0, ep * NB * std::max(1, n_orb - 1), s->st);
    if (err == cudaSuccess) err = cudaMemsetAsync(s->ints, 0, sizeof(int) * 3 * B, s->st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s->st);
    if (err != cudaSuccess) {
        int rc = cuda_fail(err, "create system");
        free_system(s);
        return rc;
    }
    s->status = s->ints;
    s->active = s->ints + B;
    s->counts = s->ints + 2 * B;
    s->g.active = s->active;
    s->mg = make_hierarchy(s->g, s->pvec + 6 * NB, B);
    const size_t M = (size_t)n_orb * n_orb;
    s->S = s->small;
    s->lam = s->S + M * B;
    s->Linv = s->lam + M * B;
    s->sigma = s->Linv + M * B;
    s->e4 = s->sigma + (size_t)n_orb * B;
    s->emat = s->e4 + (size_t)kE4Stride * B;
    s->mp = s->emat + (size_t)emat_stride(n_orb) * B;
    s->atoms = s->mp + (size_t)kMpStride * B;
    s->forces = s->atoms + (size_t)4 * kMaxAtoms * B;  // [B][kMaxAtoms][3]
    *out = s;
    return LBKS_OK;
}

int copy_field(const lbks_system* s, int system, const double* base, double* host, size_t cap, const char* what) {
    if (system < 0 || system >= s->B) return fail(LBKS_EINVAL, "system index out of range");
    if (cap < s->N) return fail(LBKS_EINVAL, "capacity %zu < %zu", cap, s->N);
    cudaError_t e = cudaMemcpyAsync(host, base + (size_t)system * s->N, sizeof(double) * s->N,
                                    cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, what);
}

}  // namespace

int lbks::relax_variant_for(int precision, int n_orb, double omega, int nx, int ny, int nz) {
    return variant_for(precision, n_orb, omega, nx, ny, nz);
}

extern "C" {

int lbks_set_psi_tile(int shape) {
    if (shape < -1 || shape >= kPsiShapes) {
        fail(LBKS_EINVAL, "shape must be in [-1, %d]", kPsiShapes - 1);
        return -2;
    }
    return g_psi_shape.exchange(shape);
}

int lbks_get_psi_tile(const lbks_system* s, int* shape, double* ms) {
    if (!s || !shape) return fail(LBKS_EINVAL, "null argument");
    *shape = (s->variant >> kPsiShapeShift) & 0xff;
    if (ms)
        for (int k = 0; k < kPsiShapes; ++k) ms[k] = s->tune_shape_ms[k];
    return LBKS_OK;
}

int lbks_set_relax_variant(int mode) {
    if (mode < 0 || mode > kRelaxVariants) return -1;
    return g_variant_mode.exchange(mode);
}

int lbks_get_relax_variant(const lbks_system* s, int* variant, double* ms) {
    if (!s || !variant) return fail(LBKS_EINVAL, "null argument");
    *variant = s->variant & kRelaxVariantMask;
    if (ms)
        for (int v = 0; v < kRelaxVariants; ++v) ms[v] = s->tune_ms[v];
    return LBKS_OK;
}

void lbks_params_default(lbks_params* p) {
    if (!p) return;
    p->omega = 1.0;
    p->theta = 0.5;
    p->n_inner = 50;
    p->mix = 0.5;
    p->e_tol = 1e-6;
    p->max_cycles = 200;
    p->precision = LBKS_FP64;
    p->softening = 0.0;
    p->poisson_rtol = 1e-11;
    p->poisson_adapt = 0.0;
    p->poisson_max_iter = 20000;
    p->polish_tol = 1e-4;
    p->storage = LBKS_STORE_POPULATIONS;
    p->eig_tol = 2e-6;
    p->rho_tol = 2e-6;
    p->seed = 0;
}

int lbks_last_error(char* buf, size_t cap) {
    if (buf && cap) {
        const size_t n = std::min(cap - 1, g_err.size());
        memcpy(buf, g_err.data(), n);
        buf[n] = '\0';
    }
    return (int)g_err.size();
}

const char* lbks_version(void) { return "lbks 0.2 (sm_103a)"; }

uint64_t lbks_kernel_launches(void) { return g_launches.load(); }

uint32_t lbks_set_wait_limit(uint32_t polls) { return set_gram_tc_wait_limit(polls); }

uint64_t lbks_wait_timeouts(void) { return gram_tc_timeouts(); }

size_t lbks_system_bytes(const lbks_params* p, int nx, int ny, int nz, int n_orb) {
    if (!valid_params(p) || nx < 2 || ny < 2 || nz < 2 || n_orb < 1 || n_orb > kMaxOrbWide) return 0;
    return bytes_of(p, nx, ny, nz, n_orb, 1);
}

size_t lbks_batch_bytes(const lbks_params* p, int nx, int ny, int nz, int n_orb, int n_systems) {
    if (!valid_params(p) || nx < 2 || ny < 2 || nz < 2 || n_orb < 1 || n_orb > kMaxOrbWide || n_systems < 1)
        return 0;
    return bytes_of(p, nx, ny, nz, n_orb, n_systems);
}

int lbks_create_system(const lbks_params* p, int nx, int ny, int nz, double h, int n_orb, lbks_system** out) {
    return create(p, nx, ny, nz, h, n_orb, 1, out);
}

int lbks_create_batch(const lbks_params* p, int nx, int ny, int nz, double h, int n_orb, int n_systems,
                      lbks_system** out) {
    return create(p, nx, ny, nz, h, n_orb, n_systems, out);
}

int lbks_destroy_system(lbks_system* s) {
    if (!s) return fail(LBKS_EINVAL, "system is NULL");
    // the system's own streams; work it queued on caller streams has finished
    // when lbks_scf returned (it synchronises before returning)
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->cap) cudaStreamSynchronize(s->cap);
    free_system(s);
    return LBKS_OK;
}

int lbks_set_geometry(lbks_system* s, int n_atoms, const double* xyz, const double* Z) {
    if (!s) return fail(LBKS_EINVAL, "system is NULL");
    if (s->B != 1) return fail(LBKS_EINVAL, "batched handle: use lbks_batch_set_geometry and lbks_batch_init");
    int rc = check_atoms(s, n_atoms, xyz, Z);
    if (rc != LBKS_OK) return rc;
    s->xyz[0].assign(xyz, xyz + 3 * n_atoms);
    s->Z[0].assign(Z, Z + n_atoms);
    s->has_atoms[0] = 1;
    return initialise(s);
}

int lbks_batch_set_geometry(lbks_system* s, int system, int n_atoms, const double* xyz, const double* Z) {
    if (!s) return fail(LBKS_EINVAL, "system is NULL");
    if (system < 0 || system >= s->B) return fail(LBKS_EINVAL, "system index out of range");
    int rc = check_atoms(s, n_atoms, xyz, Z);
    if (rc != LBKS_OK) return rc;
    s->xyz[system].assign(xyz, xyz + 3 * n_atoms);
    s->Z[system].assign(Z, Z + n_atoms);
    s->has_atoms[system] = 1;
    s->ready = false;
    return LBKS_OK;
}

int lbks_batch_init(lbks_system* s) {
    if (!s) return fail(LBKS_EINVAL, "system is NULL");
    return initialise(s);
}

int lbks_scf(lbks_system* s, void* stream, lbks_result* out) {
    if (!s) return fail(LBKS_EINVAL, "system is NULL");
    if (s->B != 1) return fail(LBKS_EINVAL, "batched handle: use lbks_batch_scf");
    return run_cycles(s, 0, 0, (cudaStream_t)stream, out);
}

int lbks_scf_cycles(lbks_system* s, int n, void* stream, lbks_result* out) {
    if (!s || n < 0) return fail(LBKS_EINVAL, "bad argument");
    return run_cycles(s, 1, n, (cudaStream_t)stream, out);
}

int lbks_batch_scf(lbks_system* s, void* stream, lbks_result* out) {
    if (!s) return fail(LBKS_EINVAL, "system is NULL");
    return run_cycles(s, 0, 0, (cudaStream_t)stream, out);
}

int lbks_batch_energy(const lbks_system* s, int system, lbks_energy_terms* out) {
    if (!s || !out) return fail(LBKS_EINVAL, "null argument");
    if (system < 0 || system >= s->B) return fail(LBKS_EINVAL, "system index out of range");
    if (!s->ready) return fail(LBKS_EINVAL, "geometry has not been set");
    *out = s->terms[system];
    return LBKS_OK;
}

int lbks_energy(const lbks_system* s, lbks_energy_terms* out) { return lbks_batch_energy(s, 0, out); }

int lbks_batch_forces(lbks_system* s, int system, double* forces, size_t cap) {
    if (!s || !forces) return fail(LBKS_EINVAL, "null argument");
    if (system < 0 || system >= s->B) return fail(LBKS_EINVAL, "system index out of range");
    if (!s->ready) return fail(LBKS_EINVAL, "geometry has not been set");
    const int na = (int)s->Z[system].size();
    if (cap < (size_t)3 * na) return fail(LBKS_EINVAL, "capacity %zu < %d", cap, 3 * na);
    int max_atoms = 1;
    for (int i = 0; i < s->B; ++i) max_atoms = std::max(max_atoms, (int)s->Z[i].size());
    Grid g = s->g;
    g.active = nullptr;  // every system, converged or not
    cudaError_t e = launch_forces(g, s->h, s->counts, s->atoms, s->a, s->rho, s->forces, max_atoms, s->sc, s->B, s->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(forces, s->forces + (size_t)system * 3 * kMaxAtoms, sizeof(double) * 3 * na,
                            cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_fail(e, "lbks_forces");
    // nucleus-nucleus term (bare Coulomb, as E_nn)
    const std::vector<double>& xyz = s->xyz[system];
    const std::vector<double>& Z = s->Z[system];
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < na; ++b) {
            if (b == a) continue;
            const double d[3] = {xyz[3 * a] - xyz[3 * b], xyz[3 * a + 1] - xyz[3 * b + 1], xyz[3 * a + 2] - xyz[3 * b + 2]};
            const double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int k = 0; k < 3; ++k) forces[3 * a + k] += Z[a] * Z[b] * d[k] / (r * r * r);
        }
    return LBKS_OK;
}

int lbks_forces(lbks_system* s, double* forces, size_t cap) { return lbks_batch_forces(s, 0, forces, cap); }

int lbks_move_atoms(lbks_system* s, const double* xyz) {
    if (!s || !xyz) return fail(LBKS_EINVAL, "null argument");
    if (s->B != 1) return fail(LBKS_EINVAL, "batched handle: move atoms with lbks_batch_set_geometry");
    if (!s->ready) return fail(LBKS_EINVAL, "geometry has not been set");
    const int na = (int)s->Z[0].size();
    int rc = check_atoms(s, na, xyz, s->Z[0].data());
    if (rc != LBKS_OK) return rc;
    s->xyz[0].assign(xyz, xyz + 3 * na);
    std::vector<double> atoms;
    std::vector<int> counts;
    pack_atoms(s, atoms, counts);
    cudaStream_t st = s->st;
    host_active(s)[0] = 1;
    cudaError_t e = cudaMemcpyAsync(s->atoms, atoms.data(), sizeof(double) * atoms.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_vext(s->g, s->h, s->counts, s->atoms, s->a, s->vext, 1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host atom array is a temporary
    if (e != cudaSuccess) return cuda_fail(e, "lbks_move_atoms");
    rc = upload_active(s, st);
    if (rc != LBKS_OK) return rc;
    return evaluate(s, st, 1);  // potential of the current orbitals at the new nuclei, unmixed
}

int lbks_md(lbks_system* s, int n_steps, double dt, const double* masses, double* velocities, void* stream,
            double* energies, double* xyz_traj) {
    if (!s || n_steps < 0 || !(dt > 0.0) || !masses || !velocities) return fail(LBKS_EINVAL, "bad argument");
    if (s->B != 1) return fail(LBKS_EINVAL, "batched handle: one geometry per handle");
    if (!s->ready) return fail(LBKS_EINVAL, "geometry has not been set");
    const int na = (int)s->Z[0].size();
    for (int a = 0; a < na; ++a)
        if (!(masses[a] > 0.0)) return fail(LBKS_EINVAL, "mass %d must be positive", a);
    std::vector<double> R = s->xyz[0], F(3 * na), Fn(3 * na);
    lbks_result res{};
    auto record = [&](int k) {
        double ek = 0.0;
        for (int a = 0; a < na; ++a)
            for (int c = 0; c < 3; ++c) ek += 0.5 * masses[a] * velocities[3 * a + c] * velocities[3 * a + c];
        if (energies) {
            energies[2 * k] = res.E_total;
            energies[2 * k + 1] = ek;
        }
        if (xyz_traj) std::copy(R.begin(), R.end(), xyz_traj + (size_t)k * 3 * na);
    };
    int rc = lbks_scf(s, stream, &res);
    if (rc != LBKS_OK) return rc;
    rc = lbks_forces(s, F.data(), F.size());
    if (rc != LBKS_OK) return rc;
    record(0);
    for (int k = 1; k <= n_steps; ++k) {  // velocity Verlet
        for (int a = 0; a < na; ++a)
            for (int c = 0; c < 3; ++c) {
                const int i = 3 * a + c;
                R[i] += dt * velocities[i] + 0.5 * dt * dt * F[i] / masses[a];
            }
        rc = lbks_move_atoms(s, R.data());
        if (rc == LBKS_OK) rc = lbks_scf(s, stream, &res);
        if (rc == LBKS_OK) rc = lbks_forces(s, Fn.data(), Fn.size());
        if (rc != LBKS_OK) return rc;
        for (int a = 0; a < na; ++a)
            for (int c = 0; c < 3; ++c) {
                const int i = 3 * a + c;
                velocities[i] += 0.5 * dt * (F[i] + Fn[i]) / masses[a];
            }
        F = Fn;
        record(k);
    }
    return LBKS_OK;
}

int lbks_relax_geometry(lbks_system* s, int max_steps, double fmax, double step, const int* fixed, void* stream,
                        lbks_result* out, double* xyz_out, int* steps_out) {
    if (!s || max_steps < 0 || !(fmax > 0.0) || !(step > 0.0)) return fail(LBKS_EINVAL, "bad argument");
    if (s->B != 1) return fail(LBKS_EINVAL, "batched handle: one geometry per handle");
    if (!s->ready) return fail(LBKS_EINVAL, "geometry has not been set");
    const int na = (int)s->Z[0].size();
    lbks_result res;
    int total_cycles = 0, total_steps = 0, total_iters = 0;
    double total_wall = 0.0, total_poisson = 0.0;
    auto solve = [&](lbks_result* r) {
        const int code = lbks_scf(s, stream, r);
        total_cycles += r->cycles;
        total_steps += r->steps;
        total_iters += r->poisson_iters;
        total_wall += r->wall_s;
        total_poisson += r->poisson_s;
        return code;
    };
    int rc = solve(&res);
    if (rc != LBKS_OK && rc != LBKS_ENOTCONV) return rc;
    std::vector<double> R = s->xyz[0], F(3 * na), trial(3 * na);
    // forces with the fixed nuclei's rows zeroed (they neither move nor count for convergence)
    auto free_forces = [&](std::vector<double>& f) {
        const int code = lbks_forces(s, f.data(), f.size());
        if (code == LBKS_OK && fixed)
            for (int a = 0; a < na; ++a)
                if (fixed[a]) f[3 * a] = f[3 * a + 1] = f[3 * a + 2] = 0.0;
        return code;
    };
    rc = free_forces(F);
    if (rc != LBKS_OK) return rc;
    double E = res.E_total, alpha = 1.0;
    int steps = 0;
    bool at_R = true, done = false;
    // inverse Hessian estimate (BFGS), starting from step * identity
    const int n3 = 3 * na;
    std::vector<double> Hi((size_t)n3 * n3, 0.0), p(n3), Fnew(n3), hy(n3);
    for (int k = 0; k < n3; ++k) Hi[(size_t)k * n3 + k] = step;
    auto fmax_of = [&](const std::vector<double>& f) {
        double m = 0.0;
        for (int a = 0; a < na; ++a)
            m = std::max(m, std::sqrt(f[3 * a] * f[3 * a] + f[3 * a + 1] * f[3 * a + 1] + f[3 * a + 2] * f[3 * a + 2]));
        return m;
    };
    while (steps < max_steps) {
        if (fmax_of(F) < fmax) {
            done = true;
            break;
        }
        ++steps;
        // quasi-Newton direction p = Hi F; no nucleus moved more than 0.2 bohr
        double pf = 0.0;
        for (int i = 0; i < n3; ++i) {
            double t = 0.0;
            for (int k = 0; k < n3; ++k) t += Hi[(size_t)i * n3 + k] * F[k];
            p[i] = t;
            pf += t * F[i];
        }
        if (!(pf > 0.0)) {  // not a descent direction: start the estimate again
            for (int i = 0; i < n3; ++i)
                for (int k = 0; k < n3; ++k) Hi[(size_t)i * n3 + k] = i == k ? step : 0.0;
            for (int i = 0; i < n3; ++i) p[i] = step * F[i];
        }
        double pm = 0.0;
        for (int a = 0; a < na; ++a)
            pm = std::max(pm, std::sqrt(p[3 * a] * p[3 * a] + p[3 * a + 1] * p[3 * a + 1] + p[3 * a + 2] * p[3 * a + 2]));
        const double scale = alpha * pm > 0.2 ? 0.2 / pm : alpha;
        for (int k = 0; k < n3; ++k) trial[k] = R[k] + scale * p[k];
        rc = lbks_move_atoms(s, trial.data());
        if (rc != LBKS_OK) return rc;
        lbks_result tr;
        rc = solve(&tr);
        if (rc != LBKS_OK && rc != LBKS_ENOTCONV) return rc;
        if (tr.E_total < E) {  // accept; update the inverse Hessian with s = dR, y = -dF
            rc = free_forces(Fnew);
            if (rc != LBKS_OK) return rc;
            double sy = 0.0;
            for (int k = 0; k < n3; ++k) {
                trial[k] -= R[k];           // s
                p[k] = F[k] - Fnew[k];      // y (gradient change)
                sy += trial[k] * p[k];
            }
            if (sy > 1e-12) {  // curvature condition: H+ = (I - r s y^T) H (I - r y s^T) + r s s^T, r = 1 / s.y
                double yhy = 0.0;
                for (int i = 0; i < n3; ++i) {
                    double t = 0.0;
                    for (int k = 0; k < n3; ++k) t += Hi[(size_t)i * n3 + k] * p[k];
                    hy[i] = t;
                    yhy += p[i] * t;
                }
                const double r = 1.0 / sy;
                for (int i = 0; i < n3; ++i)
                    for (int k = 0; k < n3; ++k)
                        Hi[(size_t)i * n3 + k] += (1.0 + r * yhy) * r * trial[i] * trial[k] -
                                                  r * (hy[i] * trial[k] + trial[i] * hy[k]);
            }
            for (int k = 0; k < n3; ++k) R[k] += trial[k];
            F = Fnew;
            E = tr.E_total;
            res = tr;
            alpha = std::min(1.0, alpha * 2.0);
            at_R = true;
        } else {  // undo, and halve the step along the same direction next time
            alpha *= 0.5;
            at_R = false;
        }
    }
    if (!at_R) {  // leave the handle at the returned geometry, relaxed there
        rc = lbks_move_atoms(s, R.data());
        if (rc == LBKS_OK) rc = solve(&res);
        if (rc != LBKS_OK && rc != LBKS_ENOTCONV) return rc;
        rc = free_forces(F);
        if (rc != LBKS_OK) return rc;
        if (fmax_of(F) < fmax) done = true;
    }
    res.cycles = total_cycles;
    res.steps = total_steps;
    res.poisson_iters = total_iters;
    res.wall_s = total_wall;
    res.poisson_s = total_poisson;
    if (out) *out = res;
    if (xyz_out) std::copy(R.begin(), R.end(), xyz_out);
    if (steps_out) *steps_out = steps;
    if (!done) return fail(LBKS_ENOTCONV, "largest force %.3e Ha/bohr after %d steps", fmax_of(F), steps);
    return LBKS_OK;
}

int lbks_batch_get_density(const lbks_system* s, int system, double* host, size_t cap) {
    if (!s || !host) return fail(LBKS_EINVAL, "null argument");
    return copy_field(s, system, s->rho, host, cap, "lbks_get_density");
}

int lbks_get_density(const lbks_system* s, double* host, size_t cap) { return lbks_batch_get_density(s, 0, host, cap); }

int lbks_get_orbitals(const lbks_system* s, double* host, size_t cap) {
    if (!s || !host) return fail(LBKS_EINVAL, "null argument");
    const size_t n = s->N * s->n_orb;
    if (cap < n) return fail(LBKS_EINVAL, "capacity %zu < %zu", cap, n);
    if (s->ops->psi_elem == sizeof(double)) {
        cudaError_t e = cudaMemcpyAsync(host, s->psi, sizeof(double) * n, cudaMemcpyDeviceToHost, s->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
        return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_get_orbitals");
    }
    std::vector<float> tmp(n);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), s->psi, sizeof(float) * n, cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return cuda_fail(e, "lbks_get_orbitals");
    for (size_t i = 0; i < n; ++i) host[i] = tmp[i];
    return LBKS_OK;
}

int lbks_get_potential(const lbks_system* s, int which, double* host, size_t cap) {
    if (!s || !host) return fail(LBKS_EINVAL, "null argument");
    const double* src = which == 0 ? s->vin : which == 1 ? s->vout : which == 2 ? s->vh : which == 3 ? s->vext : nullptr;
    if (!src) return fail(LBKS_EINVAL, "which must be 0..3");
    return copy_field(s, 0, src, host, cap, "lbks_get_potential");
}

// ------------------------------------------------------------- step-level calls
int lbks_relax_step(int precision, int nx, int ny, int nz, int n_orb, double h, double omega, double theta,
                    double dt, const void* f_in, const void* u_in, const double* V, const double* sigma_in,
                    void* f_out, void* psi_out, double* S_out, double* lambda_out, double* sigma_out,
                    void* stream) {
    const PrecisionOps* ops = ops_for(precision);
    if (!ops) return fail(LBKS_EINVAL, "unknown precision %d", precision);
    if (nx < 2 || ny < 2 || nz < 2 || (size_t)nx * ny * nz >= (1ull << 31))
        return fail(LBKS_EINVAL, "bad grid %d x %d x %d", nx, ny, nz);
    if (n_orb < 1 || n_orb > kMaxOrbWide) return fail(LBKS_EINVAL, "n_orb must be in [1, %d]", kMaxOrbWide);
    if (!f_in || !V || !sigma_in || !f_out || !psi_out || !S_out || !lambda_out || !sigma_out)
        return fail(LBKS_EINVAL, "null device pointer");
    if (f_in == f_out) return fail(LBKS_EINVAL, "f_in and f_out must not alias");
    if (!(h > 0.0) || !(omega > 0.0 && omega < 2.0)) return fail(LBKS_EINVAL, "bad h or omega");
    Workspace* w = nullptr;
    int rc = workspace(stream, 0, &w);
    if (rc != LBKS_OK) return rc;
    RelaxIO io{f_in, u_in, V, sigma_in, f_out, psi_out, S_out, lambda_out, sigma_out};
    cudaError_t e = ops->relax(n_orb, make_grid(nx, ny, nz), make_coef(omega, theta, dt, h), io, w->sc, 1,
                               variant_for(precision, n_orb, omega, nx, ny, nz), (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_relax_step");
}

int lbks_relax_step_psi(int precision, int nx, int ny, int nz, int n_orb, double h, double theta, double dt,
                        const void* psi_in, const double* lambda_in, const double* Vc, const double* sigma_in,
                        void* psi_out, double* S_out, double* lambda_out, double* sigma_out, void* stream) {
    if (precision != LBKS_FP64 && precision != LBKS_FP32)
        return fail(LBKS_EINVAL, "orbital storage needs LBKS_FP64 or LBKS_FP32");
    const PrecisionOps* ops = ops_for(precision);
    if (nx < 2 || ny < 2 || nz < 2 || (size_t)nx * ny * nz >= (1ull << 31))
        return fail(LBKS_EINVAL, "bad grid %d x %d x %d", nx, ny, nz);
    if (n_orb < 1 || n_orb > kMaxOrbWide) return fail(LBKS_EINVAL, "n_orb must be in [1, %d]", kMaxOrbWide);
    if (!psi_in || !Vc || !sigma_in || !psi_out || !S_out || !lambda_out || !sigma_out)
        return fail(LBKS_EINVAL, "null device pointer");
    if (psi_in == psi_out) return fail(LBKS_EINVAL, "psi_in and psi_out must not alias");
    if (!(h > 0.0) || !(theta > 0.0)) return fail(LBKS_EINVAL, "bad h or theta");
    const size_t N = (size_t)nx * ny * nz;
    // forced kernel, else the TMA kernel where it applies, else the tiled one
    const int mode = g_variant_mode.load();
    const bool tma_ok = psi_tma_applies(nx, psi_in, Vc, ops->psi_elem);
    int kernel = mode > 0 ? mode - 1 : (tma_ok ? kPsiKernelTma : kPsiKernelTiled);
    if ((kernel == kPsiKernelTma && !tma_ok) || (kernel == kPsiKernelZ && n_orb > kMaxOrb)) kernel = kPsiKernelTiled;
    const int shape = g_psi_shape.load();
    if (kernel == kPsiKernelTiled && n_orb <= kMaxOrb && shape > 0) kernel |= shape << kPsiShapeShift;
    // the W field goes through workspace scratch unless the kernel forms it
    const bool wide = n_orb > kMaxOrb && lambda_in && kernel != kPsiKernelTma;
    Workspace* w = nullptr;
    int rc = workspace(stream, wide ? (ops->psi_elem * N * (n_orb - 1) + 7) / 8 : 0, &w);
    if (rc != LBKS_OK) return rc;
    const Grid g = make_grid(nx, ny, nz);
    cudaError_t e = cudaSuccess;
    if (wide) e = ops->w_field(n_orb, make_grid((int)N, 1, 1), 1.0, psi_in, lambda_in, w->pvec, 1, (cudaStream_t)stream);
    RelaxIO io{psi_in, wide ? w->pvec : nullptr, Vc, sigma_in, psi_out, psi_out, S_out, lambda_out, sigma_out,
               wide ? nullptr : lambda_in};
    if (e == cudaSuccess)
        e = ops->relax_psi(n_orb, g, make_coef(1.0, theta, dt, h), io, w->sc, 1, kernel, (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_relax_step_psi");
}

int lbks_overlap(int precision, size_t n_sites, int n_orb, double h, const void* psi, double* S, int tensor_cores,
                 void* stream) {
    const PrecisionOps* ops = ops_for(precision);
    if (!ops) return fail(LBKS_EINVAL, "unknown precision %d", precision);
    if (n_orb < 1 || n_orb > kMaxOrbWide || !psi || !S || !(h > 0.0)) return fail(LBKS_EINVAL, "bad argument");
    if (n_sites == 0 || n_sites >= (1ull << 31)) return fail(LBKS_EINVAL, "n_sites must be in [1, 2^31)");
    Workspace* w = nullptr;
    int rc = workspace(stream, 0, &w);
    if (rc != LBKS_OK) return rc;
    const Grid g = make_grid((int)n_sites, 1, 1);
    cudaError_t e = tensor_cores && precision != LBKS_FP64
                        ? launch_gram_tc(n_orb, g, h, (const float*)psi, S, nullptr, nullptr, w->sc, 1,
                                         (cudaStream_t)stream)
                        : ops->gram(n_orb, g, h, psi, S, w->sc, 1, (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_overlap");
}

int lbks_energy_matrix(int precision, int nx, int ny, int nz, int n_orb, double h, double theta, const void* psi,
                       const double* V, double* out, void* stream) {
    const PrecisionOps* ops = ops_for(precision);
    if (!ops) return fail(LBKS_EINVAL, "unknown precision %d", precision);
    if (nx < 2 || ny < 2 || nz < 2 || (size_t)nx * ny * nz >= (1ull << 31))
        return fail(LBKS_EINVAL, "bad grid %d x %d x %d", nx, ny, nz);
    if (n_orb < 1 || n_orb > kMaxOrbWide) return fail(LBKS_EINVAL, "n_orb must be in [1, %d]", kMaxOrbWide);
    if (!psi || !V || !out) return fail(LBKS_EINVAL, "null device pointer");
    if (!(h > 0.0) || !(theta > 0.0)) return fail(LBKS_EINVAL, "bad h or theta");
    Workspace* w = nullptr;
    int rc = workspace(stream, 0, &w);
    if (rc != LBKS_OK) return rc;
    cudaError_t e = ops->energy_matrix(n_orb, make_grid(nx, ny, nz), make_coef(1.0, theta, theta * h * h, h), psi, V,
                                       out, w->sc, 1, (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_energy_matrix");
}

int lbks_w_field(int precision, size_t n_sites, int n_orb, double omega, const void* psi, const double* lambda,
                 void* u_out, void* stream) {
    const PrecisionOps* ops = ops_for(precision);
    if (!ops) return fail(LBKS_EINVAL, "unknown precision %d", precision);
    if (n_orb < 1 || n_orb > kMaxOrbWide || !psi || !lambda || (n_orb > 1 && !u_out))
        return fail(LBKS_EINVAL, "bad argument");
    if (n_sites == 0) return LBKS_OK;
    if (n_sites >= (1ull << 31)) return fail(LBKS_EINVAL, "n_sites must be below 2^31");
    cudaError_t e = ops->w_field(n_orb, make_grid((int)n_sites, 1, 1), omega, psi, lambda, u_out, 1,
                                 (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_w_field");
}

int lbks_cholesky_inverse(int n, const double* S, double* Linv, int* status, void* stream) {
    if (n < 1 || n > kMaxOrbWide || !S || !Linv || !status) return fail(LBKS_EINVAL, "bad argument");
    cudaError_t e = launch_cholesky(n, S, Linv, status, nullptr, 1, (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_cholesky_inverse");
}

int lbks_orth_apply(int precision, size_t n_sites, int n_orb, const double* Linv, void* f, void* psi,
                    void* stream) {
    const PrecisionOps* ops = ops_for(precision);
    if (!ops) return fail(LBKS_EINVAL, "unknown precision %d", precision);
    if (n_orb < 1 || n_orb > kMaxOrbWide || !Linv) return fail(LBKS_EINVAL, "bad argument");
    if (n_sites == 0 || (!f && !psi)) return LBKS_OK;
    if (n_sites >= (1ull << 31)) return fail(LBKS_EINVAL, "n_sites must be below 2^31");
    cudaError_t e = ops->orth_apply(n_orb, make_grid((int)n_sites, 1, 1), Linv, f, psi, 1, (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_orth_apply");
}

int lbks_hartree(int nx, int ny, int nz, double h, const double* rho, double* v, double rtol, int max_iter,
                 int* iters_out, double* relres_out, void* stream) {
    if (nx < 2 || ny < 2 || nz < 2 || (size_t)nx * ny * nz >= (1ull << 31) || !(h > 0.0) || !rho || !v ||
        !(rtol > 0.0) || max_iter < 0)
        return fail(LBKS_EINVAL, "bad argument");
    const Grid g = make_grid(nx, ny, nz);
    Workspace* w = nullptr;
    int rc = workspace(stream, 6 * (size_t)g.N + mg_coarse_doubles(nx, ny, nz), &w);
    if (rc != LBKS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const MGHierarchy H = make_hierarchy(g, w->pvec + 6 * (size_t)g.N, 1);
    const PoissonBufs pb = poisson_bufs(w->pvec, g.N, w->cg, w->mp, H);
    cudaError_t e = launch_multipoles_from_rho(g, h, rho, w->mp, w->sc, 1, st);
    if (e == cudaSuccess) e = launch_poisson_start(g, h, rho, v, rtol, pb, w->sc, 1, st);
    if (e != cudaSuccess) return cuda_fail(e, "lbks_hartree");
    CGState hcg;
    int done = 0;
    while (true) {
        e = cudaMemcpyAsync(&hcg, w->cg, sizeof hcg, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "lbks_hartree readback");
        if (hcg.done || done >= max_iter) break;
        const int chunk = std::min(2, max_iter - done);
        e = launch_poisson_iterate(g, v, rtol, chunk, pb, H, w->sc, 1, st);
        if (e != cudaSuccess) return cuda_fail(e, "lbks_hartree iterate");
        done += chunk;
    }
    if (iters_out) *iters_out = hcg.iters;
    if (relres_out) *relres_out = hcg.relres;
    if (!hcg.done) return fail(LBKS_ENOTCONV, "Hartree PCG: relative residual %.3e after %d iterations", hcg.relres,
                               hcg.iters);
    return LBKS_OK;
}

int lbks_lda(size_t n_sites, const double* rho, double* eps, double* v, void* stream) {
    if (!rho || !eps || !v) return fail(LBKS_EINVAL, "null argument");
    if (n_sites == 0) return LBKS_OK;
    cudaError_t e = launch_lda(n_sites, rho, eps, v, (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_lda");
}

}  // extern "C"

// --------------------------------------------------------- concurrent dynamics
namespace {
std::atomic<int> g_cd_kernel{-1};
}  // namespace

int lbks::cd_kernel_mode() { return g_cd_kernel.load(); }

namespace {

CdCoef make_cd_coef(double theta, double h) {
    const Coef c = make_coef(1.0, theta, theta * h * h, h);
    CdCoef d;
    d.dt = c.dt;
    const double w[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    for (int k = 0; k < 3; ++k) {
        d.xi[k] = c.xi[k];
        d.chi[k] = c.chi[k];
        d.wq[k] = w[k] * (k - 1.0) * 4.5;  // w_p q_p, q_p = (v^2 - 3 c_s^2) / (2 c_s^4)
    }
    return d;
}

cudaError_t cd_step_launch(int precision, int NO, const Grid& g, const CdCoef& c, const CdIO& io, const Scratch& sc,
                           int B, cudaStream_t st) {
    return precision == LBKS_FP64 ? launch_cd_step<double>(NO, g, c, io, sc, B, st)
                                  : launch_cd_step<float>(NO, g, c, io, sc, B, st);
}

cudaError_t cd_overlap_launch(int precision, int NO, const Grid& g, const void* phi, double h, double* S, double* lam,
                              const Scratch& sc, int B, cudaStream_t st) {
    return precision == LBKS_FP64 ? launch_cd_overlap<double>(NO, g, phi, h, S, lam, sc, B, st)
                                  : launch_cd_overlap<float>(NO, g, phi, h, S, lam, sc, B, st);
}

// Device small arrays of the dynamics: Lambda (two buffers), S, the U
// coefficients (step and start) and the energy matrix of 2 n_orb rows.
size_t cd_small_doubles(int no) { return 3 * (size_t)no * no * 2 + 2 * (size_t)no + emat_stride(2 * no); }
double* cd_lam(lbks_system* s, int k) { return s->cd_small + (size_t)k * s->n_orb * s->n_orb * 2; }
double* cd_S(lbks_system* s) { return cd_lam(s, 2); }
double* cd_ucoef(lbks_system* s, int half) { return cd_S(s) + (size_t)s->n_orb * s->n_orb * 2 + half * s->n_orb; }
double* cd_emat(lbks_system* s) { return cd_ucoef(s, 0) + 2 * s->n_orb; }

// Density of the current level (its 2 n_orb planes as real rows), Hartree,
// potential (unmixed, into V_in and V_out), energies at the current nuclei
// and the Hellmann-Feynman forces; E_total and the electron count out.
int cd_rebuild(lbks_system* s, cudaStream_t st, double* e_total, double* n_el) {
    const int no2 = 2 * s->n_orb;
    const void* phi = s->cd_lev[s->cd_cur];
    cudaError_t e = s->ops->density(no2, s->g, s->h, phi, s->rho, s->rho, s->mp, s->cd_sc, 1, st);
    if (e != cudaSuccess) return cuda_fail(e, "density (dynamics)");
    int rc = hartree_solve(s, st);
    if (rc != LBKS_OK) return rc;
    e = launch_potential(s->g, s->h, s->rho, s->vext, s->vh, s->vout, s->vin, 1, 1.0, s->e4, s->sc, 1, st);
    if (e != cudaSuccess) return cuda_fail(e, "potential (dynamics)");
    e = s->ops->energy_matrix(no2, s->g, s->c, phi, s->vout, cd_emat(s), s->cd_sc, 1, st);
    if (e != cudaSuccess) return cuda_fail(e, "energy matrix (dynamics)");
    std::vector<double> kin(no2);
    e = cudaMemcpyAsync(host_e4(s, 0), s->e4, sizeof(double) * kE4Stride, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "energy readback (dynamics)");
    const double* h4 = host_e4(s, 0);
    const double e_ext = h4[0], e_h = 0.5 * h4[1], e_xc = h4[2];
    *n_el = h4[3];
    e = cudaMemcpy(kin.data(), cd_emat(s) + (size_t)no2 * no2, sizeof(double) * no2, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "kinetic readback (dynamics)");
    double ts = 0.0;
    for (double k : kin) ts += k;
    const std::vector<double>& xyz = s->xyz[0];
    const std::vector<double>& Z = s->Z[0];
    double enn = 0.0;
    for (size_t a = 0; a < Z.size(); ++a)
        for (size_t b = 0; b < a; ++b) {
            const double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1],
                         dz = xyz[3 * a + 2] - xyz[3 * b + 2];
            enn += Z[a] * Z[b] / std::sqrt(dx * dx + dy * dy + dz * dz);
        }
    *e_total = 2.0 * ts + e_ext + e_h + e_xc + enn;
    s->cd_F.assign(3 * Z.size(), 0.0);
    return lbks_forces(s, s->cd_F.data(), s->cd_F.size());
}

// One step: next = prev + 2i (tau/dt) D(cur) + u K_q cur, then the levels rotate.
int cd_advance(lbks_system* s, cudaStream_t st) {
    const int nxt = 3 - s->cd_prev - s->cd_cur;
    const bool w = s->n_orb > 1;
    CdIO io{};
    io.prev = s->cd_lev[s->cd_prev];
    io.cur = s->cd_lev[s->cd_cur];
    io.out = s->cd_lev[nxt];
    io.V = s->vin;
    io.lam = w ? cd_lam(s, s->cd_lam) : nullptr;
    io.ucoef = s->cd_u ? cd_ucoef(s, 0) : nullptr;
    io.S_out = w ? cd_S(s) : nullptr;
    io.lam_out = w ? cd_lam(s, 1 - s->cd_lam) : nullptr;
    io.alpha = 1.0;
    io.c_re = 0.0;
    io.c_im = 2.0 * s->cd_tau / (s->prm.theta * s->h * s->h);
    io.h = s->h;
    cudaError_t e = cd_step_launch(s->prm.precision == LBKS_FP64 ? LBKS_FP64 : LBKS_FP32, s->n_orb, s->g,
                                   make_cd_coef(s->prm.theta, s->h), io, s->sc, 1, st);
    if (e != cudaSuccess) return cuda_fail(e, "concurrent-dynamics step");
    s->cd_prev = s->cd_cur;
    s->cd_cur = nxt;
    if (w) s->cd_lam = 1 - s->cd_lam;
    ++s->cd_steps;
    s->cd_time += s->cd_tau;
    return LBKS_OK;
}

}  // namespace

extern "C" {

int lbks_set_cd_kernel(int mode) {
    if (mode < -1 || mode > 1) {
        fail(LBKS_EINVAL, "mode must be -1, 0 or 1");
        return -2;
    }
    return g_cd_kernel.exchange(mode);
}

int lbks_cd_start(lbks_system* s, const lbks_cd_params* p, const double* E_target, void* stream, double* energy) {
    if (!s || !p) return fail(LBKS_EINVAL, "null argument");
    if (s->B != 1) return fail(LBKS_EINVAL, "batched handle: one system per dynamics");
    if (!s->ready) return fail(LBKS_EINVAL, "geometry has not been set");
    if (s->n_orb > kMaxOrb) return fail(LBKS_EINVAL, "concurrent dynamics takes up to %d orbitals", kMaxOrb);
    if (s->prm.omega != 1.0) return fail(LBKS_EINVAL, "concurrent dynamics is built on the omega = 1 step");
    const double dt = s->prm.theta * s->h * s->h;
    const double tau = p->tau > 0.0 ? p->tau : 0.5 * dt;
    if (!(tau <= dt) || !std::isfinite(p->kappa)) return fail(LBKS_EINVAL, "tau must be in (0, theta h^2]");
    if (p->n_pot < 0) return fail(LBKS_EINVAL, "n_pot must be >= 0");
    if (p->kappa != 0.0 && !E_target) return fail(LBKS_EINVAL, "kappa != 0 needs E_target");
    cudaStream_t st = s->st;
    (void)stream;
    const int no = s->n_orb;
    const size_t N = s->N, ep = s->ops->psi_elem, level = ep * N * 2 * no;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        if (!s->cd_lev[k]) e = cudaMalloc(&s->cd_lev[k], level);
    if (e == cudaSuccess && !s->cd_small) e = cudaMalloc((void**)&s->cd_small, sizeof(double) * cd_small_doubles(no));
    if (e == cudaSuccess && !s->cd_sc.partial) {
        s->cd_sc.max_blocks = num_sms() * 8;
        s->cd_sc.max_vals = scratch_vals(2 * no);
        s->cd_sc.systems = 1;
        e = cudaMalloc(&s->cd_sc.partial, sizeof(double) * (size_t)s->cd_sc.max_blocks * s->cd_sc.max_vals);
        if (e == cudaSuccess) e = cudaMalloc(&s->cd_sc.counter, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemsetAsync(s->cd_sc.counter, 0, sizeof(unsigned), st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "concurrent-dynamics allocation");
    s->cd_tau = tau;
    s->cd_npot = p->n_pot > 0 ? p->n_pot : 10;
    s->cd_u = p->kappa != 0.0;
    std::vector<double> uc(2 * no, 0.0);
    for (int j = 0; j < no && s->cd_u; ++j) {
        uc[j] = 2.0 * tau * p->kappa * E_target[j];
        uc[no + j] = tau * p->kappa * E_target[j];
    }
    e = cudaMemcpyAsync(cd_ucoef(s, 0), uc.data(), sizeof(double) * 2 * no, cudaMemcpyHostToDevice, st);
    // level 0: the handle's orthonormal orbitals, imaginary parts zero
    void* L0 = s->cd_lev[0];
    for (int j = 0; j < no && e == cudaSuccess; ++j) {
        char* dst = static_cast<char*>(L0) + (size_t)2 * j * N * ep;
        e = cudaMemcpyAsync(dst, static_cast<const char*>(s->psi) + (size_t)j * N * ep, N * ep,
                            cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(dst + N * ep, 0, N * ep, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "concurrent-dynamics start");
    s->cd_prev = 1;
    s->cd_cur = 0;
    host_active(s)[0] = 1;
    int rc = upload_active(s, st);
    if (rc != LBKS_OK) return rc;
    double e_tot = 0.0, n_el = 0.0;
    rc = cd_rebuild(s, st, &e_tot, &n_el);
    if (rc != LBKS_OK) return rc;
    // second level (Taylor, second order): phi1 = phi0 + i s D(phi0) - s^2 D0(D0(phi0)) / 2 + tau kappa E K_q phi0
    const int prec = s->prm.precision == LBKS_FP64 ? LBKS_FP64 : LBKS_FP32;
    const CdCoef cc = make_cd_coef(s->prm.theta, s->h);
    const double sr = tau / dt;
    const bool w = no > 1;
    if (w) e = cd_overlap_launch(prec, no, s->g, L0, s->h, cd_S(s), cd_lam(s, 0), s->sc, 1, st);
    CdIO io{};
    io.V = s->vin;
    io.h = s->h;
    // X = D0(phi0) into level 2, Y = D0(X) into level 1
    io.cur = L0;
    io.out = s->cd_lev[2];
    io.c_re = 1.0;
    if (e == cudaSuccess) e = cd_step_launch(prec, no, s->g, cc, io, s->sc, 1, st);
    io.cur = s->cd_lev[2];
    io.out = s->cd_lev[1];
    if (e == cudaSuccess) e = cd_step_launch(prec, no, s->g, cc, io, s->sc, 1, st);
    // phi1 = phi0 + i s D(phi0) - s^2 Y / 2 + (u/2) K_q phi0 into level 2, with its overlap
    io.prev = L0;
    io.alpha = 1.0;
    io.extra = s->cd_lev[1];
    io.beta = -0.5 * sr * sr;
    io.cur = L0;
    io.out = s->cd_lev[2];
    io.c_re = 0.0;
    io.c_im = sr;
    io.lam = w ? cd_lam(s, 0) : nullptr;
    io.ucoef = s->cd_u ? cd_ucoef(s, 1) : nullptr;
    io.S_out = w ? cd_S(s) : nullptr;
    io.lam_out = w ? cd_lam(s, 1) : nullptr;
    if (e == cudaSuccess) e = cd_step_launch(prec, no, s->g, cc, io, s->sc, 1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "concurrent-dynamics start");
    s->cd_prev = 0;
    s->cd_cur = 2;
    s->cd_lam = 1;
    s->cd_steps = 1;
    s->cd_time = tau;
    s->cd_ready = true;
    if (energy) {
        energy[0] = e_tot;
        energy[1] = n_el;
    }
    return LBKS_OK;
}

int lbks_cd_run(lbks_system* s, int n_blocks, const double* masses, double* velocities, void* stream,
                double* energies, double* xyz_traj) {
    if (!s || n_blocks < 0) return fail(LBKS_EINVAL, "bad argument");
    if (!s->cd_ready) return fail(LBKS_EINVAL, "lbks_cd_start has not run on this handle");
    const int na = (int)s->Z[0].size();
    if (masses) {
        if (!velocities) return fail(LBKS_EINVAL, "moving nuclei need velocities");
        for (int a = 0; a < na; ++a)
            if (!(masses[a] > 0.0)) return fail(LBKS_EINVAL, "mass %d must be positive", a);
    }
    (void)stream;
    cudaStream_t st = s->st;
    std::vector<double> R = s->xyz[0];
    auto kinetic = [&]() {
        double ek = 0.0;
        for (int a = 0; a < na && masses; ++a)
            for (int c = 0; c < 3; ++c) ek += 0.5 * masses[a] * velocities[3 * a + c] * velocities[3 * a + c];
        return ek;
    };
    for (int b = 0; b < n_blocks; ++b) {
        for (int k = 0; k < s->cd_npot; ++k) {
            int rc = cd_advance(s, st);
            if (rc != LBKS_OK) return rc;
        }
        const double tb = s->cd_npot * s->cd_tau;
        const std::vector<double> F = s->cd_F;
        if (masses) {  // velocity Verlet, first half: positions
            for (int a = 0; a < na; ++a)
                for (int c = 0; c < 3; ++c) {
                    const int i = 3 * a + c;
                    R[i] += tb * velocities[i] + 0.5 * tb * tb * F[i] / masses[a];
                }
            int rc = check_atoms(s, na, R.data(), s->Z[0].data());
            if (rc != LBKS_OK) return rc;
            s->xyz[0] = R;
            std::vector<double> atoms;
            std::vector<int> counts;
            pack_atoms(s, atoms, counts);
            cudaError_t e =
                cudaMemcpyAsync(s->atoms, atoms.data(), sizeof(double) * atoms.size(), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = launch_vext(s->g, s->h, s->counts, s->atoms, s->a, s->vext, 1, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host atom array is a temporary
            if (e != cudaSuccess) return cuda_fail(e, "lbks_cd_run: move nuclei");
        }
        double e_tot = 0.0, n_el = 0.0;
        int rc = cd_rebuild(s, st, &e_tot, &n_el);
        if (rc != LBKS_OK) return rc;
        if (masses)  // second half: velocities with the new forces
            for (int a = 0; a < na; ++a)
                for (int c = 0; c < 3; ++c) {
                    const int i = 3 * a + c;
                    velocities[i] += 0.5 * tb * (F[i] + s->cd_F[i]) / masses[a];
                }
        if (energies) {
            energies[3 * b] = e_tot;
            energies[3 * b + 1] = kinetic();
            energies[3 * b + 2] = n_el;
        }
        if (xyz_traj) std::copy(R.begin(), R.end(), xyz_traj + (size_t)b * 3 * na);
    }
    return LBKS_OK;
}

int lbks_cd_get_orbitals(const lbks_system* s, int level, double* host, size_t cap) {
    if (!s || !host) return fail(LBKS_EINVAL, "null argument");
    if (!s->cd_ready) return fail(LBKS_EINVAL, "lbks_cd_start has not run on this handle");
    if (level != 0 && level != 1) return fail(LBKS_EINVAL, "level must be 0 (older) or 1 (current)");
    const size_t n = (size_t)2 * s->n_orb * s->N;
    if (cap < n) return fail(LBKS_EINVAL, "capacity %zu < %zu", cap, n);
    const void* src = s->cd_lev[level == 0 ? s->cd_prev : s->cd_cur];
    cudaError_t e;
    if (s->ops->psi_elem == 8) {
        e = cudaMemcpy(host, src, sizeof(double) * n, cudaMemcpyDeviceToHost);
    } else {
        std::vector<float> tmp(n);
        e = cudaMemcpy(tmp.data(), src, sizeof(float) * n, cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < n && e == cudaSuccess; ++i) host[i] = tmp[i];
    }
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_cd_get_orbitals");
}

int lbks_cd_get_state(const lbks_system* s, double* time, int64_t* steps, double* forces, size_t cap) {
    if (!s) return fail(LBKS_EINVAL, "null argument");
    if (!s->cd_ready) return fail(LBKS_EINVAL, "lbks_cd_start has not run on this handle");
    if (time) *time = s->cd_time;
    if (steps) *steps = s->cd_steps;
    if (forces) {
        if (cap < s->cd_F.size()) return fail(LBKS_EINVAL, "capacity %zu < %zu", cap, s->cd_F.size());
        std::copy(s->cd_F.begin(), s->cd_F.end(), forces);
    }
    return LBKS_OK;
}

int lbks_cd_step(int precision, int nx, int ny, int nz, int n_orb, double h, double theta, double tau,
                 const void* phi_prev, const void* phi, const double* V, const double* lambda, const double* u_coef,
                 void* phi_next, double* S_next, double* lambda_next, void* stream) {
    if (precision != LBKS_FP64 && precision != LBKS_FP32)
        return fail(LBKS_EINVAL, "concurrent dynamics needs LBKS_FP64 or LBKS_FP32");
    if (nx < 2 || ny < 2 || nz < 2 || (size_t)nx * ny * nz >= (1ull << 31))
        return fail(LBKS_EINVAL, "bad grid %d x %d x %d", nx, ny, nz);
    if (n_orb < 1 || n_orb > kMaxOrb) return fail(LBKS_EINVAL, "n_orb must be in [1, %d]", kMaxOrb);
    if (!phi || !V || !phi_next) return fail(LBKS_EINVAL, "null device pointer");
    if (phi == phi_next || phi_prev == phi_next) return fail(LBKS_EINVAL, "phi_next must not alias its inputs");
    if (!(h > 0.0) || !(theta > 0.0) || !(tau > 0.0)) return fail(LBKS_EINVAL, "bad h, theta or tau");
    if (lambda_next && !S_next) return fail(LBKS_EINVAL, "lambda_next needs S_next");
    Workspace* w = nullptr;
    int rc = workspace(stream, 0, &w);
    if (rc != LBKS_OK) return rc;
    CdIO io{};
    io.prev = phi_prev;
    io.alpha = 1.0;
    io.cur = phi;
    io.out = phi_next;
    io.V = V;
    io.lam = n_orb > 1 ? lambda : nullptr;
    io.ucoef = u_coef;
    io.S_out = S_next;
    io.lam_out = lambda_next;
    io.c_re = 0.0;
    io.c_im = 2.0 * tau / (theta * h * h);
    io.h = h;
    cudaError_t e = cd_step_launch(precision, n_orb, make_grid(nx, ny, nz), make_cd_coef(theta, h), io, w->sc, 1,
                                   (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_cd_step");
}

int lbks_cd_overlap(int precision, size_t n_sites, int n_orb, double h, const void* phi, double* S, double* lambda,
                    void* stream) {
    if (precision != LBKS_FP64 && precision != LBKS_FP32)
        return fail(LBKS_EINVAL, "concurrent dynamics needs LBKS_FP64 or LBKS_FP32");
    if (n_orb < 1 || n_orb > kMaxOrb) return fail(LBKS_EINVAL, "n_orb must be in [1, %d]", kMaxOrb);
    if (!phi || !S) return fail(LBKS_EINVAL, "null device pointer");
    if (n_sites == 0 || n_sites >= (1ull << 31)) return fail(LBKS_EINVAL, "bad n_sites");
    Workspace* w = nullptr;
    int rc = workspace(stream, 0, &w);
    if (rc != LBKS_OK) return rc;
    cudaError_t e = cd_overlap_launch(precision, n_orb, make_grid((int)n_sites, 1, 1), phi, h, S, lambda, w->sc, 1,
                                      (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_cd_overlap");
}

}  // extern "C"
