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
    return nullptr;
}

constexpr int kScratchVals = kMaxOrb * kMaxOrb + kMaxOrb;  // largest reduction width

cudaError_t alloc_scratch(Scratch& sc) {
    sc.max_blocks = num_sms() * 8;
    sc.max_vals = kScratchVals;
    cudaError_t e = cudaMalloc(&sc.partial, sizeof(double) * (size_t)sc.max_blocks * sc.max_vals);
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&sc.counter, sizeof(unsigned) * 4);
    if (e != cudaSuccess) return e;
    return cudaMemset(sc.counter, 0, sizeof(unsigned) * 4);
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
        cudaError_t e = alloc_scratch(w->sc);
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

// Symmetric eigenvalues by cyclic Jacobi rotations (n <= 8), ascending.
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
           p->poisson_rtol > 0.0 && p->poisson_max_iter >= 1;
}

}  // namespace
}  // namespace lbks

using namespace lbks;

struct lbks_system {
    lbks_params prm;
    int nx, ny, nz, n_orb;
    double h, dt, a;
    Grid g;
    Coef c;
    const PrecisionOps* ops;
    size_t N;
    int dev;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    void* u = nullptr;
    void* psi = nullptr;
    double *vin = nullptr, *vout = nullptr, *vext = nullptr, *vh = nullptr, *rho = nullptr;
    double* pvec = nullptr;  // b, r, p, ap, z, tmp, then the multigrid levels
    CGState* cg = nullptr;
    MGHierarchy mg;
    cudaGraphExec_t poisson_graph = nullptr;  // kPoissonChunk preconditioned CG iterations
    uint64_t poisson_nodes = 0;
    double* small = nullptr;  // S, lam, sigma, Linv, e4, emat, mp, atoms
    int* status = nullptr;
    double *S, *lam, *sigma, *Linv, *e4, *emat, *mp, *atoms;
    Scratch sc;
    double* host = nullptr;  // pinned: e4[4], emat[NO^2+NO], status, cg
    cudaStream_t st = nullptr;   // internal stream for synchronous calls
    cudaStream_t cap = nullptr;  // capture stream
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    uint64_t graph_nodes[2] = {0, 0};
    std::vector<double> xyz, Z;
    bool has_geometry = false;
    lbks_energy_terms terms;
    int poisson_iters = 0;
};

namespace {

constexpr int kSmall = 4 * kMaxOrb * kMaxOrb + 4 + kScratchVals + 16;
constexpr int kMaxAtoms = 256;

constexpr int kPoissonChunk = 2;  // PCG iterations per graph launch between convergence checks

PoissonBufs poisson_bufs(double* v, size_t N, CGState* cg, double* mp) {
    return PoissonBufs{v, v + N, v + 2 * N, v + 3 * N, v + 4 * N, v + 5 * N, cg, mp};
}

int poisson_graph(lbks_system* s) {
    if (s->poisson_graph) return LBKS_OK;
    const PoissonBufs pb = poisson_bufs(s->pvec, s->N, s->cg, s->mp);
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    g_capturing = true;
    cudaError_t ee = launch_poisson_iterate(s->g, s->vh, s->prm.poisson_rtol, kPoissonChunk, pb, s->mg, s->sc, s->cap);
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

int hartree_solve(lbks_system* s, cudaStream_t st) {
    const PoissonBufs pb = poisson_bufs(s->pvec, s->N, s->cg, s->mp);
    int rc = poisson_graph(s);
    if (rc != LBKS_OK) return rc;
    cudaError_t e = launch_poisson_start(s->g, s->h, s->rho, s->vh, s->prm.poisson_rtol, pb, s->sc, st);
    if (e != cudaSuccess) return cuda_fail(e, "poisson start");
    CGState* hcg = reinterpret_cast<CGState*>(s->host + 8 + kScratchVals);
    int done_iters = 0;
    while (true) {
        e = cudaMemcpyAsync(hcg, s->cg, sizeof(CGState), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "poisson readback");
        if (hcg->done) break;
        if (done_iters >= s->prm.poisson_max_iter) {
            s->poisson_iters += hcg->iters;
            return fail(LBKS_ENOTCONV, "Hartree PCG: relative residual %.3e after %d iterations", hcg->relres,
                        hcg->iters);
        }
        e = cudaGraphLaunch(s->poisson_graph, st);
        if (e != cudaSuccess) return cuda_fail(e, "poisson iterate");
        count_launches(s->poisson_nodes);
        done_iters += kPoissonChunk;
    }
    s->poisson_iters += hcg->iters;
    return LBKS_OK;
}

// Density, Hartree, xc, potential (mixed unless first), energies of the
// current orthonormal orbitals.
int evaluate(lbks_system* s, cudaStream_t st, int first) {
    cudaError_t e = s->ops->density(s->n_orb, s->g, s->h, s->psi, s->rho, s->mp, s->sc, st);
    if (e != cudaSuccess) return cuda_fail(e, "density");
    int rc = hartree_solve(s, st);
    if (rc != LBKS_OK) return rc;
    e = launch_potential(s->g, s->h, s->rho, s->vext, s->vh, s->vout, s->vin, first, s->prm.mix, s->e4, s->sc, st);
    if (e != cudaSuccess) return cuda_fail(e, "potential");
    e = s->ops->energy_matrix(s->n_orb, s->g, s->c, s->psi, s->vout, s->emat, s->sc, st);
    if (e != cudaSuccess) return cuda_fail(e, "energy matrix");
    const int no = s->n_orb;
    double* h4 = s->host;
    double* hm = s->host + 4;
    int* hstat = reinterpret_cast<int*>(s->host + 4 + kScratchVals);
    e = cudaMemcpyAsync(h4, s->e4, sizeof(double) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hm, s->emat, sizeof(double) * (no * no + no), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hstat, s->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "energy readback");
    if (*hstat != 0) return fail(LBKS_ENOTCONV, "overlap matrix not positive definite at orbital %d", *hstat - 1);

    lbks_energy_terms& t = s->terms;
    memset(&t, 0, sizeof t);
    double ts = 0.0;
    for (int j = 0; j < no; ++j) ts += hm[no * no + j];
    t.T_s = 2.0 * ts;
    t.E_ext = h4[0];
    t.E_H = 0.5 * h4[1];
    t.E_xc = h4[2];
    t.n_electrons = h4[3];
    double enn = 0.0;
    const int na = (int)s->Z.size();
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < i; ++j) {
            const double dx = s->xyz[3 * i] - s->xyz[3 * j], dy = s->xyz[3 * i + 1] - s->xyz[3 * j + 1],
                         dz = s->xyz[3 * i + 2] - s->xyz[3 * j + 2];
            enn += s->Z[i] * s->Z[j] / std::sqrt(dx * dx + dy * dy + dz * dz);
        }
    t.E_nn = enn;
    t.E_total = t.T_s + t.E_ext + t.E_H + t.E_xc + t.E_nn;
    std::vector<double> H(no * no);
    for (int j = 0; j < no; ++j) {
        t.orbital_energies[j] = hm[j * no + j];
        for (int k = 0; k < no; ++k) H[j * no + k] = 0.5 * (hm[j * no + k] + hm[k * no + j]);
    }
    jacobi_eigenvalues(no, H, t.eigenvalues);
    return LBKS_OK;
}

// n_inner - 1 steps of Eq. KSLB and one orthonormalising step, starting from f[start].
cudaError_t enqueue_cycle(lbks_system* s, cudaStream_t st, int start) {
    int cur = start;
    const int n = s->prm.n_inner;
    for (int t = 0; t < n; ++t) {
        RelaxIO io{s->f[cur], t == 0 ? nullptr : s->u, s->vin, s->sigma, s->f[1 - cur], s->psi, s->S, s->lam, s->sigma};
        cudaError_t e = s->ops->relax(s->n_orb, s->g, s->c, io, s->sc, st);
        if (e != cudaSuccess) return e;
        cur ^= 1;
        if (t < n - 1) {
            e = s->ops->w_field(s->n_orb, s->N, s->prm.omega, s->psi, s->lam, s->u, st);
            if (e != cudaSuccess) return e;
        }
    }
    cudaError_t e = launch_cholesky(s->n_orb, s->S, s->Linv, s->status, st);
    if (e == cudaSuccess) e = s->ops->orth_apply(s->n_orb, s->N, s->Linv, s->f[cur], s->psi, st);
    if (e == cudaSuccess) e = launch_fill(s->sigma, (size_t)s->n_orb, 1.0, st);
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

int run_cycles(lbks_system* s, int fixed, int n, cudaStream_t st, lbks_result* out) {
    if (!s->has_geometry) return fail(LBKS_EINVAL, "lbks_set_geometry has not been called");
    const auto t0 = std::chrono::steady_clock::now();
    double prev = s->terms.E_total, de = INFINITY;
    int cycles = 0, converged = 0, rc = LBKS_OK;
    const int start_iters = s->poisson_iters;
    const int limit = fixed ? n : s->prm.max_cycles;
    int steps = 0;
    for (int c = 0; c < limit; ++c) {
        rc = cycle_graph(s, s->cur);
        if (rc != LBKS_OK) return rc;
        cudaError_t e = cudaGraphLaunch(s->graph[s->cur], st);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        count_launches(s->graph_nodes[s->cur]);
        s->cur ^= (s->prm.n_inner & 1);
        steps += s->prm.n_inner;
        rc = evaluate(s, st, 0);
        if (rc != LBKS_OK) return rc;
        ++cycles;
        de = std::fabs(s->terms.E_total - prev);
        prev = s->terms.E_total;
        if (!std::isfinite(s->terms.E_total)) return fail(LBKS_ENOTCONV, "total energy is not finite");
        if (!fixed && de < s->prm.e_tol) {
            converged = 1;
            break;
        }
    }
    if (out) {
        memset(out, 0, sizeof *out);
        out->E_total = s->terms.E_total;
        out->dE = de;
        for (int j = 0; j < s->n_orb; ++j) out->eigenvalues[j] = s->terms.eigenvalues[j];
        out->n_electrons = s->terms.n_electrons;
        out->cycles = cycles;
        out->steps = steps;
        out->converged = converged;
        out->poisson_iters = s->poisson_iters - start_iters;
        out->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!fixed && !converged) return fail(LBKS_ENOTCONV, "not converged after %d cycles (|dE| = %.3e)", cycles, de);
    return LBKS_OK;
}

void free_system(lbks_system* s) {
    for (int k = 0; k < 2; ++k) {
        if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
        if (s->f[k]) cudaFree(s->f[k]);
    }
    if (s->poisson_graph) cudaGraphExecDestroy(s->poisson_graph);
    void* ptrs[] = {s->u, s->psi, s->vin, s->vout, s->vext, s->vh, s->rho, s->pvec, s->cg, s->small, s->status,
                    s->sc.partial, s->sc.counter};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (s->host) cudaFreeHost(s->host);
    if (s->st) cudaStreamDestroy(s->st);
    if (s->cap) cudaStreamDestroy(s->cap);
    delete s;
}

}  // namespace

extern "C" {

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
    p->poisson_max_iter = 20000;
}

int lbks_last_error(char* buf, size_t cap) {
    if (buf && cap) {
        const size_t n = std::min(cap - 1, g_err.size());
        memcpy(buf, g_err.data(), n);
        buf[n] = '\0';
    }
    return (int)g_err.size();
}

const char* lbks_version(void) { return "lbks 0.1 (sm_103a)"; }

uint64_t lbks_kernel_launches(void) { return g_launches.load(); }

size_t lbks_system_bytes(const lbks_params* p, int nx, int ny, int nz, int n_orb) {
    if (!valid_params(p) || nx < 2 || ny < 2 || nz < 2 || n_orb < 1 || n_orb > kMaxOrb) return 0;
    const size_t N = (size_t)nx * ny * nz;
    const size_t e = ops_for(p->precision)->elem;
    return e * N * ((size_t)n_orb * 19 * 2 + (size_t)std::max(1, n_orb - 1) + n_orb) + sizeof(double) * N * 11 +
           sizeof(double) * mg_coarse_doubles(nx, ny, nz) +
           sizeof(double) * ((size_t)num_sms() * 8 * kScratchVals + kSmall);
}

int lbks_create_system(const lbks_params* p, int nx, int ny, int nz, double h, int n_orb, lbks_system** out) {
    if (!out) return fail(LBKS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!valid_params(p)) return fail(LBKS_EINVAL, "invalid lbks_params");
    if (nx < 2 || ny < 2 || nz < 2) return fail(LBKS_EINVAL, "grid must be at least 2 sites per axis");
    if (!(h > 0.0)) return fail(LBKS_EINVAL, "h must be positive");
    if (n_orb < 1 || n_orb > kMaxOrb) return fail(LBKS_EINVAL, "n_orb must be in [1, %d]", kMaxOrb);
    if ((size_t)nx * ny * nz >= (1ull << 31)) return fail(LBKS_EINVAL, "grid has 2^31 sites or more");
    lbks_system* s = new lbks_system();
    s->prm = *p;
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->n_orb = n_orb;
    s->h = h;
    s->dt = p->theta * h * h * (2.0 - p->omega) / p->omega;
    s->a = p->softening > 0.0 ? p->softening : h;
    s->g = make_grid(nx, ny, nz);
    s->c = make_coef(p->omega, p->theta, s->dt, h);
    s->ops = ops_for(p->precision);
    s->N = (size_t)nx * ny * nz;
    cudaGetDevice(&s->dev);
    memset(&s->terms, 0, sizeof s->terms);
    const size_t e = s->ops->elem, N = s->N;
    cudaError_t err = cudaSuccess;
    auto A = [&](void** ptr, size_t bytes) {
        if (err == cudaSuccess) err = cudaMalloc(ptr, bytes);
    };
    A(&s->f[0], e * N * 19 * n_orb);
    A(&s->f[1], e * N * 19 * n_orb);
    A(&s->u, e * N * std::max(1, n_orb - 1));
    A(&s->psi, e * N * n_orb);
    A((void**)&s->vin, 8 * N);
    A((void**)&s->vout, 8 * N);
    A((void**)&s->vext, 8 * N);
    A((void**)&s->vh, 8 * N);
    A((void**)&s->rho, 8 * N);
    A((void**)&s->pvec, 8 * (6 * N + mg_coarse_doubles(nx, ny, nz)));
    A((void**)&s->cg, sizeof(CGState));
    A((void**)&s->small, sizeof(double) * (kSmall + 4 * kMaxAtoms));
    A((void**)&s->status, sizeof(int) * 4);
    if (err == cudaSuccess) err = alloc_scratch(s->sc);
    if (err == cudaSuccess) err = cudaMallocHost((void**)&s->host, sizeof(double) * (16 + kScratchVals + 16));
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaMemset(s->vh, 0, 8 * N);
    if (err == cudaSuccess) err = cudaMemset(s->u, 0, e * N * std::max(1, n_orb - 1));
    if (err == cudaSuccess) err = cudaMemset(s->status, 0, sizeof(int) * 4);
    if (err != cudaSuccess) {
        int rc = cuda_fail(err, "lbks_create_system");
        free_system(s);
        return rc;
    }
    s->mg = make_hierarchy(s->g, s->pvec + 6 * N);
    const int M = kMaxOrb * kMaxOrb;
    s->S = s->small;
    s->lam = s->S + M;
    s->Linv = s->lam + M;
    s->sigma = s->Linv + M;
    s->e4 = s->sigma + M;
    s->emat = s->e4 + 4;
    s->mp = s->emat + kScratchVals;
    s->atoms = s->mp + 16;
    *out = s;
    return LBKS_OK;
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
    if (!s || !xyz || !Z) return fail(LBKS_EINVAL, "null argument");
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
    s->xyz.assign(xyz, xyz + 3 * n_atoms);
    s->Z.assign(Z, Z + n_atoms);
    std::vector<double> atoms(4 * n_atoms);
    for (int i = 0; i < n_atoms; ++i) {
        atoms[4 * i] = xyz[3 * i];
        atoms[4 * i + 1] = xyz[3 * i + 1];
        atoms[4 * i + 2] = xyz[3 * i + 2];
        atoms[4 * i + 3] = Z[i];
    }
    cudaStream_t st = s->st;
    cudaError_t e = cudaMemcpyAsync(s->atoms, atoms.data(), sizeof(double) * 4 * n_atoms, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_vext(s->g, s->h, n_atoms, s->atoms, s->a, s->vext, st);
    // Gaussian start (see include/lbks.h)
    std::vector<int> order(n_atoms);
    for (int i = 0; i < n_atoms; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return Z[a] > Z[b]; });
    OrbitalStart starts[kMaxOrb];
    for (int j = 0; j < s->n_orb; ++j) {
        const int I = order[j % n_atoms], m = j / n_atoms;
        starts[j].cx = xyz[3 * I] + 0.25 * std::sin(1.0 + 2.1 * j);
        starts[j].cy = xyz[3 * I + 1] + 0.25 * std::sin(2.0 + 3.3 * j);
        starts[j].cz = xyz[3 * I + 2] + 0.25 * std::sin(3.0 + 4.7 * j);
        starts[j].width = 1.2 * (1.0 + 0.35 * m);
    }
    if (e == cudaSuccess) e = s->ops->init_orbitals(s->n_orb, s->g, s->h, starts, s->psi, st);
    if (e == cudaSuccess) e = s->ops->gram(s->n_orb, s->g, s->h, s->psi, s->S, s->sc, st);
    if (e == cudaSuccess) e = launch_cholesky(s->n_orb, s->S, s->Linv, s->status, st);
    if (e == cudaSuccess) e = s->ops->orth_apply(s->n_orb, s->N, s->Linv, nullptr, s->psi, st);
    if (e == cudaSuccess) e = s->ops->equilibrium(s->n_orb, s->N, s->c, s->psi, s->f[0], st);
    if (e == cudaSuccess) e = launch_fill(s->sigma, (size_t)s->n_orb, 1.0, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->vh, 0, sizeof(double) * s->N, st);
    if (e != cudaSuccess) return cuda_fail(e, "lbks_set_geometry");
    s->cur = 0;
    s->has_geometry = true;
    s->poisson_iters = 0;
    int rc = evaluate(s, st, 1);
    if (rc != LBKS_OK) s->has_geometry = false;
    return rc;
}

int lbks_scf(lbks_system* s, void* stream, lbks_result* out) {
    if (!s) return fail(LBKS_EINVAL, "system is NULL");
    return run_cycles(s, 0, 0, (cudaStream_t)stream, out);
}

int lbks_scf_cycles(lbks_system* s, int n, void* stream, lbks_result* out) {
    if (!s || n < 0) return fail(LBKS_EINVAL, "bad argument");
    return run_cycles(s, 1, n, (cudaStream_t)stream, out);
}

int lbks_energy(const lbks_system* s, lbks_energy_terms* out) {
    if (!s || !out) return fail(LBKS_EINVAL, "null argument");
    if (!s->has_geometry) return fail(LBKS_EINVAL, "lbks_set_geometry has not been called");
    *out = s->terms;
    return LBKS_OK;
}

int lbks_get_density(const lbks_system* s, double* host, size_t cap) {
    if (!s || !host) return fail(LBKS_EINVAL, "null argument");
    if (cap < s->N) return fail(LBKS_EINVAL, "capacity %zu < %zu", cap, s->N);
    cudaError_t e = cudaMemcpy(host, s->rho, sizeof(double) * s->N, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_get_density");
}

int lbks_get_orbitals(const lbks_system* s, double* host, size_t cap) {
    if (!s || !host) return fail(LBKS_EINVAL, "null argument");
    const size_t n = s->N * s->n_orb;
    if (cap < n) return fail(LBKS_EINVAL, "capacity %zu < %zu", cap, n);
    if (s->ops->elem == sizeof(double)) {
        cudaError_t e = cudaMemcpy(host, s->psi, sizeof(double) * n, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_get_orbitals");
    }
    std::vector<float> tmp(n);
    cudaError_t e = cudaMemcpy(tmp.data(), s->psi, sizeof(float) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "lbks_get_orbitals");
    for (size_t i = 0; i < n; ++i) host[i] = tmp[i];
    return LBKS_OK;
}

int lbks_get_potential(const lbks_system* s, int which, double* host, size_t cap) {
    if (!s || !host) return fail(LBKS_EINVAL, "null argument");
    if (cap < s->N) return fail(LBKS_EINVAL, "capacity %zu < %zu", cap, s->N);
    const double* src = which == 0 ? s->vin : which == 1 ? s->vout : which == 2 ? s->vh : which == 3 ? s->vext : nullptr;
    if (!src) return fail(LBKS_EINVAL, "which must be 0..3");
    cudaError_t e = cudaMemcpy(host, src, sizeof(double) * s->N, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_get_potential");
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
    if (n_orb < 1 || n_orb > kMaxOrb) return fail(LBKS_EINVAL, "n_orb must be in [1, %d]", kMaxOrb);
    if (!f_in || !V || !sigma_in || !f_out || !psi_out || !S_out || !lambda_out || !sigma_out)
        return fail(LBKS_EINVAL, "null device pointer");
    if (f_in == f_out) return fail(LBKS_EINVAL, "f_in and f_out must not alias");
    if (!(h > 0.0) || !(omega > 0.0 && omega < 2.0)) return fail(LBKS_EINVAL, "bad h or omega");
    Workspace* w = nullptr;
    int rc = workspace(stream, 0, &w);
    if (rc != LBKS_OK) return rc;
    RelaxIO io{f_in, u_in, V, sigma_in, f_out, psi_out, S_out, lambda_out, sigma_out};
    cudaError_t e = ops->relax(n_orb, make_grid(nx, ny, nz), make_coef(omega, theta, dt, h), io, w->sc,
                               (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_relax_step");
}

int lbks_w_field(int precision, size_t n_sites, int n_orb, double omega, const void* psi, const double* lambda,
                 void* u_out, void* stream) {
    const PrecisionOps* ops = ops_for(precision);
    if (!ops) return fail(LBKS_EINVAL, "unknown precision %d", precision);
    if (n_orb < 1 || n_orb > kMaxOrb || !psi || !lambda || (n_orb > 1 && !u_out))
        return fail(LBKS_EINVAL, "bad argument");
    if (n_sites == 0) return LBKS_OK;
    cudaError_t e = ops->w_field(n_orb, n_sites, omega, psi, lambda, u_out, (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_w_field");
}

int lbks_cholesky_inverse(int n, const double* S, double* Linv, int* status, void* stream) {
    if (n < 1 || n > kMaxOrb || !S || !Linv || !status) return fail(LBKS_EINVAL, "bad argument");
    cudaError_t e = launch_cholesky(n, S, Linv, status, (cudaStream_t)stream);
    return e == cudaSuccess ? LBKS_OK : cuda_fail(e, "lbks_cholesky_inverse");
}

int lbks_orth_apply(int precision, size_t n_sites, int n_orb, const double* Linv, void* f, void* psi,
                    void* stream) {
    const PrecisionOps* ops = ops_for(precision);
    if (!ops) return fail(LBKS_EINVAL, "unknown precision %d", precision);
    if (n_orb < 1 || n_orb > kMaxOrb || !Linv) return fail(LBKS_EINVAL, "bad argument");
    if (n_sites == 0 || (!f && !psi)) return LBKS_OK;
    cudaError_t e = ops->orth_apply(n_orb, n_sites, Linv, f, psi, (cudaStream_t)stream);
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
    const PoissonBufs pb = poisson_bufs(w->pvec, g.N, w->cg, w->mp);
    const MGHierarchy H = make_hierarchy(g, w->pvec + 6 * (size_t)g.N);
    cudaError_t e = launch_multipoles_from_rho(g, h, rho, w->mp, w->sc, st);
    if (e == cudaSuccess) e = launch_poisson_start(g, h, rho, v, rtol, pb, w->sc, st);
    if (e != cudaSuccess) return cuda_fail(e, "lbks_hartree");
    CGState hcg;
    int done = 0;
    while (true) {
        e = cudaMemcpyAsync(&hcg, w->cg, sizeof hcg, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "lbks_hartree readback");
        if (hcg.done || done >= max_iter) break;
        const int chunk = std::min(2, max_iter - done);
        e = launch_poisson_iterate(g, v, rtol, chunk, pb, H, w->sc, st);
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
