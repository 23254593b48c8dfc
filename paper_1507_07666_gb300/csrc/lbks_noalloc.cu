// lbks_relax_step_noalloc: the relaxation step of lbks_relax_step with its
// reduction scratch in a fixed device array of this library instead of
// memory obtained from cudaMalloc.
#include "lbks.h"
#include "lbks_internal.cuh"

#include <mutex>
#include <string>

namespace lbks {
namespace {

constexpr int kStaticBlocks = 2048;                        // most blocks one launch may use
constexpr int kStaticVals = kMaxOrb * (kMaxOrb + 1) / 2;   // overlap pairs of up to kMaxOrb orbitals
constexpr size_t kStaticPartials = (size_t)kStaticBlocks * kStaticVals;

// Block partials followed by the arrival counter (32 doubles of room).
// Every GPU that loads the library holds these ~590 KB until the process exits.
static __device__ __align__(256) double g_relax_scratch[kStaticPartials + 32];

std::mutex g_mu;
double* g_addr[64] = {nullptr};  // device address of g_relax_scratch, per device

int fail(int code, const std::string& m) { return set_last_error(code, m.c_str()); }

// Resolves the array's device address once per device (with that device
// current).  In host code the symbol names a host-side shadow, not device
// memory, so the address must come from cudaGetSymbolAddress.
int static_scratch(Scratch* sc) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LBKS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(LBKS_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_relax_scratch);
        if (e != cudaSuccess || !p)
            return fail(LBKS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<double*>(p);
    }
    sc->partial = g_addr[dev];
    sc->counter = reinterpret_cast<unsigned*>(g_addr[dev] + kStaticPartials);
    sc->max_blocks = kStaticBlocks;
    sc->max_vals = kStaticVals;
    return LBKS_OK;
}

}  // namespace
}  // namespace lbks

using namespace lbks;

extern "C" int lbks_relax_step_noalloc(int precision, int nx, int ny, int nz, int n_orb, double h, double omega,
                                       double theta, double dt, const void* f_in, const void* u_in,
                                       const double* V, const double* sigma_in, void* f_out, void* psi_out,
                                       double* S_out, double* lambda_out, double* sigma_out, void* stream) {
    const PrecisionOps* ops = precision == LBKS_FP64   ? &ops_f64()
                              : precision == LBKS_FP32 ? &ops_f32()
                              : precision == LBKS_BF16 ? &ops_bf16()
                                                       : nullptr;
    int rc = LBKS_OK;
    if (!ops) rc = fail(LBKS_EINVAL, "unknown precision");
    else if (nx < 2 || ny < 2 || nz < 2 || (size_t)nx * ny * nz >= (1ull << 31))
        rc = fail(LBKS_EINVAL, "bad grid");
    else if (n_orb < 1 || n_orb > kMaxOrb)
        rc = fail(LBKS_EINVAL, "n_orb exceeds the fixed scratch of lbks_relax_step_noalloc (at most 8 orbitals)");
    else if (!f_in || !V || !sigma_in || !f_out || !psi_out || !S_out || !lambda_out || !sigma_out)
        rc = fail(LBKS_EINVAL, "null device pointer");
    else if (f_in == f_out)
        rc = fail(LBKS_EINVAL, "f_in and f_out must not alias");
    else if (!(h > 0.0) || !(omega > 0.0 && omega < 2.0))
        rc = fail(LBKS_EINVAL, "bad h or omega");
    if (rc != LBKS_OK) return rc;
    Scratch sc;
    rc = static_scratch(&sc);
    if (rc != LBKS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // The last block of every launch leaves the counter at zero; clear it
    // anyway so that a launch that never finished cannot poison this one.
    cudaError_t e = cudaMemsetAsync(sc.counter, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        RelaxIO io{f_in, u_in, V, sigma_in, f_out, psi_out, S_out, lambda_out, sigma_out};
        e = ops->relax(n_orb, make_grid(nx, ny, nz), make_coef(omega, theta, dt, h), io, sc, 1,
                       relax_variant_for(precision, n_orb, omega, nx, ny, nz), st);
    }
    if (e != cudaSuccess) return fail(LBKS_ECUDA, std::string("lbks_relax_step_noalloc: ") + cudaGetErrorString(e));
    return LBKS_OK;
}
