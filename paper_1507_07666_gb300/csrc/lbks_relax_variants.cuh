// Definitions of the two-site, the prefetching and the bulk-copy stream-collide launchers
// (declared in lbks_relax.cuh); each lbks_relax_<precision>_<variant>.cu
// includes this and instantiates one of them for its precision.
#pragma once

#include "lbks_relax.cuh"
#include "lbks_bulk.cuh"

namespace lbks {

// Dispatch on (NO, omega == 1, batched) to the compile-time kernels.
template <typename TS, typename T, template <typename, typename, int, bool, bool> class L>
cudaError_t dispatch_variant(int NO, bool om1, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc,
                             int B, cudaStream_t st) {
    const bool b = B > 1;
#define LBKS_CASE(N)                                                                                 \
    case N:                                                                                          \
        return om1 ? (b ? L<TS, T, N, true, true>::run(g, c, io, sc, B, st)                          \
                        : L<TS, T, N, true, false>::run(g, c, io, sc, B, st))                        \
                   : (b ? L<TS, T, N, false, true>::run(g, c, io, sc, B, st)                         \
                        : L<TS, T, N, false, false>::run(g, c, io, sc, B, st));
    switch (NO) {
        LBKS_CASE(1) LBKS_CASE(2) LBKS_CASE(3) LBKS_CASE(4) LBKS_CASE(5) LBKS_CASE(6) LBKS_CASE(7) LBKS_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef LBKS_CASE
}

template <typename TS, typename T, int NO, bool OM1, bool BATCHED>
struct PairLaunch {
    static cudaError_t run(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                           cudaStream_t st) {
        return launch_stream_collide_pair<TS, T, NO, OM1, BATCHED>(g, c, io, sc, B, st);
    }
};
template <typename TS, typename T, int NO, bool OM1, bool BATCHED>
struct PrefetchLaunch {
    static cudaError_t run(const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                           cudaStream_t st) {
        return launch_stream_collide<TS, T, NO, OM1, BATCHED, true>(g, c, io, sc, B, st);
    }
};

template <typename TS, typename T>
cudaError_t launch_relax_bulk(int NO, const Grid& g, const Coef& c, const RelaxIO& io, const Scratch& sc, int B,
                              bool exact, cudaStream_t st) {
    return launch_stream_collide_bulk<TS, T>(NO, g, c, io, sc, B, exact, device_wait_limit(), st);
}

// Orbital counts LO..HI only.
template <typename TS, typename T, int LO, int HI>
cudaError_t launch_relax_pairs_range(int NO, bool om1, const Grid& g, const Coef& c, const RelaxIO& io,
                                     const Scratch& sc, int B, cudaStream_t st) {
    const bool b = B > 1;
#define LBKS_CASE(N)                                                                                 \
    case N:                                                                                          \
        if constexpr (N >= LO && N <= HI)                                                            \
            return om1 ? (b ? PairLaunch<TS, T, N, true, true>::run(g, c, io, sc, B, st)              \
                            : PairLaunch<TS, T, N, true, false>::run(g, c, io, sc, B, st))            \
                       : (b ? PairLaunch<TS, T, N, false, true>::run(g, c, io, sc, B, st)             \
                            : PairLaunch<TS, T, N, false, false>::run(g, c, io, sc, B, st));          \
        return cudaErrorInvalidValue;
    switch (NO) {
        LBKS_CASE(1) LBKS_CASE(2) LBKS_CASE(3) LBKS_CASE(4) LBKS_CASE(5) LBKS_CASE(6) LBKS_CASE(7) LBKS_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef LBKS_CASE
}
template <typename TS, typename T>
cudaError_t launch_relax_prefetch(int NO, bool om1, const Grid& g, const Coef& c, const RelaxIO& io,
                                  const Scratch& sc, int B, cudaStream_t st) {
    return dispatch_variant<TS, T, PrefetchLaunch>(NO, om1, g, c, io, sc, B, st);
}

}  // namespace lbks
