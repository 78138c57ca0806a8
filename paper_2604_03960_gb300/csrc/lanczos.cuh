// lanczos.cuh -- internal interface of the device Lanczos solver.
#pragma once
#include <functional>

#include "common.cuh"

namespace dmrg {

constexpr int LZ_MAXK = 24;

// Device-resident Lanczos state (one per solve).
struct LzState {
    double alpha[LZ_MAXK];
    double beta[LZ_MAXK + 1];   // beta[j] couples v_{j-1} and v_j
    double y[LZ_MAXK];          // lowest eigenvector of T
    double amax, E, scale;
    int K, m, active, nan;
};

struct LanczosWork {
    double *V = nullptr;        // K vectors of length n
    double *w = nullptr;        // work vector
    double *partials = nullptr;
    LzState *lz = nullptr;
    double *c = nullptr;
    unsigned *counter = nullptr;
};

using MatvecFn = std::function<dmrg_status(const double *x, double *y)>;

size_t lanczos_work_bytes(long long n, int K, int num_sms);
LanczosWork lanczos_work_carve(void *base, long long n, int K, int num_sms);
// theta: start vector on entry, normalised Ritz vector on exit; the Ritz
// value is left in work.lz->E (device).
// sink (may be null): where each new Lanczos vector's right-operand split
// for the next tensor-core matvec is written as well
dmrg_status lanczos_run(dmrg_ctx *ctx, const LanczosWork &w, long long n, int K, double *theta,
                        const MatvecFn &matvec, const SplitSink *sink = nullptr);

}  // namespace dmrg
