// Step-size schedule of the TV perturbations (shared by the single-context and the
// batched drivers; the ell draw is also used on the device by the TV-check cycle kernel).
//   NTVS (Appendix C): ell_k = rand(k, ell_{k-1}), a uniform integer between the two
//     (inclusive) taken from draw k of a SplitMix64 stream; try t of the cycle uses
//     beta0 * alpha^(ell_k + t).
//   OTVS (Appendix B): ell is never reset, ell_k = ell_{k-1}; otherwise as NTVS.  The
//     paper's OTVS is this rule with N = 1, alpha = 1/2, beta0 = 1 and the TV check.
//   decoupled (Sec. VI): beta_{k,n} = beta0 * alpha^n * gamma^k, n and k counted from 0,
//     no ell; defined without the TV check.
#pragma once
#include <cmath>
#include <cstdint>

#include "ntvs.h"

#ifdef __CUDACC__
#define NTVS_HD __host__ __device__
#else
#define NTVS_HD
#endif

namespace ntvs {

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) in counter form: output n of stream seed.
NTVS_HD inline uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// rand(k, ell_{k-1}) of the NTVS rule
NTVS_HD inline int64_t draw_ell(uint64_t seed, int64_t k, int64_t ell_prev) {
    const int64_t lo = k < ell_prev ? k : ell_prev, hi = k < ell_prev ? ell_prev : k;
    const uint64_t span = (uint64_t)(hi - lo) + 1u;
    return lo + (int64_t)(splitmix64_at(seed, (uint64_t)k) % span);
}

// ell at the start of cycle k (the decoupled rule records k)
inline int64_t cycle_ell(const ntvs_params& p, int64_t k, int64_t ell_prev) {
    if (p.step_rule == NTVS_STEP_OTVS) return ell_prev;
    if (p.step_rule == NTVS_STEP_DECOUPLED) return k;
    return draw_ell(p.seed, k, ell_prev);
}

// beta of a try at step n of cycle k with the current ell
inline double step_beta(const ntvs_params& p, int64_t k, int n, int64_t ell) {
    if (p.step_rule == NTVS_STEP_DECOUPLED) return p.beta0 * std::pow(p.alpha, (double)n) * std::pow(p.gamma, (double)k);
    return p.beta0 * std::pow(p.alpha, (double)ell);
}

// whether ell advances after a try (not under the decoupled rule)
inline bool ell_advances(const ntvs_params& p) { return p.step_rule != NTVS_STEP_DECOUPLED; }

}  // namespace ntvs
