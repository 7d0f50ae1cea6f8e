// Contiguous cost-balanced blocks of a batch of macro Gauss points for several
// processes (one GPU each).  Host code; no device work.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/rve.h"
#include "rve_internal.h"

namespace {

// Greedy feasibility of a largest block cost `cap`: the fewest contiguous blocks
// whose costs stay within cap (each point has cost <= cap).
int64_t blocks_needed(const std::vector<double>& cost, double cap) {
    int64_t n = 1;
    double acc = 0.0;
    for (double c : cost) {
        if (acc + c > cap) {
            ++n;
            acc = c;
        } else {
            acc += c;
        }
    }
    return n;
}

}  // namespace

extern "C" int rve_partition_blocks(int64_t G, const double* cost, int n_ranks, int64_t* offsets,
                                    double* imbalance) {
    if (G < 0 || n_ranks < 1 || !offsets || (G > 0 && !cost)) {
        rve::set_error("rve_partition_blocks: invalid argument");
        return RVE_ERR_INVALID_ARGUMENT;
    }
    std::vector<double> c(cost, cost + G);
    double total = 0.0, cmax = 0.0;
    for (double v : c) {
        if (!(v > 0.0) || !std::isfinite(v)) {
            rve::set_error("rve_partition_blocks: every cost must be positive and finite");
            return RVE_ERR_INVALID_ARGUMENT;
        }
        total += v;
        cmax = std::max(cmax, v);
    }
    offsets[0] = 0;
    if (G == 0) {
        for (int r = 1; r <= n_ranks; ++r) offsets[r] = 0;
        if (imbalance) *imbalance = 1.0;
        return RVE_OK;
    }
    // smallest cap for which n_ranks contiguous blocks suffice (bisection on the
    // linear-partition bound; the greedy test is monotone in cap)
    double lo = std::max(cmax, total / n_ranks), hi = total;
    for (int it = 0; it < 100 && hi - lo > 1e-12 * total; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (blocks_needed(c, mid) <= n_ranks)
            hi = mid;
        else
            lo = mid;
    }
    // boundaries: greedy with cap hi, then the remaining ranks get empty blocks
    int r = 0;
    double acc = 0.0, worst = 0.0;
    for (int64_t g = 0; g < G; ++g) {
        if (acc + c[g] > hi && r + 1 < n_ranks) {
            worst = std::max(worst, acc);
            offsets[++r] = g;
            acc = 0.0;
        }
        acc += c[g];
    }
    worst = std::max(worst, acc);
    for (int k = r + 1; k <= n_ranks; ++k) offsets[k] = G;
    if (imbalance) *imbalance = worst / (total / n_ranks);
    return RVE_OK;
}
