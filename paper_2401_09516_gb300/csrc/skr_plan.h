// Launch planning for a batch of independent chains (App. E.2.2's cut of the
// sorted list into chains, run as thread-block clusters): which cluster size
// each chain gets, how the GPU's CTAs are shared between chains of different
// sizes, and in which order a launch hands its chains out.
//
// Input: the measured table of skr_tuned.inc (written by tune.py on the GPU):
// microseconds per Arnoldi step of one cluster of cs CTAs on n unknowns, with
// the GPU full.  A chain's time is estimated as (systems) x (steps per system)
// x (time per step), steps per system taken proportional to sqrt(n) (the
// growth of a 2D elliptic problem's iteration count with the grid side); only
// ratios between chains matter.
//
// Plan:
//   1. each chain starts at the cluster size with the least CTA time per
//      step (t x cs; ties to the smaller cluster);
//   2. the ideal makespan L is the total CTA time over the GPU's CTAs; a
//      chain whose own time exceeds L gets the smallest larger cluster that
//      brings it under L (or the fastest), and L is recomputed (a few rounds);
//   3. chains of one cluster size form one launch; each launch gets clusters
//      in proportion to its CTA time, at most one per chain and at most as
//      many as fit, and the CTAs left over go to the launch that would finish
//      last;
//   4. inside a launch, chains are handed out longest first.
// Launches of different cluster sizes run concurrently on their own streams;
// their clusters never wait on one another, so a cluster that finds no SM
// free simply starts later.
#pragma once

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace skr {

#include "skr_tuned.inc"

// Microseconds per Arnoldi step of one cluster of cs CTAs on n unknowns:
// log-log interpolation in n between the table's rows (the first row below
// it, linear in n beyond the last), log-linear in cs between its columns.
inline double tuned_step_us(long long n, int cs) {
    auto col = [&](int j) {
        const double x = std::log((double)std::max<long long>(n, 1));
        if (n <= SKR_TUNE_N[0]) return SKR_TUNE_US[0][j];
        for (int i = 1; i < SKR_TUNE_ROWS; i++) {
            if (n <= SKR_TUNE_N[i]) {
                const double x0 = std::log((double)SKR_TUNE_N[i - 1]), x1 = std::log((double)SKR_TUNE_N[i]);
                const double y0 = std::log(SKR_TUNE_US[i - 1][j]), y1 = std::log(SKR_TUNE_US[i][j]);
                return std::exp(y0 + (y1 - y0) * (x - x0) / (x1 - x0));
            }
        }
        return SKR_TUNE_US[SKR_TUNE_ROWS - 1][j] * (double)n / (double)SKR_TUNE_N[SKR_TUNE_ROWS - 1];
    };
    if (cs <= SKR_TUNE_CS[0]) return col(0);
    for (int j = 1; j < SKR_TUNE_COLS; j++) {
        if (cs <= SKR_TUNE_CS[j]) {
            const double c0 = std::log((double)SKR_TUNE_CS[j - 1]), c1 = std::log((double)SKR_TUNE_CS[j]);
            const double a = (std::log((double)cs) - c0) / (c1 - c0);
            return std::exp((1.0 - a) * std::log(col(j - 1)) + a * std::log(col(j)));
        }
    }
    return col(SKR_TUNE_COLS - 1);
}

// Relative Arnoldi steps per system of n unknowns.
inline double plan_step_weight(long long n) { return std::sqrt((double)std::max<long long>(n, 1)); }

// Cluster size with the least CTA time per step (ties to the smaller).
inline int plan_efficient_cs(long long n) {
    int best = SKR_TUNE_CS[0];
    double bv = tuned_step_us(n, best) * best;
    for (int j = 1; j < SKR_TUNE_COLS; j++) {
        const int cs = SKR_TUNE_CS[j];
        const double v = tuned_step_us(n, cs) * cs;
        if (v < bv * (1.0 - 1e-9)) {
            bv = v;
            best = cs;
        }
    }
    return best;
}

struct LaunchClass {
    int cs = 1;
    int slots = 0;
    std::vector<int> chains;   // chain indices, longest first
    double est_us = 0.0;       // estimated time of the launch
};

// chain_n[c]: unknowns of chain c's systems; chain_len[c]: its systems.
// maxc(cs): clusters of cs CTAs that fit at once (0 if none); cap_ctas:
// CTAs that fit at once; max_clusters: cap on clusters over all launches
// (0 = none).  Returns the launches (empty if nothing can be scheduled).
template <typename MaxClusters>
std::vector<LaunchClass> plan_launches(const std::vector<long long> &chain_n, const std::vector<long long> &chain_len,
                                       int cap_ctas, MaxClusters maxc, int max_clusters) {
    const int nc = (int)chain_n.size();
    std::vector<LaunchClass> out;
    if (nc == 0 || cap_ctas < 1) return out;
    auto chain_us = [&](int c, int cs) {
        return (double)chain_len[c] * plan_step_weight(chain_n[c]) * tuned_step_us(chain_n[c], cs);
    };
    auto usable = [&](int cs) { return cs <= cap_ctas && maxc(cs) > 0; };
    std::vector<int> cs(nc);
    for (int c = 0; c < nc; c++) {
        cs[c] = plan_efficient_cs(chain_n[c]);
        while (!usable(cs[c]) && cs[c] > 1) cs[c] /= 2;
    }
    // 2. chains longer than the ideal makespan get larger clusters
    for (int round = 0; round < 6; round++) {
        double tot = 0.0;
        for (int c = 0; c < nc; c++) tot += chain_us(c, cs[c]) * cs[c];
        const double L = tot / cap_ctas;
        bool changed = false;
        for (int c = 0; c < nc; c++) {
            if (chain_us(c, cs[c]) <= L) continue;
            int best = cs[c];
            for (int j = 0; j < SKR_TUNE_COLS; j++) {
                const int q = SKR_TUNE_CS[j];
                if (q <= cs[c] || !usable(q)) continue;
                if (chain_us(c, q) < chain_us(c, best)) best = q;
                if (chain_us(c, best) <= L) break;
            }
            if (best != cs[c]) {
                cs[c] = best;
                changed = true;
            }
        }
        if (!changed) break;
    }
    // 3. one launch per cluster size
    for (int j = 0; j < SKR_TUNE_COLS; j++) {
        LaunchClass k;
        k.cs = SKR_TUNE_CS[j];
        for (int c = 0; c < nc; c++)
            if (cs[c] == k.cs) k.chains.push_back(c);
        if (k.chains.empty()) continue;
        std::stable_sort(k.chains.begin(), k.chains.end(),
                         [&](int a, int b) { return chain_us(a, k.cs) > chain_us(b, k.cs); });
        out.push_back(k);
    }
    std::vector<double> work(out.size(), 0.0), longest(out.size(), 0.0);
    double tot = 0.0;
    for (size_t i = 0; i < out.size(); i++) {
        for (int c : out[i].chains) {
            work[i] += chain_us(c, out[i].cs);
            longest[i] = std::max(longest[i], chain_us(c, out[i].cs));
        }
        tot += work[i] * out[i].cs;
    }
    const int cap_clusters = max_clusters > 0 ? max_clusters : (1 << 30);
    int used_ctas = 0, used_clusters = 0;
    auto limit = [&](size_t i) {
        return std::min<int>((int)out[i].chains.size(), maxc(out[i].cs));
    };
    for (size_t i = 0; i < out.size(); i++) {
        const double share = tot > 0.0 ? work[i] * out[i].cs / tot : 1.0 / out.size();
        int s = (int)std::floor(share * cap_ctas / out[i].cs);
        s = std::max(1, std::min(s, limit(i)));
        out[i].slots = s;
        used_ctas += s * out[i].cs;
        used_clusters += s;
    }
    // too many (the minimum of one cluster each can overshoot): trim the largest
    while ((used_ctas > cap_ctas || used_clusters > cap_clusters)) {
        size_t w = out.size();
        for (size_t i = 0; i < out.size(); i++)
            if (out[i].slots > 1 && (w == out.size() || out[i].slots * out[i].cs > out[w].slots * out[w].cs)) w = i;
        if (w == out.size()) break;
        out[w].slots -= 1;
        used_ctas -= out[w].cs;
        used_clusters -= 1;
    }
    // CTAs left over: to the launch that would finish last
    auto finish = [&](size_t i) { return std::max(work[i] / out[i].slots, longest[i]); };
    for (;;) {
        size_t w = out.size();
        for (size_t i = 0; i < out.size(); i++) {
            if (out[i].slots >= limit(i) || used_ctas + out[i].cs > cap_ctas || used_clusters + 1 > cap_clusters)
                continue;
            if (finish(i) <= longest[i] * (1.0 + 1e-9)) continue;   // more clusters would not help
            if (w == out.size() || finish(i) > finish(w)) w = i;
        }
        if (w == out.size()) break;
        out[w].slots += 1;
        used_ctas += out[w].cs;
        used_clusters += 1;
    }
    for (size_t i = 0; i < out.size(); i++) out[i].est_us = finish(i);
    return out;
}

}  // namespace skr
