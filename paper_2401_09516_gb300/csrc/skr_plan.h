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
// Plan: see plan_launches below (a makespan model of the launches, searched
// over the cluster size of each group of equal-size chains).
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

// Relative Arnoldi steps per system of n unknowns: they grow like the grid
// side for these elliptic problems, sqrt(n) in 2D and cbrt(n) in 3D.
inline double plan_step_weight(long long n, bool three_d = false) {
    const double x = (double)std::max<long long>(n, 1);
    return three_d ? std::cbrt(x) : std::sqrt(x);
}

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

// Finish time of chains of the given durations (descending) handed out
// longest first to `slots` clusters, each taking the next chain when free.
inline double plan_lpt_makespan(const std::vector<double> &dur_desc, int slots) {
    if (dur_desc.empty()) return 0.0;
    if (slots < 1) return 1e300;
    std::vector<double> fin(std::min<size_t>((size_t)slots, dur_desc.size()), 0.0);
    for (double d : dur_desc) {
        size_t w = 0;
        for (size_t i = 1; i < fin.size(); i++)
            if (fin[i] < fin[w]) w = i;
        fin[w] += d;
    }
    double mx = 0.0;
    for (double f : fin) mx = std::max(mx, f);
    return mx;
}

// chain_n[c]: unknowns of chain c's systems; chain_len[c]: its systems.
// maxc(cs): clusters of cs CTAs that fit at once (0 if none); cap_ctas:
// CTAs that fit at once; max_clusters: cap on clusters over all launches
// (0 = none).  Returns the launches (empty if nothing can be scheduled).
//
// Model: a chain of len systems of n unknowns takes len x w(n) x t(n, cs)
// (the measured table; steps per system w(n) proportional to the grid side,
// sqrt(n) in 2D, cbrt(n) in 3D); a launch's finish time is its chains' longest-first list
// schedule over its clusters; the plan's time is the latest launch's.
// Clusters go one at a time to the launch that finishes last while CTAs
// (and the cluster cap) allow; the cluster size of each group of equal-n
// chains is chosen by coordinate descent on the plan's time, starting from
// one CTA per cluster.
template <typename MaxClusters>
std::vector<LaunchClass> plan_launches(const std::vector<long long> &chain_n, const std::vector<long long> &chain_len,
                                       int cap_ctas, MaxClusters maxc, int max_clusters,
                                       const std::vector<char> *chain_3d = nullptr) {
    const int nc = (int)chain_n.size();
    std::vector<LaunchClass> out;
    if (nc == 0 || cap_ctas < 1) return out;
    const int cap_clusters = max_clusters > 0 ? max_clusters : (1 << 30);
    std::vector<int> cands;
    for (int j = 0; j < SKR_TUNE_COLS; j++)
        if (SKR_TUNE_CS[j] <= cap_ctas && maxc(SKR_TUNE_CS[j]) > 0) cands.push_back(SKR_TUNE_CS[j]);
    if (cands.empty()) return out;
    auto chain_us = [&](int c, int cs) {
        const bool d3 = chain_3d && (*chain_3d)[c];
        return (double)chain_len[c] * plan_step_weight(chain_n[c], d3) * tuned_step_us(chain_n[c], cs);
    };
    // groups of chains with equal n
    std::vector<long long> gn;
    std::vector<int> gof(nc);
    for (int c = 0; c < nc; c++) {
        auto it = std::find(gn.begin(), gn.end(), chain_n[c]);
        if (it == gn.end()) {
            gof[c] = (int)gn.size();
            gn.push_back(chain_n[c]);
        } else {
            gof[c] = (int)(it - gn.begin());
        }
    }
    const int ng = (int)gn.size();
    // launches and cluster counts for one cluster size per group; returns the plan's time
    auto build = [&](const std::vector<int> &gcs, std::vector<LaunchClass> &L) {
        L.clear();
        for (int cs : cands) {
            LaunchClass k;
            k.cs = cs;
            for (int c = 0; c < nc; c++)
                if (gcs[gof[c]] == cs) k.chains.push_back(c);
            if (k.chains.empty()) continue;
            std::stable_sort(k.chains.begin(), k.chains.end(),
                             [&](int a, int b) { return chain_us(a, cs) > chain_us(b, cs); });
            L.push_back(k);
        }
        std::vector<std::vector<double>> dur(L.size());
        int used_ctas = 0, used_clusters = 0;
        for (size_t i = 0; i < L.size(); i++) {
            for (int c : L[i].chains) dur[i].push_back(chain_us(c, L[i].cs));
            L[i].slots = 1;
            used_ctas += L[i].cs;
            used_clusters += 1;
        }
        if (used_ctas > cap_ctas || used_clusters > cap_clusters) return 1e300;
        for (size_t i = 0; i < L.size(); i++) L[i].est_us = plan_lpt_makespan(dur[i], L[i].slots);
        for (;;) {
            size_t w = 0;
            for (size_t i = 1; i < L.size(); i++)
                if (L[i].est_us > L[w].est_us) w = i;
            LaunchClass &k = L[w];
            const int lim = std::min<int>((int)k.chains.size(), maxc(k.cs));
            if (k.slots >= lim || used_ctas + k.cs > cap_ctas || used_clusters + 1 > cap_clusters) break;
            k.slots += 1;
            used_ctas += k.cs;
            used_clusters += 1;
            k.est_us = plan_lpt_makespan(dur[w], k.slots);
        }
        double t = 0.0;
        for (const LaunchClass &k : L) t = std::max(t, k.est_us);
        // CTAs still free: to the other launches, latest first (the model is
        // an estimate; idle SMs help no one)
        for (bool grew = true; grew;) {
            grew = false;
            size_t w = L.size();
            for (size_t i = 0; i < L.size(); i++) {
                const int lim = std::min<int>((int)L[i].chains.size(), maxc(L[i].cs));
                if (L[i].slots >= lim || used_ctas + L[i].cs > cap_ctas || used_clusters + 1 > cap_clusters) continue;
                if (w == L.size() || L[i].est_us > L[w].est_us) w = i;
            }
            if (w < L.size()) {
                L[w].slots += 1;
                used_ctas += L[w].cs;
                used_clusters += 1;
                L[w].est_us = plan_lpt_makespan(dur[w], L[w].slots);
                grew = true;
            }
        }
        return t;
    };
    std::vector<int> gcs(ng, cands[0]);
    std::vector<LaunchClass> best;
    double bt = build(gcs, best);
    for (int round = 0; round < 8; round++) {
        bool improved = false;
        for (int g = ng - 1; g >= 0; g--) {   // largest grids first (usually listed last)
            const int keep = gcs[g];
            for (int cs : cands) {
                if (cs == keep) continue;
                gcs[g] = cs;
                std::vector<LaunchClass> L;
                const double t = build(gcs, L);
                if (t < bt * (1.0 - 1e-9)) {
                    bt = t;
                    best = L;
                    improved = true;
                    break;
                }
                gcs[g] = keep;
            }
            if (improved) break;
        }
        if (!improved) break;
    }
    if (bt >= 1e299) return out;
    return best;
}

}  // namespace skr
