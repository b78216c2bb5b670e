// Residency planning of the subdomain cache (see sddm_cache.h): which cells
// are loaded where, which are evicted, and in which groups a wave is traced.
// Host code only; the device side carries the plans out (cell_cache.cu).
#include <algorithm>
#include <cstdio>

#include "sddm_cache.h"

namespace sddm {
namespace {
int64_t round_up(int64_t x, int64_t u) { return (x + u - 1) / u * u; }
}  // namespace

int64_t CellPlanner::cell_bytes(int c) const {
    return round_up(64 * node_cnt[c], kUnit) + round_up(48 * tri_cnt[c], kUnit);
}

std::string CellPlanner::init(const std::vector<int64_t> &nc, const std::vector<int64_t> &tc, int64_t bytes) {
    node_cnt = nc;
    tri_cnt = tc;
    n_cells = (int)nc.size();
    budget = bytes / kUnit * kUnit;
    int64_t largest = 0;
    for (int c = 0; c < n_cells; ++c) largest = std::max(largest, cell_bytes(c));
    if (largest > budget) {
        char msg[200];
        std::snprintf(msg, sizeof msg,
                      "sddm_build: cell_cache_bytes (%lld) is smaller than the largest subdomain BVH (%lld bytes)",
                      (long long)bytes, (long long)largest);
        return msg;
    }
    if (budget / 64 >= (1LL << 31) || budget / 48 >= (1LL << (31 - kLeafBits)))
        return "sddm_build: cell_cache_bytes too large for the node and leaf encoding";
    off.assign(n_cells, -1);
    stamp.assign(n_cells, 0);
    free_.clear();
    free_[0] = budget;
    clock = 0;
    hits = 0;
    return "";
}

// First fit in the free ranges; when nothing fits, evict the least recently
// used resident cell outside the current group and try again.
bool CellPlanner::allocate(int c, const std::vector<char> &in_group, int64_t &where, std::vector<int> &evicted) {
    const int64_t need = cell_bytes(c);
    for (;;) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= need) {
                where = it->first;
                const int64_t rest = it->second - need;
                free_.erase(it);
                if (rest > 0) free_[where + need] = rest;
                return true;
            }
        }
        int victim = -1;
        for (int y = 0; y < n_cells; ++y)
            if (off[y] >= 0 && !in_group[y] && (victim < 0 || stamp[y] < stamp[victim])) victim = y;
        if (victim < 0) return false;
        // the victim's range back to the free list, merged with its neighbours
        int64_t o = off[victim], len = cell_bytes(victim);
        off[victim] = -1;
        evicted.push_back(victim);
        auto nx = free_.lower_bound(o);
        if (nx != free_.end() && nx->first == o + len) {
            len += nx->second;
            free_.erase(nx);
        }
        auto pv = free_.lower_bound(o);
        if (pv != free_.begin()) {
            --pv;
            if (pv->first + pv->second == o) {
                o = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[o] = len;
    }
}

std::vector<CellPlanner::Group> CellPlanner::plan_wave(const std::vector<int64_t> &cell_rays, int *perm) {
    std::vector<int> pending;
    for (int c = 0; c < n_cells; ++c)
        if (cell_rays[c] > 0) pending.push_back(c);
    std::stable_sort(pending.begin(), pending.end(), [&](int x, int y) { return cell_rays[x] > cell_rays[y]; });
    std::vector<Group> plan;
    int pos = 0;
    int64_t placed = 0;
    std::vector<char> done(n_cells, 0);
    while (!pending.empty()) {
        Group gp;
        std::vector<char> in_group(n_cells, 0);
        for (int c : pending)
            if (off[c] >= 0) {
                gp.cells.push_back(c);
                in_group[c] = 1;
                ++hits;
            }
        for (int c : pending) {
            if (in_group[c]) continue;
            Load ld;
            ld.cell = c;
            if (!allocate(c, in_group, ld.where, ld.evicted)) continue;
            off[c] = ld.where;
            gp.cells.push_back(c);
            in_group[c] = 1;
            gp.loads.push_back(std::move(ld));
        }
        if (gp.cells.empty()) return {};   // cannot happen: init checked the largest cell
        gp.begin = placed;
        for (int c : gp.cells) {
            gp.where.push_back(off[c]);
            perm[pos++] = c;
            placed += cell_rays[c];
            stamp[c] = ++clock;
            done[c] = 1;
        }
        gp.end = placed;
        std::vector<int> rest;
        for (int c : pending)
            if (!in_group[c]) rest.push_back(c);
        pending.swap(rest);
        plan.push_back(std::move(gp));
    }
    for (int c = 0; c < n_cells; ++c)
        if (!done[c]) perm[pos++] = c;
    return plan;
}

}  // namespace sddm
