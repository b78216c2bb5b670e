// Host check of the subdomain-cache planner (cell_plan.cpp) and of the index
// relocation the device applies after each load, run by
// tests/test_host_bvh_cpu.py. A grid BVH over a random triangle soup is
// packed the way sddm_build packs it (per-cell node and triangle runs, child
// and leaf indices absolute), then many waves of random per-cell ray counts
// are planned against a budget of about a quarter of the cells. Each plan is
// carried out on a host copy of the cache, and every cell of every group
// must then be complete where the trace will read it:
//  1. perm is a permutation of the cells and the group ranges tile the queue;
//  2. the cells of a group never overlap and stay inside the budget;
//  3. from its relocated root a group cell reaches only its own nodes and
//     triangle records, and exactly its own triangles.
#include <cstdio>
#include <cstring>
#include <random>
#include <set>
#include <string>
#include <vector>

#include "sddm_cache.h"

namespace sddm {
void set_error(const std::string &) {}
}
using namespace sddm;

static int as_int(float f) {
    int i;
    std::memcpy(&i, &f, 4);
    return i;
}
static float as_float(int i) {
    float f;
    std::memcpy(&f, &i, 4);
    return f;
}

int main() {
    std::mt19937 g(11);
    std::uniform_real_distribution<float> U(0.f, 1.f);
    const int nt = 20000;
    std::vector<BuildTri> tris(nt);
    for (int i = 0; i < nt; ++i) {
        float c[3] = {U(g) * 8, U(g) * 6, U(g) * 3};
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) tris[i].v[k][a] = c[a] + (U(g) - 0.5f) * 0.3f;
        tris[i].id = (uint32_t)i;
        tris[i].obj = (uint32_t)i;
        tris[i].flags = 0;
    }
    const float lo[3] = {-0.5f, -0.5f, -0.5f}, hi[3] = {8.5f, 6.5f, 3.5f};
    const int dims[3] = {4, 4, 2};
    std::vector<PackedBVH> cells;
    build_grid(tris, dims, lo, hi, 4, 16, 1e-6f, cells, 4);
    const int nc = (int)cells.size();
    // pack as sddm_build does
    std::vector<float4> nodes, trefs;
    std::vector<int64_t> nbase, ncnt, tbase, tcnt;
    std::vector<std::set<int>> members(nc);
    for (int c = 0; c < nc; ++c) {
        const int nb = (int)(nodes.size() / 4), tb = (int)(trefs.size() / 3);
        nbase.push_back(nb);
        tbase.push_back(tb);
        ncnt.push_back((int64_t)cells[c].nodes.size() / 4);
        tcnt.push_back((int64_t)cells[c].tris.size() / 3);
        for (size_t k = 0; k < cells[c].nodes.size(); k += 4) {
            float4 n3 = cells[c].nodes[k + 3];
            int ch[2] = {as_int(n3.x), as_int(n3.y)};
            for (int q = 0; q < 2; ++q) {
                if (ch[q] >= 0) {
                    ch[q] += nb;
                } else {
                    const int v = ~ch[q];
                    ch[q] = ~((((v >> kLeafBits) + tb) << kLeafBits) | (v & ((1 << kLeafBits) - 1)));
                }
            }
            n3.x = as_float(ch[0]);
            n3.y = as_float(ch[1]);
            cells[c].nodes[k + 3] = n3;
        }
        nodes.insert(nodes.end(), cells[c].nodes.begin(), cells[c].nodes.end());
        trefs.insert(trefs.end(), cells[c].tris.begin(), cells[c].tris.end());
        for (size_t k = 0; k < cells[c].tris.size(); k += 3) members[c].insert(as_int(cells[c].tris[k].w));
    }
    CellPlanner probe;
    int64_t total = 0;
    for (int c = 0; c < nc; ++c) {
        probe.node_cnt = ncnt;
        probe.tri_cnt = tcnt;
        probe.n_cells = nc;
        total += probe.cell_bytes(c);
    }
    CellPlanner pl;
    const int64_t budget = total / 4;
    std::string why = pl.init(ncnt, tcnt, budget);
    if (!why.empty()) {
        std::printf("init: %s\n", why.c_str());
        return 1;
    }
    std::string small = CellPlanner().init(ncnt, tcnt, 1024);
    if (small.empty()) {
        std::printf("a budget below the largest cell was accepted\n");
        return 1;
    }
    std::vector<float4> cache((size_t)(budget / 16));
    std::vector<int> root(nc, -1);
    std::vector<int> perm(nc);
    int64_t loads = 0, bad = 0;
    for (int wave = 0; wave < 60; ++wave) {
        std::vector<int64_t> rays(nc, 0);
        for (int c = 0; c < nc; ++c)
            if (U(g) < 0.7f) rays[c] = (int64_t)(U(g) * 1000) + 1;
        const auto plan = pl.plan_wave(rays, perm.data());
        // 1. permutation and ranges
        std::vector<int> seen(nc, 0);
        for (int c : perm) ++seen[c];
        for (int c = 0; c < nc; ++c) bad += seen[c] != 1;
        int64_t at = 0, want = 0;
        for (int64_t r : rays) want += r;
        int pos = 0;
        for (const auto &gp : plan) {
            bad += gp.begin != at;
            for (int c : gp.cells) {
                bad += perm[pos++] != c;
                at += rays[c];
            }
            bad += gp.end != at;
            // carry out the loads: copy, relocate, root
            for (const auto &ld : gp.loads) {
                const int c = ld.cell;
                for (int y : ld.evicted)
                    for (int q : gp.cells) bad += y == q;   // never evict a cell of this group
                const int64_t node_bytes = (64 * ncnt[c] + CellPlanner::kUnit - 1) / CellPlanner::kUnit *
                                           CellPlanner::kUnit;
                if (ld.where < 0 || ld.where + pl.cell_bytes(c) > budget || ld.where % CellPlanner::kUnit) {
                    ++bad;
                    continue;
                }
                float4 *base = cache.data() + ld.where / 16;
                std::memcpy(base, nodes.data() + 4 * nbase[c], 64 * ncnt[c]);
                std::memcpy(base + node_bytes / 16, trefs.data() + 3 * tbase[c], 48 * tcnt[c]);
                const int new_node = (int)(ld.where / 64), new_tri = (int)((ld.where + node_bytes) / 48);
                for (int64_t i = 0; i < ncnt[c]; ++i) {
                    float4 &n3 = base[4 * i + 3];
                    n3.x = as_float(relocate_child(as_int(n3.x), new_node - (int)nbase[c], new_tri - (int)tbase[c]));
                    n3.y = as_float(relocate_child(as_int(n3.y), new_node - (int)nbase[c], new_tri - (int)tbase[c]));
                }
                root[c] = new_node;
                ++loads;
            }
            // 2. the group's cells do not overlap one another
            std::vector<std::pair<int64_t, int64_t>> spans;
            for (size_t j = 0; j < gp.cells.size(); ++j)
                spans.push_back({gp.where[j], gp.where[j] + pl.cell_bytes(gp.cells[j])});
            std::sort(spans.begin(), spans.end());
            for (size_t k = 1; k < spans.size(); ++k) bad += spans[k].first < spans[k - 1].second;
            // 3. every group cell complete where the trace reads it (later
            // groups of the wave may evict it again, after its trace)
            for (size_t j = 0; j < gp.cells.size(); ++j) {
                const int c = gp.cells[j];
                const int64_t o = gp.where[j];
                if (o < 0) {
                    ++bad;
                    continue;
                }
                const int64_t node_bytes = (64 * ncnt[c] + CellPlanner::kUnit - 1) / CellPlanner::kUnit *
                                           CellPlanner::kUnit;
                const int64_t n0 = o / 64, n1 = n0 + ncnt[c], t0 = (o + node_bytes) / 48, t1 = t0 + tcnt[c];
                std::set<int> got;
                std::vector<int> stack = {root[c]};
                bad += root[c] != n0;
                while (!stack.empty()) {
                    const int nd = stack.back();
                    stack.pop_back();
                    if (nd < n0 || nd >= n1) {
                        ++bad;
                        break;
                    }
                    const float4 n3 = cache[4 * (size_t)nd + 3];
                    for (int ch : {as_int(n3.x), as_int(n3.y)}) {
                        if (ch >= 0) {
                            stack.push_back(ch);
                            continue;
                        }
                        const int v = ~ch, first = v >> kLeafBits, cnt = v & ((1 << kLeafBits) - 1);
                        for (int i = 0; i < cnt; ++i) {
                            if (first + i < t0 || first + i >= t1) {
                                ++bad;
                                continue;
                            }
                            got.insert(as_int(cache[3 * (size_t)(first + i)].w));
                        }
                    }
                }
                bad += got != members[c];
            }
        }
        bad += at != want;
    }
    std::printf("cache planner: %d cells, budget %lld of %lld bytes, %lld loads, %lld hits over 60 waves; "
                "violations %lld\n", nc, (long long)budget, (long long)total, (long long)loads, (long long)pl.hits,
                (long long)bad);
    return bad ? 1 : 0;
}
