// Host check of the BVH builder (bvh_build.cpp), run by tests/test_host_bvh_cpu.py:
//  1. the global BVH holds every triangle once, in leaves of at most leaf_size;
//  2. its closest hit along random rays equals brute force over the triangles
//     (an FP64 walk of the packed nodes, whose padded boxes must not cull a hit);
//  3. the grid build references, in every cell, each triangle that has a point
//     inside that cell (points sampled on the triangle).
// Prints one line per check and exits non-zero on the first failure.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <set>
#include <string>
#include <vector>

#include "sddm_internal.h"

namespace sddm {
void set_error(const std::string &) {}
}
using namespace sddm;

static int as_int(float f) {
    int i;
    std::memcpy(&i, &f, 4);
    return i;
}

static double hit_t(const double o[3], const double d[3], const BuildTri &t) {
    double e1[3], e2[3], s[3], p[3], q[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = (double)t.v[1][a] - t.v[0][a];
        e2[a] = (double)t.v[2][a] - t.v[0][a];
        s[a] = o[a] - t.v[0][a];
    }
    p[0] = d[1] * e2[2] - d[2] * e2[1];
    p[1] = d[2] * e2[0] - d[0] * e2[2];
    p[2] = d[0] * e2[1] - d[1] * e2[0];
    const double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
    if (std::fabs(det) < 1e-15) return INFINITY;
    const double u = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) / det;
    if (u < 0.0 || u > 1.0) return INFINITY;
    q[0] = s[1] * e1[2] - s[2] * e1[1];
    q[1] = s[2] * e1[0] - s[0] * e1[2];
    q[2] = s[0] * e1[1] - s[1] * e1[0];
    const double v = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) / det;
    if (v < 0.0 || u + v > 1.0) return INFINITY;
    const double t_ = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) / det;
    return t_ > 1e-9 ? t_ : INFINITY;
}

static bool box_hit(const double o[3], const double d[3], const float lo[3], const float hi[3], double tmax) {
    double t0 = 0.0, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        const double inv = 1.0 / d[a];
        double ta = (lo[a] - o[a]) * inv, tb = (hi[a] - o[a]) * inv;
        t0 = std::max(t0, std::min(ta, tb));
        t1 = std::min(t1, std::max(ta, tb));
    }
    return t0 <= t1;
}

int main() {
    std::mt19937 g(7);
    std::uniform_real_distribution<float> U(0.f, 1.f);
    const int nt = 3000, leaf = 4;
    std::vector<BuildTri> tris(nt);
    for (int i = 0; i < nt; ++i) {
        float c[3] = {U(g) * 4, U(g) * 3, U(g) * 2};
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) tris[i].v[k][a] = c[a] + (U(g) - 0.5f) * 0.5f;
        tris[i].id = (uint32_t)i;
        tris[i].obj = (uint32_t)i;
        tris[i].flags = 0;
    }
    std::vector<uint32_t> ids(nt);
    for (int i = 0; i < nt; ++i) ids[i] = (uint32_t)i;
    const float lo[3] = {-0.5f, -0.5f, -0.5f}, hi[3] = {4.5f, 3.5f, 2.5f};
    PackedBVH b;
    build_bvh(tris, ids, lo, hi, leaf, 16, b);

    // 1. every triangle once, leaves within the size limit
    std::vector<int> seen(nt, 0);
    int bad_leaf = 0;
    for (size_t n = 0; n < b.nodes.size() / 4; ++n)
        for (int c = 0; c < 2; ++c) {
            const int ref = as_int(c ? b.nodes[4 * n + 3].y : b.nodes[4 * n + 3].x);
            if (ref >= 0) continue;
            const int v = ~ref, first = v >> kLeafBits, count = v & ((1 << kLeafBits) - 1);
            if (count > leaf && count > kMaxLeaf) ++bad_leaf;
            for (int i = 0; i < count; ++i) ++seen[as_int(b.tris[3 * (first + i)].w)];
        }
    int wrong = 0;
    for (int i = 0; i < nt; ++i) wrong += seen[i] != 1;
    std::printf("triangles referenced once: %d of %d wrong, oversized leaves %d\n", wrong, nt, bad_leaf);
    if (wrong || bad_leaf) return 1;
    // packed triangles carry their three vertices bit for bit (the watertight
    // test needs the endpoints a shared edge has in both of its triangles)
    int moved = 0;
    for (size_t k = 0; k < b.tris.size(); k += 3) {
        const BuildTri &t = tris[as_int(b.tris[k].w)];
        for (int v = 0; v < 3; ++v) {
            const float4 &p = b.tris[k + v];
            moved += p.x != t.v[v][0] || p.y != t.v[v][1] || p.z != t.v[v][2];
        }
    }
    std::printf("packed vertices differing from the input: %d\n", moved);
    if (moved) return 1;

    // 2. closest hits through the packed BVH equal brute force
    int mism = 0;
    for (int r = 0; r < 3000; ++r) {
        double o[3] = {U(g) * 4.0, U(g) * 3.0, U(g) * 2.0}, d[3] = {U(g) - 0.5, U(g) - 0.5, U(g) - 0.5};
        const double nrm = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (double &x : d) x /= nrm;
        double best = INFINITY;
        for (const BuildTri &t : tris) best = std::min(best, hit_t(o, d, t));
        double got = INFINITY;
        std::vector<int> stack = {0};
        while (!stack.empty()) {
            const int node = stack.back();
            stack.pop_back();
            const float4 *p = &b.nodes[4 * (size_t)node];
            const float blo[2][3] = {{p[0].x, p[0].z, p[2].x}, {p[1].x, p[1].z, p[2].z}};
            const float bhi[2][3] = {{p[0].y, p[0].w, p[2].y}, {p[1].y, p[1].w, p[2].w}};
            for (int c = 0; c < 2; ++c) {
                if (!box_hit(o, d, blo[c], bhi[c], got)) continue;
                const int ref = as_int(c ? p[3].y : p[3].x);
                if (ref >= 0) {
                    stack.push_back(ref);
                    continue;
                }
                const int v = ~ref, first = v >> kLeafBits, count = v & ((1 << kLeafBits) - 1);
                for (int i = 0; i < count; ++i)
                    got = std::min(got, hit_t(o, d, tris[as_int(b.tris[3 * (first + i)].w)]));
            }
        }
        if (!((std::isinf(best) && std::isinf(got)) || std::fabs(best - got) <= 1e-12 * std::max(1.0, best))) ++mism;
    }
    std::printf("closest hits differing from brute force: %d of 3000\n", mism);
    if (mism) return 1;

    // 3. grid membership
    const int dims[3] = {3, 2, 2};
    std::vector<PackedBVH> cells;
    build_grid(tris, dims, lo, hi, leaf, 16, 1e-6f, cells, 2);
    std::vector<std::set<int>> members(cells.size());
    for (size_t c = 0; c < cells.size(); ++c)
        for (size_t k = 0; k < cells[c].tris.size(); k += 3) members[c].insert(as_int(cells[c].tris[k].w));
    int missing = 0;
    for (int i = 0; i < nt; ++i) {
        const BuildTri &t = tris[i];
        for (int s = 0; s < 64; ++s) {
            float a = U(g), bb = U(g);
            if (a + bb > 1.f) {
                a = 1.f - a;
                bb = 1.f - bb;
            }
            float x[3];
            for (int q = 0; q < 3; ++q)
                x[q] = t.v[0][q] + a * (t.v[1][q] - t.v[0][q]) + bb * (t.v[2][q] - t.v[0][q]);
            int ci[3];
            for (int q = 0; q < 3; ++q)
                ci[q] = std::min(dims[q] - 1, std::max(0, (int)std::floor((x[q] - lo[q]) / ((hi[q] - lo[q]) / dims[q]))));
            const int cell = (ci[2] * dims[1] + ci[1]) * dims[0] + ci[0];
            if (!members[cell].count(i)) ++missing;
        }
    }
    std::printf("sampled triangle points whose cell lacks the triangle: %d\n", missing);
    return missing ? 1 : 0;
}
