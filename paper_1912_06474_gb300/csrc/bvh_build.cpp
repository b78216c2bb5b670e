// Host construction of the acceleration structures.
//
// Sec. 5 cuts the scene domain into small subdomains; every
// subdomain here gets its own bounding volume hierarchy over the triangles
// that overlap it (duplicated by reference, bounds clipped to the subdomain),
// so tracing inside a subdomain touches only that subdomain's data. A grid of
// one cell gives the global hierarchy used by the classical (pixel-split)
// method.
//
// Hierarchy: binary, binned surface-area heuristic, leaves of at most
// `leaf_size` triangles; node boxes are padded outward so that float slab
// tests never cull a box the ray touches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "sddm_internal.h"

namespace sddm {
namespace {

struct Box {
    float lo[3] = {INFINITY, INFINITY, INFINITY};
    float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void grow(const Box &b) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
        }
    }
    void grow_pt(float x, float y, float z) {
        lo[0] = std::min(lo[0], x); hi[0] = std::max(hi[0], x);
        lo[1] = std::min(lo[1], y); hi[1] = std::max(hi[1], y);
        lo[2] = std::min(lo[2], z); hi[2] = std::max(hi[2], z);
    }
    bool empty() const { return !(lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2]); }
    double area() const {
        if (empty()) return 0.0;
        double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

struct Ref {
    Box b;
    float c[3];
    uint32_t tri;
};

constexpr int kMaxBuildDepth = 60;   // beyond it splits are median splits (bounded tree depth)

class Builder {
   public:
    Builder(const std::vector<BuildTri> &tris, int leaf, int bins, PackedBVH &out)
        : tris_(tris), leaf_(std::max(1, std::min(leaf, kMaxLeaf))), bins_(std::max(4, std::min(bins, 64))),
          out_(out) {}

    void run(std::vector<Ref> &refs) {
        out_.nodes.clear();
        out_.tris.clear();
        refs_ = &refs;
        int n = (int)refs.size();
        Box all;
        for (auto &r : refs) all.grow(r.b);
        // the root is always an interior node at index 0
        out_.nodes.resize(4);
        int child0, child1;
        Box b0, b1;
        int mid = n <= leaf_ ? 0 : split(0, n, 0);
        if ((mid <= 0 || mid >= n) && n > kMaxLeaf) mid = n / 2;
        if (mid <= 0 || mid >= n) {
            child0 = make_leaf(0, n);
            b0 = all;
            child1 = ~0;   // empty leaf (count 0), empty box
        } else {
            for (int i = 0; i < mid; ++i) b0.grow(refs[i].b);
            for (int i = mid; i < n; ++i) b1.grow(refs[i].b);
            child0 = recurse(0, mid, 1);
            child1 = recurse(mid, n, 1);
        }
        write_node(0, b0, b1, child0, child1);
    }

   private:
    const std::vector<BuildTri> &tris_;
    int leaf_, bins_;
    PackedBVH &out_;
    std::vector<Ref> *refs_ = nullptr;

    static void pad(Box &b, float out4[6]) {
        for (int a = 0; a < 3; ++a) {
            if (b.empty()) {   // a point far outside any scene: rays practically never meet it
                out4[2 * a] = 1e30f;
                out4[2 * a + 1] = 1e30f;
                continue;
            }
            float m = std::max(std::fabs(b.lo[a]), std::fabs(b.hi[a]));
            float p = 1e-5f + 2e-6f * m;
            out4[2 * a] = b.lo[a] - p;
            out4[2 * a + 1] = b.hi[a] + p;
        }
    }

    void write_node(int idx, Box b0, Box b1, int c0, int c1) {
        float p0[6], p1[6];
        pad(b0, p0);
        pad(b1, p1);
        float4 *n = &out_.nodes[4 * (size_t)idx];
        n[0] = make_float4(p0[0], p0[1], p0[2], p0[3]);
        n[1] = make_float4(p1[0], p1[1], p1[2], p1[3]);
        n[2] = make_float4(p0[4], p0[5], p1[4], p1[5]);
        float cc0, cc1;
        std::memcpy(&cc0, &c0, 4);
        std::memcpy(&cc1, &c1, 4);
        n[3] = make_float4(cc0, cc1, 0.f, 0.f);
    }

    int make_leaf(int begin, int end) {
        int first = (int)(out_.tris.size() / 3);
        std::vector<Ref> &refs = *refs_;
        for (int i = begin; i < end; ++i) {
            const BuildTri &t = tris_[refs[i].tri];
            float id, ob, fl;
            std::memcpy(&id, &t.id, 4);
            std::memcpy(&ob, &t.obj, 4);
            std::memcpy(&fl, &t.flags, 4);
            out_.tris.push_back(make_float4(t.v[0][0], t.v[0][1], t.v[0][2], id));
            out_.tris.push_back(make_float4(t.v[1][0], t.v[1][1], t.v[1][2], ob));
            out_.tris.push_back(make_float4(t.v[2][0], t.v[2][1], t.v[2][2], fl));
        }
        int count = end - begin;
        return ~((first << kLeafBits) | count);
    }

    int recurse(int begin, int end, int depth) {
        int n = end - begin;
        if (n <= leaf_) return make_leaf(begin, end);
        int mid = split(begin, end, depth);
        if (mid <= begin || mid >= end) {
            if (n <= kMaxLeaf) return make_leaf(begin, end);
            mid = begin + n / 2;
        }
        int idx = (int)(out_.nodes.size() / 4);
        out_.nodes.resize(out_.nodes.size() + 4);
        std::vector<Ref> &refs = *refs_;
        Box b0, b1;
        for (int i = begin; i < mid; ++i) b0.grow(refs[i].b);
        for (int i = mid; i < end; ++i) b1.grow(refs[i].b);
        int c0 = recurse(begin, mid, depth + 1);
        int c1 = recurse(mid, end, depth + 1);
        write_node(idx, b0, b1, c0, c1);
        return idx;
    }

    // Returns the split position after partitioning [begin, end), or begin to
    // request a leaf (only when the range fits in one).
    int split(int begin, int end, int depth) {
        std::vector<Ref> &refs = *refs_;
        int n = end - begin;
        Box cb, nb;
        for (int i = begin; i < end; ++i) {
            cb.grow_pt(refs[i].c[0], refs[i].c[1], refs[i].c[2]);
            nb.grow(refs[i].b);
        }
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (cb.hi[a] - cb.lo[a] > cb.hi[axis] - cb.lo[axis]) axis = a;
        auto median = [&](int ax) {
            int mid = begin + n / 2;
            std::nth_element(refs.begin() + begin, refs.begin() + mid, refs.begin() + end,
                             [ax](const Ref &x, const Ref &y) {
                                 return x.c[ax] < y.c[ax] || (x.c[ax] == y.c[ax] && x.tri < y.tri);
                             });
            return mid;
        };
        if (depth >= kMaxBuildDepth || cb.hi[axis] - cb.lo[axis] <= 0.0f) return median(axis);

        double best_cost = INFINITY;
        int best_axis = -1, best_bin = -1;
        std::vector<Box> bb(bins_);
        std::vector<int> cnt(bins_);
        std::vector<double> right_area(bins_);
        std::vector<int> right_cnt(bins_);
        for (int a = 0; a < 3; ++a) {
            float ext = cb.hi[a] - cb.lo[a];
            if (ext <= 0.0f) continue;
            float scale = bins_ / ext;
            std::fill(bb.begin(), bb.end(), Box());
            std::fill(cnt.begin(), cnt.end(), 0);
            for (int i = begin; i < end; ++i) {
                int k = std::min(bins_ - 1, (int)((refs[i].c[a] - cb.lo[a]) * scale));
                bb[k].grow(refs[i].b);
                cnt[k]++;
            }
            Box acc;
            int c = 0;
            for (int k = bins_ - 1; k > 0; --k) {
                acc.grow(bb[k]);
                c += cnt[k];
                right_area[k] = acc.area();
                right_cnt[k] = c;
            }
            acc = Box();
            c = 0;
            for (int k = 0; k < bins_ - 1; ++k) {
                acc.grow(bb[k]);
                c += cnt[k];
                if (c == 0 || right_cnt[k + 1] == 0) continue;
                double cost = acc.area() * c + right_area[k + 1] * right_cnt[k + 1];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = a;
                    best_bin = k;
                }
            }
        }
        if (best_axis < 0) return median(axis);
        // leaf if splitting does not pay (traversal cost 1, intersection cost 1 per triangle)
        double leaf_cost = (double)n;
        double split_cost = 1.0 + best_cost / std::max(nb.area(), 1e-30);
        if (n <= kMaxLeaf && leaf_cost <= split_cost) return begin;
        float ext = cb.hi[best_axis] - cb.lo[best_axis];
        float scale = bins_ / ext;
        float lo = cb.lo[best_axis];
        int ba = best_axis, bk = best_bin, nbins = bins_;
        auto it = std::partition(refs.begin() + begin, refs.begin() + end, [=](const Ref &r) {
            int k = std::min(nbins - 1, (int)((r.c[ba] - lo) * scale));
            return k <= bk;
        });
        int mid = (int)(it - refs.begin());
        if (mid == begin || mid == end) return median(axis);
        return mid;
    }
};

// Triangle / box overlap by the separating axis theorem (box normals,
// triangle normal, and the nine edge x axis products), in double.
bool tri_box_overlap(const BuildTri &t, const double lo[3], const double hi[3]) {
    double c[3], h[3], v[3][3];
    for (int a = 0; a < 3; ++a) {
        c[a] = 0.5 * (lo[a] + hi[a]);
        h[a] = 0.5 * (hi[a] - lo[a]);
    }
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) v[k][a] = (double)t.v[k][a] - c[a];
    for (int a = 0; a < 3; ++a) {
        double mn = std::min(v[0][a], std::min(v[1][a], v[2][a]));
        double mx = std::max(v[0][a], std::max(v[1][a], v[2][a]));
        if (mn > h[a] || mx < -h[a]) return false;
    }
    double e[3][3];
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) e[k][a] = v[(k + 1) % 3][a] - v[k][a];
    double nrm[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
                     e[0][0] * e[1][1] - e[0][1] * e[1][0]};
    double d = nrm[0] * v[0][0] + nrm[1] * v[0][1] + nrm[2] * v[0][2];
    double r = h[0] * std::fabs(nrm[0]) + h[1] * std::fabs(nrm[1]) + h[2] * std::fabs(nrm[2]);
    if (std::fabs(d) > r) return false;
    for (int k = 0; k < 3; ++k) {
        for (int a = 0; a < 3; ++a) {
            // axis = e_k x unit_a
            double ax[3] = {0, 0, 0};
            double u[3] = {0, 0, 0};
            u[a] = 1.0;
            ax[0] = e[k][1] * u[2] - e[k][2] * u[1];
            ax[1] = e[k][2] * u[0] - e[k][0] * u[2];
            ax[2] = e[k][0] * u[1] - e[k][1] * u[0];
            double p0 = ax[0] * v[0][0] + ax[1] * v[0][1] + ax[2] * v[0][2];
            double p1 = ax[0] * v[1][0] + ax[1] * v[1][1] + ax[2] * v[1][2];
            double p2 = ax[0] * v[2][0] + ax[1] * v[2][1] + ax[2] * v[2][2];
            double mn = std::min(p0, std::min(p1, p2)), mx = std::max(p0, std::max(p1, p2));
            double rr = h[0] * std::fabs(ax[0]) + h[1] * std::fabs(ax[1]) + h[2] * std::fabs(ax[2]);
            if (mn > rr || mx < -rr) return false;
        }
    }
    return true;
}

void make_refs(const std::vector<BuildTri> &tris, const std::vector<uint32_t> &ids, const float clip_lo[3],
               const float clip_hi[3], std::vector<Ref> &refs) {
    refs.clear();
    refs.reserve(ids.size());
    for (uint32_t id : ids) {
        const BuildTri &t = tris[id];
        Ref r;
        for (int k = 0; k < 3; ++k) r.b.grow_pt(t.v[k][0], t.v[k][1], t.v[k][2]);
        for (int a = 0; a < 3; ++a) {
            r.b.lo[a] = std::max(r.b.lo[a], clip_lo[a]);
            r.b.hi[a] = std::min(r.b.hi[a], clip_hi[a]);
            if (r.b.lo[a] > r.b.hi[a]) {   // touches the clip box only within padding
                float m = 0.5f * (r.b.lo[a] + r.b.hi[a]);
                r.b.lo[a] = r.b.hi[a] = m;
            }
            r.c[a] = 0.5f * (r.b.lo[a] + r.b.hi[a]);
        }
        r.tri = id;
        refs.push_back(r);
    }
}

}  // namespace

void build_bvh(const std::vector<BuildTri> &tris, const std::vector<uint32_t> &ids, const float clip_lo[3],
               const float clip_hi[3], int leaf_size, int bins, PackedBVH &out) {
    std::vector<Ref> refs;
    make_refs(tris, ids, clip_lo, clip_hi, refs);
    Builder b(tris, leaf_size, bins, out);
    b.run(refs);
}

void build_grid(const std::vector<BuildTri> &tris, const int dims[3], const float lo[3], const float hi[3],
                int leaf_size, int bins, float eps, std::vector<PackedBVH> &cells, int n_threads) {
    const int nc = dims[0] * dims[1] * dims[2];
    cells.assign(nc, PackedBVH());
    double cell[3], slack[3];
    // a triangle within the hit window's slack eps of a cell must be referenced by it
    for (int a = 0; a < 3; ++a) {
        cell[a] = ((double)hi[a] - (double)lo[a]) / dims[a];
        slack[a] = 1e-5 + 1e-6 * std::max(std::fabs((double)lo[a]), std::fabs((double)hi[a])) + 2.0 * (double)eps;
    }
    // bin triangles into the cells they overlap (cell boxes widened by the slack)
    std::vector<std::vector<uint32_t>> members(nc);
    for (uint32_t id = 0; id < (uint32_t)tris.size(); ++id) {
        const BuildTri &t = tris[id];
        int c0[3], c1[3];
        for (int a = 0; a < 3; ++a) {
            double mn = std::min((double)t.v[0][a], std::min((double)t.v[1][a], (double)t.v[2][a]));
            double mx = std::max((double)t.v[0][a], std::max((double)t.v[1][a], (double)t.v[2][a]));
            c0[a] = std::max(0, std::min(dims[a] - 1, (int)std::floor((mn - slack[a] - lo[a]) / cell[a])));
            c1[a] = std::max(0, std::min(dims[a] - 1, (int)std::floor((mx + slack[a] - lo[a]) / cell[a])));
        }
        for (int z = c0[2]; z <= c1[2]; ++z)
            for (int y = c0[1]; y <= c1[1]; ++y)
                for (int x = c0[0]; x <= c1[0]; ++x) {
                    double blo[3] = {lo[0] + x * cell[0] - slack[0], lo[1] + y * cell[1] - slack[1],
                                     lo[2] + z * cell[2] - slack[2]};
                    double bhi[3] = {lo[0] + (x + 1) * cell[0] + slack[0], lo[1] + (y + 1) * cell[1] + slack[1],
                                     lo[2] + (z + 1) * cell[2] + slack[2]};
                    if (tri_box_overlap(t, blo, bhi)) members[(z * dims[1] + y) * dims[0] + x].push_back(id);
                }
    }
    n_threads = std::max(1, std::min(n_threads, nc));
    std::vector<std::thread> pool;
    std::atomic_int next(0);
    for (int w = 0; w < n_threads; ++w) {
        pool.emplace_back([&]() {
            for (;;) {
                int c = next.fetch_add(1);
                if (c >= nc) break;
                int x = c % dims[0], y = (c / dims[0]) % dims[1], z = c / (dims[0] * dims[1]);
                float clo[3] = {(float)(lo[0] + x * cell[0] - slack[0]), (float)(lo[1] + y * cell[1] - slack[1]),
                                (float)(lo[2] + z * cell[2] - slack[2])};
                float chi[3] = {(float)(lo[0] + (x + 1) * cell[0] + slack[0]),
                                (float)(lo[1] + (y + 1) * cell[1] + slack[1]),
                                (float)(lo[2] + (z + 1) * cell[2] + slack[2])};
                build_bvh(tris, members[c], clo, chi, leaf_size, bins, cells[c]);
            }
        });
    }
    for (auto &t : pool) t.join();
}

}  // namespace sddm
