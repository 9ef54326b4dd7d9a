// bvh_build.h -- host build of the bounding-volume hierarchy over a scene's triangles
// that the tracer walks (trace.cu: nearest_in_bvh).  Host-only C++: the library builds it
// when a scene is created (api.cu), and a CPU test checks its invariants.
#pragma once

#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "gbt_internal.h"

namespace gbt {

// Host build of the triangle BVH.  Splits by a binned surface-area heuristic over
// triangle centroids on the axis of largest centroid extent; below depth kSahDepth,
// or when the centroids coincide, by the median instead, so the depth stays at most
// kSahDepth + 26 (n_tri < 2^26) and the traversal stack of kBvhStack entries suffices.
// Node boxes are unions of the triangles' padded FP32 boxes (exact min / max).
struct BvhBuilder {
    static constexpr int kBins = 16;
    static constexpr int kSahDepth = 32;
    const std::vector<float> &tbox;       // n * 6
    std::vector<double> cen;              // n * 3 centroids
    std::vector<int32_t> perm;
    std::vector<BvhNode> nodes;
    int depth_max = 0;

    BvhBuilder(const double *xyz, const std::vector<float> &tb, int64_t n) : tbox(tb)
    {
        cen.resize((size_t)n * 3);
        perm.resize((size_t)n);
        for (int64_t k = 0; k < n; ++k) {
            perm[k] = (int32_t)k;
            for (int a = 0; a < 3; ++a)
                cen[3 * k + a] = (xyz[9 * k + a] + xyz[9 * k + 3 + a] + xyz[9 * k + 6 + a]) / 3.0;
        }
    }

    void bounds(int64_t lo, int64_t hi, float *box) const
    {
        for (int a = 0; a < 3; ++a) { box[a] = INFINITY; box[3 + a] = -INFINITY; }
        for (int64_t i = lo; i < hi; ++i) {
            const float *b = &tbox[6 * (size_t)perm[i]];
            for (int a = 0; a < 3; ++a) {
                box[a] = std::min(box[a], b[a]);
                box[3 + a] = std::max(box[3 + a], b[3 + a]);
            }
        }
    }

    static double area(const double *lo, const double *hi)
    {
        const double x = hi[0] - lo[0], y = hi[1] - lo[1], z = hi[2] - lo[2];
        return x * y + y * z + z * x;
    }

    // Partition perm[lo, hi) and return the split point (lo < mid < hi).
    int64_t split(int64_t lo, int64_t hi, int depth)
    {
        double cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = lo; i < hi; ++i)
            for (int a = 0; a < 3; ++a) {
                cmin[a] = std::min(cmin[a], cen[3 * (size_t)perm[i] + a]);
                cmax[a] = std::max(cmax[a], cen[3 * (size_t)perm[i] + a]);
            }
        int ax = 0;
        for (int a = 1; a < 3; ++a)
            if (cmax[a] - cmin[a] > cmax[ax] - cmin[ax]) ax = a;
        const double ext = cmax[ax] - cmin[ax];
        const int64_t mid = lo + (hi - lo) / 2;
        if (!(ext > 0.0) || depth >= kSahDepth) {
            std::nth_element(perm.begin() + lo, perm.begin() + mid, perm.begin() + hi,
                             [&](int32_t x, int32_t y) { return cen[3 * (size_t)x + ax] < cen[3 * (size_t)y + ax]; });
            return mid;
        }
        auto bin_of = [&](int32_t k) {
            const int b = (int)((cen[3 * (size_t)k + ax] - cmin[ax]) / ext * kBins);
            return std::min(std::max(b, 0), kBins - 1);
        };
        int64_t cnt[kBins] = {};
        double blo[kBins][3], bhi[kBins][3];
        for (int b = 0; b < kBins; ++b)
            for (int a = 0; a < 3; ++a) { blo[b][a] = INFINITY; bhi[b][a] = -INFINITY; }
        for (int64_t i = lo; i < hi; ++i) {
            const int32_t k = perm[i];
            const int b = bin_of(k);
            ++cnt[b];
            const float *tb = &tbox[6 * (size_t)k];
            for (int a = 0; a < 3; ++a) {
                blo[b][a] = std::min(blo[b][a], (double)tb[a]);
                bhi[b][a] = std::max(bhi[b][a], (double)tb[3 + a]);
            }
        }
        // cost of cutting after bin c: area x count on each side
        double left_cost[kBins];
        double lo3[3] = {INFINITY, INFINITY, INFINITY}, hi3[3] = {-INFINITY, -INFINITY, -INFINITY};
        int64_t nl = 0;
        for (int c = 0; c < kBins - 1; ++c) {
            nl += cnt[c];
            for (int a = 0; a < 3; ++a) { lo3[a] = std::min(lo3[a], blo[c][a]); hi3[a] = std::max(hi3[a], bhi[c][a]); }
            left_cost[c] = nl > 0 ? area(lo3, hi3) * (double)nl : 0.0;
        }
        double best = INFINITY;
        int cut = -1;
        for (int a = 0; a < 3; ++a) { lo3[a] = INFINITY; hi3[a] = -INFINITY; }
        int64_t nr = 0;
        for (int c = kBins - 1; c >= 1; --c) {
            nr += cnt[c];
            for (int a = 0; a < 3; ++a) { lo3[a] = std::min(lo3[a], blo[c][a]); hi3[a] = std::max(hi3[a], bhi[c][a]); }
            const int64_t left = (hi - lo) - nr;
            if (left == 0 || nr == 0) continue;
            const double cost = left_cost[c - 1] + area(lo3, hi3) * (double)nr;
            if (cost < best) { best = cost; cut = c; }
        }
        if (cut < 0) {
            std::nth_element(perm.begin() + lo, perm.begin() + mid, perm.begin() + hi,
                             [&](int32_t x, int32_t y) { return cen[3 * (size_t)x + ax] < cen[3 * (size_t)y + ax]; });
            return mid;
        }
        const auto it = std::stable_partition(perm.begin() + lo, perm.begin() + hi,
                                              [&](int32_t k) { return bin_of(k) < cut; });
        return (int64_t)(it - perm.begin());
    }

    static int32_t leaf_ref(int64_t first, int64_t count)
    {
        return -(int32_t)(first * 8 + (count - 1)) - 1;
    }

    // Reference to the subtree over perm[lo, hi); node boxes are filled by the parent.
    int32_t build(int64_t lo, int64_t hi, int depth)
    {
        depth_max = std::max(depth_max, depth);
        if (hi - lo <= kBvhLeaf) return leaf_ref(lo, hi - lo);
        const int32_t id = (int32_t)nodes.size();
        nodes.push_back(BvhNode{});
        const int64_t mid = split(lo, hi, depth);
        const int32_t l = build(lo, mid, depth + 1);
        const int32_t r = build(mid, hi, depth + 1);
        BvhNode &nd = nodes[id];
        nd.ref[0] = l;
        nd.ref[1] = r;
        bounds(lo, mid, nd.box[0]);
        bounds(mid, hi, nd.box[1]);
        return id;
    }

    void run()
    {
        const int64_t n = (int64_t)perm.size();
        if (n <= kBvhLeaf) {
            // root with one leaf child: the traversal always starts at an inner node
            nodes.push_back(BvhNode{});
            nodes[0].ref[0] = leaf_ref(0, n);
            nodes[0].ref[1] = kBvhNone;
            bounds(0, n, nodes[0].box[0]);
            for (int a = 0; a < 6; ++a) nodes[0].box[1][a] = 0.0f;
            depth_max = 1;
            return;
        }
        build(0, n, 0);
    }
};

}  // namespace gbt
