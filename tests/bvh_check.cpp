// bvh_check.cpp -- CPU check of the tracer's BVH build (paper_2501_13382_gb300/csrc/bvh_build.h).
//
// Reads n triangles (int64 n, then n * 9 doubles: v0, v1, v2) from the file named on the
// command line, gives each the padded FP32 box the library gives it at scene creation,
// builds the hierarchy and checks what the traversal relies on:
//   - the leaf entries are a permutation of the triangles, each met exactly once;
//   - every leaf holds 1 .. kBvhLeaf triangles, every inner node is reached once;
//   - each child box stored in a node is exactly the union of its triangles' boxes;
//   - the depth leaves room in the kBvhStack-entry traversal stack.
// Prints "OK nodes=<n> depth=<d>" or "FAIL: <reason>" (exit status 1).
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <vector>

#include "bvh_build.h"

using namespace gbt;

static std::vector<float> tbox;
static std::vector<int> seen_entry, seen_node;
static const BvhBuilder *B = nullptr;
static const char *problem = nullptr;
static int max_leaf_depth = 0;

static void unite(float *box, const float *b)
{
    for (int a = 0; a < 3; ++a) {
        box[a] = std::min(box[a], b[a]);
        box[3 + a] = std::max(box[3 + a], b[3 + a]);
    }
}

// Union of the triangle boxes under `ref` (depth of ref), checking the subtree.
static void walk(int32_t ref, int depth, float *box)
{
    for (int a = 0; a < 3; ++a) { box[a] = INFINITY; box[3 + a] = -INFINITY; }
    if (ref < 0) {
        const int32_t v = -(ref + 1);
        const int32_t first = v >> 3, count = (v & 7) + 1;
        if (count < 1 || count > kBvhLeaf) { problem = "leaf size out of range"; return; }
        if (first < 0 || first + count > (int32_t)B->perm.size()) { problem = "leaf outside the permutation"; return; }
        max_leaf_depth = std::max(max_leaf_depth, depth);
        for (int e = first; e < first + count; ++e) {
            if (seen_entry[e]++) { problem = "leaf entry met twice"; return; }
            unite(box, &tbox[6 * (size_t)B->perm[e]]);
        }
        return;
    }
    if (ref >= (int32_t)B->nodes.size()) { problem = "node index out of range"; return; }
    if (seen_node[ref]++) { problem = "inner node reached twice"; return; }
    const BvhNode &nd = B->nodes[ref];
    for (int c = 0; c < 2; ++c) {
        if (nd.ref[c] == kBvhNone) {
            if (ref != 0 || c != 1 || B->perm.size() > (size_t)kBvhLeaf) { problem = "missing child"; return; }
            continue;
        }
        float sub[6];
        walk(nd.ref[c], depth + 1, sub);
        if (problem) return;
        for (int a = 0; a < 6; ++a)
            if (nd.box[c][a] != sub[a]) { problem = "child box is not the union of its triangles' boxes"; return; }
        unite(box, sub);
    }
}

int main(int argc, char **argv)
{
    if (argc != 2) { fprintf(stderr, "usage: bvh_check <triangles.bin>\n"); return 2; }
    FILE *f = fopen(argv[1], "rb");
    if (!f) { fprintf(stderr, "cannot open %s\n", argv[1]); return 2; }
    int64_t n = 0;
    if (fread(&n, sizeof(n), 1, f) != 1 || n < 1) { fprintf(stderr, "bad header\n"); return 2; }
    std::vector<double> xyz((size_t)n * 9);
    if (fread(xyz.data(), sizeof(double), xyz.size(), f) != xyz.size()) { fprintf(stderr, "short file\n"); return 2; }
    fclose(f);
    // the padded FP32 box of each triangle, as at scene creation
    tbox.resize((size_t)n * 6);
    for (int64_t k = 0; k < n; ++k) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int v = 0; v < 3; ++v)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], xyz[9 * k + 3 * v + a]);
                hi[a] = std::max(hi[a], xyz[9 * k + 3 * v + a]);
            }
        for (int a = 0; a < 3; ++a) {
            const double pad = 1e-3 + 2e-6 * std::max(fabs(lo[a]), fabs(hi[a]));
            tbox[6 * k + a] = nextafterf((float)(lo[a] - pad), -INFINITY);
            tbox[6 * k + 3 + a] = nextafterf((float)(hi[a] + pad), INFINITY);
        }
    }
    BvhBuilder bb(xyz.data(), tbox, n);
    bb.run();
    B = &bb;
    std::vector<int> check(n, 0);
    for (int32_t k : bb.perm) {
        if (k < 0 || k >= n || check[k]++) { printf("FAIL: leaf entries are not a permutation\n"); return 1; }
    }
    seen_entry.assign(n, 0);
    seen_node.assign(bb.nodes.size(), 0);
    float root[6];
    walk(0, 0, root);
    if (!problem) {
        for (int64_t e = 0; e < n; ++e)
            if (seen_entry[e] != 1) { problem = "a leaf entry is never reached"; break; }
        for (size_t i = 0; i < bb.nodes.size() && !problem; ++i)
            if (seen_node[i] != 1) problem = "an inner node is never reached";
    }
    if (!problem && max_leaf_depth > bb.depth_max) problem = "leaf deeper than the recorded depth";
    if (!problem && bb.depth_max + 2 > kBvhStack) problem = "depth exceeds the traversal stack";
    if (problem) { printf("FAIL: %s\n", problem); return 1; }
    printf("OK nodes=%zu depth=%d\n", bb.nodes.size(), bb.depth_max);
    return 0;
}
