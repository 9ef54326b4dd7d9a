// trace.cu -- FP64 ray-fan tracer: the RT process of Sec. 3.1 (rays and their
// specular interactions with triangular facets, Sec. 2), with the fan of
// take-off directions of Sec. 3.3.
//
// This translation unit is compiled with --fmad=false: every FP64 product and
// sum is rounded on its own, in the order written, so hit sequences are
// reproducible bit for bit by any IEEE-754 implementation of the same steps.
//
// Layout on the GB300: one thread per ray; persistent warps take strips of 32
// rays and trace each to its end.  Nearest hits come from a BVH of padded FP32
// boxes read through L1/L2 (the default), or from the triangles tested in index
// order out of shared memory (whole scene resident up to 1,024 triangles, in
// chunks above).  The per-ray segments go to padded slots ray * (R+1) + depth,
// then an exclusive scan of the per-ray counts gives the CSR offsets and a
// compaction kernel writes the flat segment list.  No host synchronisation is
// needed: the segment count stays on the device (ray_off[n_rays]).
#include <math.h>

#include <algorithm>

#include "gbt_internal.h"

namespace gbt {
namespace {

constexpr int kTraceBlock = 256;
constexpr int kTriChunk = 1024;         // most triangles per shared-memory chunk (scene resident up to this)
static_assert(kTriChunk % kTriCluster == 0, "chunks hold whole clusters");
constexpr int kScanBlock = 1024;        // threads per scan block
constexpr int kScanItems = 4;           // items per scan thread

__global__ void scene_prep_kernel(const double *__restrict__ raw, int64_t n,
                                  double *__restrict__ tri, float *__restrict__ trif)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double *v = raw + 9 * k;
    double *o = tri + 12 * k;
    double e1x = v[3] - v[0], e1y = v[4] - v[1], e1z = v[5] - v[2];
    double e2x = v[6] - v[0], e2y = v[7] - v[1], e2z = v[8] - v[2];
    double nx = e1y * e2z - e1z * e2y;
    double ny = e1z * e2x - e1x * e2z;
    double nz = e1x * e2y - e1y * e2x;
    double len = sqrt(nx * nx + ny * ny + nz * nz);
    o[0] = v[0]; o[1] = v[1]; o[2] = v[2];
    o[3] = e1x; o[4] = e1y; o[5] = e1z;
    o[6] = e2x; o[7] = e2y; o[8] = e2z;
    o[9] = nx / len; o[10] = ny / len; o[11] = nz / len;
    float *f = trif + 9 * k;
    for (int q = 0; q < 9; ++q) f[q] = (float)o[q];
}

struct TraceParams {
    double src[3];
    int64_t n_fan, ray_begin, n_rays;
    const double *dirs;        // explicit directions (n_rays * 3) or nullptr
    FanDev fan;                // generated fan when dirs is nullptr
    int max_refl;
    double max_path;
    int ground;
    double ground_z;
    int ground_mat;
    const double *tri;         // n_tri * 12
    const float *trif;         // n_tri * 9 (v0, e1, e2 in FP32)
    const int32_t *face;
    const int32_t *mat;
    int64_t n_tri;
    const float *cbox;         // n_clusters * 6
    const float *tbox;         // n_tri * 6
    int64_t n_clusters;
    const BvhNode *bvh;        // BVH nodes (root 0) or nullptr
    const int32_t *bvh_perm;
    unsigned int *status;
    int chunk;                 // triangles per shared-memory chunk (a multiple of kTriCluster)
    int64_t strip;             // Fibonacci fan: lattice step between a warp's rays (0: none)
    unsigned long long *counter;   // resident scene: next strip of 32 ray slots (zeroed)
    int64_t stride;            // max_refl + 1
    double *po, *pt, *pL, *ps0;
    int32_t *pbmat, *phit, *cnt;
};

// Moller-Trumbore test against a triangle given as v0, e1, e2 (12-double record);
// returns t or -1.  Same operation order as a plain C evaluation of
//   p = d x e2; det = e1.p; u = (o - v0).p / det; q = (o - v0) x e1;
//   v = d.q / det; t = e2.q / det  with inclusive barycentric bounds.
__device__ __forceinline__ double ray_triangle(const double o[3], const double d[3],
                                               const double *__restrict__ r)
{
    const double e1x = r[3], e1y = r[4], e1z = r[5];
    const double e2x = r[6], e2y = r[7], e2z = r[8];
    double px = d[1] * e2z - d[2] * e2y;
    double py = d[2] * e2x - d[0] * e2z;
    double pz = d[0] * e2y - d[1] * e2x;
    double det = e1x * px + e1y * py + e1z * pz;
    if (det == 0.0) return -1.0;
    double inv = 1.0 / det;
    double tx = o[0] - r[0], ty = o[1] - r[1], tz = o[2] - r[2];
    double u = (tx * px + ty * py + tz * pz) * inv;
    if (u < 0.0 || u > 1.0) return -1.0;
    double qx = ty * e1z - tz * e1y;
    double qy = tz * e1x - tx * e1z;
    double qz = tx * e1y - ty * e1x;
    double v = (d[0] * qx + d[1] * qy + d[2] * qz) * inv;
    if (v < 0.0 || u + v > 1.0) return -1.0;
    return (e2x * qx + e2y * qy + e2z * qz) * inv;
}

// One axis of a ray/box slab test: narrows [tn, tf]; false when the ray is parallel to
// the slab and outside it.
// In FP32: the boxes are padded by 1 mm + 2e-6 relative, far more than the rounding
// of these few operations at scene scale, so a box the exact ray meets is never missed.
__device__ __forceinline__ bool slab(float o, float d, float inv, float lo, float hi, float &tn,
                                     float &tf)
{
    if (d == 0.0f) return !(o < lo || o > hi);
    float t1 = (lo - o) * inv, t2 = (hi - o) * inv;
    if (t1 > t2) { const float tt = t1; t1 = t2; t2 = tt; }
    tn = fmaxf(tn, t1);
    tf = fminf(tf, t2);
    return true;
}

__device__ __forceinline__ void load_tri_chunk(double *st, float *sbox, float *stbox,
                                               int32_t *sface, const TraceParams &p, int64_t base,
                                               int count)
{
    for (int idx = threadIdx.x; idx < count * 12; idx += blockDim.x)
        st[idx] = p.tri[base * 12 + idx];
    for (int idx = threadIdx.x; idx < count * 6; idx += blockDim.x)
        stbox[idx] = p.tbox[base * 6 + idx];
    const int c0 = (int)(base / kTriCluster), nc = (count + kTriCluster - 1) / kTriCluster;
    for (int idx = threadIdx.x; idx < nc * 6; idx += blockDim.x)
        sbox[idx] = p.cbox[(int64_t)c0 * 6 + idx];
    for (int idx = threadIdx.x; idx < count; idx += blockDim.x)
        sface[idx] = p.face ? p.face[base + idx] : (int32_t)(base + idx);
}

// Ray index of thread slot tid.  On the Fibonacci lattice ray g and ray g + F (F a
// Fibonacci number near sqrt(N)) are neighbours, so a warp takes rays i0, i0 + F, ...,
// i0 + 31 F: the 32 x F index blocks are read transposed and a warp's rays meet the
// same boxes and triangles.  Outputs stay at each ray's own index; the tail past whole
// blocks keeps its order.
__device__ __forceinline__ int64_t ray_of_slot(const TraceParams &p, int64_t tid)
{
    if (p.strip > 0) {
        const int64_t blk = 32 * p.strip;
        if (tid < p.n_rays / blk * blk) {
            const int64_t r = tid % blk;
            return tid - r + (r & 31) * p.strip + (r >> 5);
        }
    }
    return tid;
}

// Take-off direction of ray i (explicit, or the generated fan of the whole source:
// the lat-long grid's cell centre, or the Fibonacci lattice).
__device__ __forceinline__ void ray_direction(const TraceParams &p, int64_t i, double d[3])
{
    if (p.dirs) {
        d[0] = p.dirs[3 * i]; d[1] = p.dirs[3 * i + 1]; d[2] = p.dirs[3 * i + 2];
    } else if (p.fan.kind == GBT_FAN_LATLONG) {
        const int64_t g = p.ray_begin + i;
        const int64_t it = g / p.fan.n_phi, ip = g - it * p.fan.n_phi;
        const double th = p.fan.th0 + ((double)it + 0.5) * p.fan.dth;
        const double ph = p.fan.ph0 + ((double)ip + 0.5) * p.fan.dph;
        d[0] = sin(th) * cos(ph);
        d[1] = sin(th) * sin(ph);
        d[2] = cos(th);
    } else {
        const int64_t g = p.ray_begin + i;
        const double golden = kPi * (3.0 - sqrt(5.0));
        double z = 1.0 - (2.0 * (double)g + 1.0) / (double)p.n_fan;
        double r = sqrt(1.0 - z * z);
        double phi = (double)g * golden;
        d[0] = r * cos(phi);
        d[1] = r * sin(phi);
        d[2] = z;
    }
}

// Nearest hit among the triangles of one staged chunk (base .. base + count), with
// tbest / best carrying the nearest so far.  Clusters in index order; a cluster whose
// (expanded) box the ray misses, or enters only beyond the best hit so far, holds no
// hit that could win, and likewise each triangle's own padded box before its FP64 test.
__device__ __forceinline__ void nearest_in_chunk(const double o[3], const double d[3], int last_face,
                                                 const double *st, const float *stbox,
                                                 const float *sbox, const int32_t *sface,
                                                 int64_t base, int count, double &tbest, int &best)
{
    const float of0 = (float)o[0], of1 = (float)o[1], of2 = (float)o[2];
    const float df0 = (float)d[0], df1 = (float)d[1], df2 = (float)d[2];
    const float id0 = 1.0f / df0, id1 = 1.0f / df1, id2 = 1.0f / df2;
    const int nc = (count + kTriCluster - 1) / kTriCluster;
    for (int c = 0; c < nc; ++c) {
        const float *bx = sbox + 6 * c;
        // upper bound: the best hit so far, widened like the boxes
        float tn = 0.0f, tf = (float)tbest * 1.000001f + 1e-3f;
        bool hit_box = slab(of0, df0, id0, bx[0], bx[3], tn, tf);
        hit_box = hit_box && slab(of1, df1, id1, bx[1], bx[4], tn, tf);
        hit_box = hit_box && slab(of2, df2, id2, bx[2], bx[5], tn, tf);
        if (!hit_box || tn > tf) continue;
        const int k1 = min(count, (c + 1) * kTriCluster);
        for (int k = c * kTriCluster; k < k1; ++k) {
            if (sface[k] == last_face) continue;
            const float *tb = stbox + 6 * k;
            float un = 0.0f, uf = (float)tbest * 1.000001f + 1e-3f;
            bool hit_tri = slab(of0, df0, id0, tb[0], tb[3], un, uf);
            hit_tri = hit_tri && slab(of1, df1, id1, tb[1], tb[4], un, uf);
            hit_tri = hit_tri && slab(of2, df2, id2, tb[2], tb[5], un, uf);
            if (!hit_tri || un > uf) continue;
            double t = ray_triangle(o, d, st + 12 * k);
            if (t > kTMin && t < tbest) { tbest = t; best = (int)(base + k + 1); }
        }
    }
}

// Conservative FP32 screen in front of the exact FP64 test: false only when that test
// is certain to reject the triangle.  With eps = 2^-24 the FP32 rounding of the inputs
// (origin, direction, v0, e1, e2) and of these operations moves u's numerator (o - v0).p
// by at most 9 eps sum_i (|o_i| + |v0_i|) |p|_i, the determinant by 8 eps sum |e1_i| |p|_i
// and v's numerator by 9 eps sum |d_i| |q|_i (|p|_i, |q|_i: the sums of the absolute
// products forming p = d x e2 and q = (o - v0) x e1); the margins below use 1e-5 in place
// of those 9 eps and 8 eps, covering also the rounding of the comparisons and the FP64
// test's own (about 1e-15 relative).  Outside the margins u < 0, u > 1, v < 0 or u + v > 1
// holds in exact arithmetic, and so in FP64; where the determinant's sign is uncertain the
// FP64 test decides.
__device__ __forceinline__ bool tri_may_hit(float of0, float of1, float of2, float df0, float df1,
                                            float df2, const float *__restrict__ f)
{
    const float v0x = f[0], v0y = f[1], v0z = f[2];
    const float e1x = f[3], e1y = f[4], e1z = f[5];
    const float e2x = f[6], e2y = f[7], e2z = f[8];
    const float px = df1 * e2z - df2 * e2y, py = df2 * e2x - df0 * e2z, pz = df0 * e2y - df1 * e2x;
    const float pax = fabsf(df1 * e2z) + fabsf(df2 * e2y), pay = fabsf(df2 * e2x) + fabsf(df0 * e2z),
                paz = fabsf(df0 * e2y) + fabsf(df1 * e2x);
    const float det = e1x * px + e1y * py + e1z * pz;
    const float bd = 1e-5f * (fabsf(e1x) * pax + fabsf(e1y) * pay + fabsf(e1z) * paz) + 1e-30f;
    const float adet = fabsf(det);
    if (!(adet > bd)) return true;
    const float tx = of0 - v0x, ty = of1 - v0y, tz = of2 - v0z;
    const float ax = fabsf(of0) + fabsf(v0x), ay = fabsf(of1) + fabsf(v0y), az = fabsf(of2) + fabsf(v0z);
    const float bu = 1e-5f * (ax * pax + ay * pay + az * paz) + 1e-30f;
    const float sgn = det > 0.0f ? 1.0f : -1.0f;
    const float su = sgn * (tx * px + ty * py + tz * pz);
    if (su < -bu || su - adet > bu + bd) return false;
    const float qx = ty * e1z - tz * e1y, qy = tz * e1x - tx * e1z, qz = tx * e1y - ty * e1x;
    const float qax = ay * fabsf(e1z) + az * fabsf(e1y), qay = az * fabsf(e1x) + ax * fabsf(e1z),
                qaz = ax * fabsf(e1y) + ay * fabsf(e1x);
    const float bv = 1e-5f * (fabsf(df0) * qax + fabsf(df1) * qay + fabsf(df2) * qaz) + 1e-30f;
    const float sv = sgn * (df0 * qx + df1 * qy + df2 * qz);
    if (sv < -bv || su + sv - adet > bu + bv + bd) return false;
    return true;
}

// Nearest hit among all triangles through the BVH.  Same candidates and the same
// winner as testing every triangle in index order: a child whose padded box the ray
// misses, or enters only beyond the best hit so far (widened like the boxes), holds
// no hit that could win; hits are compared by (t, primitive id), so the lowest id
// wins a tie whatever order the leaves are met in.
__device__ __forceinline__ void nearest_in_bvh(const TraceParams &p, const double o[3],
                                               const double d[3], int last_face, double &tbest,
                                               int &best)
{
    const float of0 = (float)o[0], of1 = (float)o[1], of2 = (float)o[2];
    const float df0 = (float)d[0], df1 = (float)d[1], df2 = (float)d[2];
    const float id0 = 1.0f / df0, id1 = 1.0f / df1, id2 = 1.0f / df2;
    int32_t sref[kBvhStack];
    float stn[kBvhStack];
    int sp = 0;
    sref[sp] = 0;
    stn[sp] = 0.0f;
    ++sp;
    while (sp > 0) {
        --sp;
        const int32_t ref = sref[sp];
        const float bound = (float)tbest * 1.000001f + 1e-3f;
        if (stn[sp] > bound) continue;
        if (ref < 0) {
            const int32_t v = -(ref + 1);
            const int32_t first = v >> 3, count = (v & 7) + 1;
            for (int e = first; e < first + count; ++e) {
                const int32_t k = p.bvh_perm[e];
                const int face = p.face ? p.face[k] : k;
                if (face == last_face) continue;
                const float *tb = p.tbox + 6 * (int64_t)k;
                float un = 0.0f, uf = (float)tbest * 1.000001f + 1e-3f;
                bool hit_tri = slab(of0, df0, id0, tb[0], tb[3], un, uf);
                hit_tri = hit_tri && slab(of1, df1, id1, tb[1], tb[4], un, uf);
                hit_tri = hit_tri && slab(of2, df2, id2, tb[2], tb[5], un, uf);
                if (!hit_tri || un > uf) continue;
                if (!tri_may_hit(of0, of1, of2, df0, df1, df2, p.trif + 9 * (int64_t)k)) continue;
                const double t = ray_triangle(o, d, p.tri + 12 * (int64_t)k);
                if (t > kTMin && (t < tbest || (t == tbest && k + 1 < best))) {
                    tbest = t;
                    best = k + 1;
                }
            }
            continue;
        }
        const float4 *nd = reinterpret_cast<const float4 *>(p.bvh + ref);
        const float4 w0 = __ldg(nd), w1 = __ldg(nd + 1), w2 = __ldg(nd + 2), w3 = __ldg(nd + 3);
        const float b0[6] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y};
        const float b1[6] = {w1.z, w1.w, w2.x, w2.y, w2.z, w2.w};
        const int32_t r0 = __float_as_int(w3.x), r1 = __float_as_int(w3.y);
        float tn0 = 0.0f, tf0 = bound, tn1 = 0.0f, tf1 = bound;
        bool h0 = r0 != kBvhNone;
        h0 = h0 && slab(of0, df0, id0, b0[0], b0[3], tn0, tf0);
        h0 = h0 && slab(of1, df1, id1, b0[1], b0[4], tn0, tf0);
        h0 = h0 && slab(of2, df2, id2, b0[2], b0[5], tn0, tf0);
        h0 = h0 && !(tn0 > tf0);
        bool h1 = r1 != kBvhNone;
        h1 = h1 && slab(of0, df0, id0, b1[0], b1[3], tn1, tf1);
        h1 = h1 && slab(of1, df1, id1, b1[1], b1[4], tn1, tf1);
        h1 = h1 && slab(of2, df2, id2, b1[2], b1[5], tn1, tf1);
        h1 = h1 && !(tn1 > tf1);
        // push the farther child first so the nearer one is taken next; the build keeps
        // the depth below kBvhStack - 1, the check only guards the array
        if (sp + 2 > kBvhStack) {
            atomicOr(p.status, STATUS_BOUNDS);
            return;
        }
        if (h0 && h1) {
            const bool near0 = tn0 <= tn1;
            sref[sp] = near0 ? r1 : r0; stn[sp] = near0 ? tn1 : tn0; ++sp;
            sref[sp] = near0 ? r0 : r1; stn[sp] = near0 ? tn0 : tn1; ++sp;
        } else if (h0) {
            sref[sp] = r0; stn[sp] = tn0; ++sp;
        } else if (h1) {
            sref[sp] = r1; stn[sp] = tn1; ++sp;
        }
    }
}

// Ground plane candidate (best 0) before any triangle.
__device__ __forceinline__ void nearest_ground(const TraceParams &p, const double o[3],
                                               const double d[3], int last_face, double &tbest,
                                               int &best)
{
    if (p.ground && last_face != -2 && d[2] != 0.0) {
        double t = (p.ground_z - o[2]) / d[2];
        if (t > kTMin && t < tbest) { tbest = t; best = 0; }
    }
}

// Writes the segment from o along d ending at the nearest hit (or the path limit) and,
// unless the ray ends there, reflects it.  Returns whether the ray continues.
__device__ __forceinline__ bool record_and_reflect(const TraceParams &p, int64_t i, double o[3],
                                                   double d[3], double &s0, int &last_face,
                                                   int &bmat, int &nref, int &nseg, double tbest,
                                                   int best)
{
    const double remaining = p.max_path - s0;
    const int64_t row = i * p.stride + nseg;
    p.po[3 * row + 0] = o[0]; p.po[3 * row + 1] = o[1]; p.po[3 * row + 2] = o[2];
    p.pt[3 * row + 0] = d[0]; p.pt[3 * row + 1] = d[1]; p.pt[3 * row + 2] = d[2];
    p.ps0[row] = s0;
    p.pbmat[row] = bmat;
    ++nseg;
    if (best < 0 || tbest >= remaining) {
        p.pL[row] = remaining;
        p.phit[row] = -1;
        return false;
    }
    p.pL[row] = tbest;
    p.phit[row] = best;
    if (nref == p.max_refl) return false;
    double n0, n1, n2;
    int face, mat;
    if (best == 0) {
        n0 = 0.0; n1 = 0.0; n2 = 1.0;
        face = -2; mat = p.ground_mat;
    } else {
        const int64_t k = best - 1;
        n0 = p.tri[12 * k + 9]; n1 = p.tri[12 * k + 10]; n2 = p.tri[12 * k + 11];
        face = p.face ? p.face[k] : (int)k;
        mat = p.mat[k];
    }
    o[0] = o[0] + tbest * d[0];
    o[1] = o[1] + tbest * d[1];
    o[2] = o[2] + tbest * d[2];
    double dn = d[0] * n0 + d[1] * n1 + d[2] * n2;
    d[0] = d[0] - 2.0 * dn * n0;
    d[1] = d[1] - 2.0 * dn * n1;
    d[2] = d[2] - 2.0 * dn * n2;
    s0 = s0 + tbest;
    last_face = face;
    bmat = mat;
    ++nref;
    return true;
}

// Scene too large for one shared-memory chunk: the block streams the triangle chunks
// for every bounce, so its rays advance bounce by bounce together.
__global__ void __launch_bounds__(kTraceBlock) trace_kernel(TraceParams p)
{
    extern __shared__ double smem[];
    const int chunk = p.chunk;
    double *st = smem;                                              // chunk * 12
    float *stbox = reinterpret_cast<float *>(smem + (size_t)chunk * 12);   // chunk * 6
    float *sbox = stbox + (size_t)chunk * 6;                        // clusters * 6
    int32_t *sface = reinterpret_cast<int32_t *>(sbox + (chunk / kTriCluster) * 6);

    const int64_t i = ray_of_slot(p, blockIdx.x * (int64_t)kTraceBlock + threadIdx.x);
    const bool active = i < p.n_rays;
    double o[3] = {p.src[0], p.src[1], p.src[2]};
    double d[3] = {0.0, 0.0, 1.0};
    if (active) ray_direction(p, i, d);
    double s0 = 0.0;
    int last_face = -1, bmat = -1, nref = 0, nseg = 0;
    bool alive = active;
    const int64_t nchunk = (p.n_tri + chunk - 1) / chunk;
    for (int bounce = 0; bounce <= p.max_refl; ++bounce) {
        double tbest = INFINITY;
        int best = -1;
        if (alive) nearest_ground(p, o, d, last_face, tbest, best);
        for (int64_t c = 0; c < nchunk; ++c) {
            const int64_t base = c * chunk;
            const int count = (int)min((int64_t)chunk, p.n_tri - base);
            __syncthreads();
            load_tri_chunk(st, sbox, stbox, sface, p, base, count);
            __syncthreads();
            if (alive) nearest_in_chunk(o, d, last_face, st, stbox, sbox, sface, base, count, tbest, best);
        }
        if (alive) alive = record_and_reflect(p, i, o, d, s0, last_face, bmat, nref, nseg, tbest, best);
        if (!__syncthreads_or(alive)) break;
    }
    if (active) p.cnt[i] = nseg;
}

// Scene resident in shared memory: after the one load, every warp takes strips of 32
// ray slots from an atomic counter and traces each ray to its end on its own, with no
// block barrier per bounce, so a long ray delays only its own warp.
__global__ void __launch_bounds__(kTraceBlock) trace_resident_kernel(TraceParams p)
{
    extern __shared__ double smem[];
    const int chunk = p.chunk;
    double *st = smem;
    float *stbox = reinterpret_cast<float *>(smem + (size_t)chunk * 12);
    float *sbox = stbox + (size_t)chunk * 6;
    int32_t *sface = reinterpret_cast<int32_t *>(sbox + (chunk / kTriCluster) * 6);
    if (p.n_tri > 0) load_tri_chunk(st, sbox, stbox, sface, p, 0, (int)p.n_tri);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (;;) {
        int64_t q = 0;
        if (lane == 0) q = atomicAdd(p.counter, 1ull);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q * 32 >= p.n_rays) break;
        const int64_t i = ray_of_slot(p, q * 32 + lane);
        if (i >= p.n_rays) continue;
        double o[3] = {p.src[0], p.src[1], p.src[2]};
        double d[3];
        ray_direction(p, i, d);
        double s0 = 0.0;
        int last_face = -1, bmat = -1, nref = 0, nseg = 0;
        for (bool alive = true; alive;) {
            double tbest = INFINITY;
            int best = -1;
            nearest_ground(p, o, d, last_face, tbest, best);
            if (p.n_tri > 0)
                nearest_in_chunk(o, d, last_face, st, stbox, sbox, sface, 0, (int)p.n_tri, tbest, best);
            alive = record_and_reflect(p, i, o, d, s0, last_face, bmat, nref, nseg, tbest, best);
        }
        p.cnt[i] = nseg;
    }
}

// Scene in a BVH (global memory, L2-resident): persistent warps take strips of 32 ray
// slots and trace each ray to its end on its own, like the resident kernel.
__global__ void __launch_bounds__(kTraceBlock) trace_bvh_kernel(TraceParams p)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int64_t q = 0;
        if (lane == 0) q = atomicAdd(p.counter, 1ull);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q * 32 >= p.n_rays) break;
        const int64_t i = ray_of_slot(p, q * 32 + lane);
        if (i >= p.n_rays) continue;
        double o[3] = {p.src[0], p.src[1], p.src[2]};
        double d[3];
        ray_direction(p, i, d);
        double s0 = 0.0;
        int last_face = -1, bmat = -1, nref = 0, nseg = 0;
        for (bool alive = true; alive;) {
            double tbest = INFINITY;
            int best = -1;
            nearest_ground(p, o, d, last_face, tbest, best);
            nearest_in_bvh(p, o, d, last_face, tbest, best);
            alive = record_and_reflect(p, i, o, d, s0, last_face, bmat, nref, nseg, tbest, best);
        }
        p.cnt[i] = nseg;
    }
}

// ---- exclusive scan of per-ray counts (3 phases, deterministic) ----

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    int excl = x - v + (warp > 0 ? warp_sums[warp - 1] : 0);
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    return excl;
}

__global__ void __launch_bounds__(kScanBlock) scan_block_sums(const int32_t *__restrict__ cnt,
                                                              int64_t n, int32_t *__restrict__ bsum)
{
    __shared__ int ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock * kScanItems;
    int local = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + q;
        if (idx < n) local += cnt[idx];
    }
    int tot;
    block_exclusive_scan(local, ws, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanBlock) scan_of_block_sums(int32_t *bsum, int64_t nb)
{
    __shared__ int ws[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        int64_t idx = base + threadIdx.x;
        int v = idx < nb ? bsum[idx] : 0;
        int tot;
        int ex = block_exclusive_scan(v, ws, &tot);
        int c = carry;
        if (idx < nb) bsum[idx] = ex + c;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanBlock) scan_final(const int32_t *__restrict__ cnt, int64_t n,
                                                         const int32_t *__restrict__ bsum,
                                                         int32_t *__restrict__ off)
{
    __shared__ int ws[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock * kScanItems;
    int vals[kScanItems];
    int local = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + q;
        vals[q] = idx < n ? cnt[idx] : 0;
        local += vals[q];
    }
    int tot;
    int ex = block_exclusive_scan(local, ws, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int64_t idx = base + (int64_t)threadIdx.x * kScanItems + q;
        if (idx < n) off[idx] = ex;
        ex += vals[q];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) off[n] = ex;
}

struct CompactParams {
    int64_t n_rays, stride, ray_begin;
    const int32_t *cnt, *off;
    const double *po, *pt, *pL, *ps0;
    const int32_t *pbmat, *phit;
    double *o, *t, *L, *s0;
    int32_t *ray, *depth, *bmat, *hit;
};

__global__ void compact_kernel(CompactParams p)
{
    const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (slot >= p.n_rays * p.stride) return;
    const int64_t i = slot / p.stride;
    const int dep = (int)(slot - i * p.stride);
    if (dep >= p.cnt[i]) return;
    const int64_t j = (int64_t)p.off[i] + dep;
    p.o[3 * j + 0] = p.po[3 * slot + 0];
    p.o[3 * j + 1] = p.po[3 * slot + 1];
    p.o[3 * j + 2] = p.po[3 * slot + 2];
    p.t[3 * j + 0] = p.pt[3 * slot + 0];
    p.t[3 * j + 1] = p.pt[3 * slot + 1];
    p.t[3 * j + 2] = p.pt[3 * slot + 2];
    p.L[j] = p.pL[slot];
    p.s0[j] = p.ps0[slot];
    p.ray[j] = (int32_t)(p.ray_begin + i);
    p.depth[j] = dep;
    p.bmat[j] = p.pbmat[slot];
    p.hit[j] = p.phit[slot];
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__global__ void csr_ray_depth_kernel(const int32_t *__restrict__ off, int64_t n_rays,
                                     int64_t ray_begin, int32_t *__restrict__ ray,
                                     int32_t *__restrict__ depth)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_rays) return;
    for (int32_t j = off[i], d = 0; j < off[i + 1]; ++j, ++d) {
        ray[j] = (int32_t)(ray_begin + i);
        depth[j] = d;
    }
}

}  // namespace

void csr_ray_depth_launch(TraceDev &td, cudaStream_t s)
{
    if (td.n_rays == 0) return;
    csr_ray_depth_kernel<<<(unsigned)((td.n_rays + 255) / 256), 256, 0, s>>>(
        td.ray_off, td.n_rays, td.ray_begin, td.ray, td.depth);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}

void scene_prepare(SceneDev &sd, const double *tri_raw_dev, cudaStream_t s)
{
    if (sd.n_tri == 0) return;
    const int bs = 128;
    scene_prep_kernel<<<(unsigned)((sd.n_tri + bs - 1) / bs), bs, 0, s>>>(tri_raw_dev, sd.n_tri,
                                                                          sd.tri, sd.trif);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}

size_t trace_scratch_bytes(int64_t n_rays, int max_refl)
{
    const size_t cap = (size_t)n_rays * (max_refl + 1);
    const size_t nb = (size_t)((n_rays + kScanBlock * kScanItems - 1) / (kScanBlock * kScanItems));
    size_t b = 0;
    b += align_up(cap * 3 * sizeof(double), 256) * 2;   // po, pt
    b += align_up(cap * sizeof(double), 256) * 2;       // pL, ps0
    b += align_up(cap * sizeof(int32_t), 256) * 2;      // pbmat, phit
    b += align_up((size_t)n_rays * sizeof(int32_t), 256);   // cnt
    b += align_up((nb + 1) * sizeof(int32_t), 256);     // block sums
    b += 256;                                           // strip counter
    return b;
}

void trace_launch(const SceneDev &sd, TraceDev &td, const gbt_source_desc &src, void *scratch,
                  size_t scratch_bytes, cudaStream_t s)
{
    const int64_t n = td.n_rays;
    const int64_t stride = td.max_refl + 1;
    const size_t cap = (size_t)n * stride;
    char *w = static_cast<char *>(scratch);
    auto take = [&](size_t bytes) {
        char *p = w;
        w += align_up(bytes, 256);
        return p;
    };
    TraceParams p{};
    p.src[0] = src.pos[0]; p.src[1] = src.pos[1]; p.src[2] = src.pos[2];
    p.n_fan = td.n_fan;
    p.ray_begin = td.ray_begin;
    p.n_rays = n;
    p.dirs = src.fan == GBT_FAN_EXPLICIT ? src.dirs : nullptr;
    p.fan = td.fan;
    p.max_refl = td.max_refl;
    p.max_path = td.max_path;
    p.ground = sd.ground;
    p.ground_z = sd.ground_z;
    p.ground_mat = sd.ground_material;
    p.tri = sd.tri;
    p.trif = sd.trif;
    p.face = sd.face;
    p.mat = sd.mat;
    p.n_tri = sd.n_tri;
    p.cbox = sd.cbox;
    p.tbox = sd.tbox;
    p.n_clusters = sd.n_clusters;
    p.bvh = sd.bvh;
    p.bvh_perm = sd.bvh_perm;
    p.status = status_word();
    // coherent warps on a Fibonacci fan: the largest Fibonacci number <= sqrt(N) / 2
    p.strip = 0;
    if (!p.dirs && td.fan.kind == GBT_FAN_FIBONACCI && td.n_fan >= 4096) {
        int64_t f0 = 1, f1 = 2;   // lattice neighbours are set by the whole fan's size
        while (f1 * f1 * 4 <= td.n_fan) { const int64_t f2 = f0 + f1; f0 = f1; f1 = f2; }
        p.strip = f0;
    }
    // the whole scene resident in shared memory when it fits one chunk
    const int64_t nt = std::max<int64_t>(sd.n_tri, 1);
    p.chunk = (int)std::min<int64_t>(kTriChunk, (nt + kTriCluster - 1) / kTriCluster * kTriCluster);
    p.stride = stride;
    p.po = reinterpret_cast<double *>(take(cap * 3 * sizeof(double)));
    p.pt = reinterpret_cast<double *>(take(cap * 3 * sizeof(double)));
    p.pL = reinterpret_cast<double *>(take(cap * sizeof(double)));
    p.ps0 = reinterpret_cast<double *>(take(cap * sizeof(double)));
    p.pbmat = reinterpret_cast<int32_t *>(take(cap * sizeof(int32_t)));
    p.phit = reinterpret_cast<int32_t *>(take(cap * sizeof(int32_t)));
    p.cnt = reinterpret_cast<int32_t *>(take((size_t)n * sizeof(int32_t)));
    const int64_t per = (int64_t)kScanBlock * kScanItems;
    const int64_t nb = (n + per - 1) / per;
    int32_t *bsum = reinterpret_cast<int32_t *>(take((size_t)(nb + 1) * sizeof(int32_t)));
    p.counter = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long)));
    if ((size_t)(w - static_cast<char *>(scratch)) > scratch_bytes)
        fail(GBT_ERR_INVALID_ARG, "trace scratch too small");

    auto chunk_smem = [](size_t c) {
        return c * 12 * sizeof(double) + c * 6 * sizeof(float) + (c / kTriCluster) * 6 * sizeof(float) +
               c * sizeof(int32_t);
    };
    const size_t smem = chunk_smem((size_t)p.chunk);
    static bool attr_set = false;
    if (!attr_set) {
        GBT_CUDA(cudaFuncSetAttribute(trace_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)chunk_smem(kTriChunk)));
        GBT_CUDA(cudaFuncSetAttribute(trace_resident_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)chunk_smem(kTriChunk)));
        attr_set = true;
    }
    // the BVH (built unless GBT_ACCEL_LINEAR) outran the shared-memory scene already at
    // 768 triangles: 3.2 ms against 5.4 ms for 1,048,576 rays through the synthetic city
    const bool use_bvh = sd.n_tri > 0 && sd.bvh && sd.accel != GBT_ACCEL_LINEAR;
    if (use_bvh) {
        int per_sm = 0;
        GBT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trace_bvh_kernel, kTraceBlock, 0));
        const int64_t strips = (n + 31) / 32;
        const int64_t blocks = std::max<int64_t>(
            1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * num_sms(),
                                 (strips + kTraceBlock / 32 - 1) / (kTraceBlock / 32)));
        GBT_CUDA(cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), s));
        trace_bvh_kernel<<<(unsigned)blocks, kTraceBlock, 0, s>>>(p);
    } else if (sd.n_tri <= p.chunk) {
        // resident scene: a persistent grid whose warps take strips of rays
        int per_sm = 0;
        GBT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trace_resident_kernel,
                                                               kTraceBlock, smem));
        const int64_t strips = (n + 31) / 32;
        const int64_t blocks = std::max<int64_t>(
            1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * num_sms(),
                                 (strips + kTraceBlock / 32 - 1) / (kTraceBlock / 32)));
        GBT_CUDA(cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), s));
        trace_resident_kernel<<<(unsigned)blocks, kTraceBlock, smem, s>>>(p);
    } else {
        trace_kernel<<<(unsigned)((n + kTraceBlock - 1) / kTraceBlock), kTraceBlock, smem, s>>>(p);
    }
    note_launches(1);
    GBT_CUDA(cudaGetLastError());

    scan_block_sums<<<(unsigned)nb, kScanBlock, 0, s>>>(p.cnt, n, bsum);
    note_launches(1);
    scan_of_block_sums<<<1, kScanBlock, 0, s>>>(bsum, nb);
    note_launches(1);
    scan_final<<<(unsigned)nb, kScanBlock, 0, s>>>(p.cnt, n, bsum, td.ray_off);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());

    CompactParams c{};
    c.n_rays = n; c.stride = stride; c.ray_begin = td.ray_begin;
    c.cnt = p.cnt; c.off = td.ray_off;
    c.po = p.po; c.pt = p.pt; c.pL = p.pL; c.ps0 = p.ps0; c.pbmat = p.pbmat; c.phit = p.phit;
    c.o = td.o; c.t = td.t; c.L = td.L; c.s0 = td.s0;
    c.ray = td.ray; c.depth = td.depth; c.bmat = td.bmat; c.hit = td.hit;
    const int64_t slots = n * stride;
    compact_kernel<<<(unsigned)((slots + 255) / 256), 256, 0, s>>>(c);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}

}  // namespace gbt
