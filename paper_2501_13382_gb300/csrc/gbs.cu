// gbs.cu -- Gaussian beam summation (Eq. 3 with the beam of Eq. 1 / Eq. 2)
// for every (receiver, segment, frequency) triple, its adjoint, and the
// receiver order they use.
//
// GB300 design of the FP32 pair kernel:
//  * A prepass turns every traced segment into an 80-byte record (origin and
//    start distance as float-float, direction, length, amplitude).
//  * Receivers are visited in Morton order, in warp tiles of 64 (two per lane:
//    receivers lane and lane + 32) held in registers, absolute (exact path) and
//    relative to the warp tile's first receiver (prefilter).
//  * Persistent CTAs of 16 warps, and every warp works on its own: it takes
//    (warp tile, segment split) items from a global queue, split s owning record
//    batches s, s + splits, ...  CTA tiles of 15 warp tiles are dispatched
//    heaviest first and splits are sized for about 16 items per warp, so no warp
//    waits for another and the queue drains on short items.
//  * A warp double-buffers its own 32-record batches (a bulk asynchronous copy
//    completed on a per-warp mbarrier, or per-lane cp.async gathers from the
//    tile's segment list with the pre-cull) and stages each batch itself.  Every
//    wait is bounded and raises a status flag instead of hanging.
//  * Prefilter (every pair, frequency independent): a paired FP32 (f32x2)
//    evaluation of the union of the per-frequency Gaussian cutoffs and the
//    window, conservative by a margin, gives one keep bit per pair.  With the
//    pre-cull, per-tile segment lists with per-entry warp-tile masks and a
//    per-warp ball test skip segments that can reach none of its receivers.
//  * Survivors (typically a few percent of pairs) are evaluated exactly, the two
//    receivers of a lane side by side in paired FP32, in the warp's frame: the
//    staging forms per segment, relative to the warp tile's first receiver c,
//    A = (c - o).t and S = s0 + A in float-float and the compensated
//    N = (c - o) x t, so a receiver at c + x' needs only x'.t (float-float) and
//    N + x' x t; then float-float s and phase (reduced in turns before the MUFU
//    sin/cos).  FP32 sums per lane fold into the item's float-float partials every 16
//    batches, and the per-split partials are merged in float-float (error-free
//    FP32 sums) in a fixed order by a second kernel, so results do not depend on
//    scheduling.
//  * The kernel holds the sums of up to 8 frequencies in registers; more (up to 16)
//    run as one launch per group of 8, each with its own partials and output rows.

#include <math.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>
#include <cmath>
#include <string>

#include "gbt_internal.h"

namespace gbt {
namespace {

constexpr int kWarpsFwd = 16;               // warps per CTA of the pair kernel (one CTA per SM)
constexpr size_t kSmemBudget = 227 * 1024;  // dynamic shared memory of one pair-kernel CTA (the maximum)
constexpr int kWRaw = 2;                    // raw record buffers per warp (double buffering)
constexpr int kR = 2;                       // receivers per lane
constexpr int kWarpRecv = 32 * kR;          // receivers per warp tile
constexpr int kTileWarps = 15;              // warp tiles per CTA tile (dispatch order, lists)
constexpr int kChunkWords = 16;             // warp-tile words per 32-entry chunk of a tile list
constexpr int kCtaRecv = kTileWarps * kWarpRecv;
constexpr int kBatch = 32;                  // segments per staged batch
constexpr long long kSpinLimit = 1LL << 22; // bounded mbarrier waits
enum { kFwd = 0, kStats = 1, kBwd = 2 };    // what the pair kernel does with survivors
constexpr int kFoldEvery = 16;              // batches between float-float folds
constexpr float kWinMargin = 0.01f;         // prefilter window slack (m)
// A warp item takes the FP32 local projection x'.t (instead of float-float) when
// K_max max|x'| <= kFastTurns.  Its rounding, at most about 3 ulp of |x'|, moves a term's
// phase by at most 3 x 2^-24 x 90 turns = 1.0e-4 rad; the roundings of different terms are
// independent, so the field moves far less (2e-7 relative on the city, 3.5e-5 with the
// projection in FP32 everywhere at 4 kHz).  The window test is a hard cutoff, so a pair
// within the FP32 projection's error bound of an end of its window is decided and
// evaluated with the float-float projection.  On that path n = N + x' x t also leaves out
// the products of the lo parts (about 1.3 ulp of |x'|; with |n| <= s the phase moves by
// at most K x 1.3 ulp(|x'|) <= 9e-5 rad).  Past the limit the float-float products stay.
constexpr float kFastTurns = 90.0f;

// Per-frequency constants, grouped in 16-byte words in the order the survivor
// path needs them (cutoff test, then the beam), so a kernel that reads them from
// shared memory (the batched launch) needs two vector loads per kept frequency.
struct alignas(16) FreqConst {
    float kb2;            // k b / 2  (Gaussian exponent factor)
    float b2;             // b^2
    float K_hi, K_lo;     // f / c in turns per metre, float-float
    float halfK;          // K / 2: second phase term K n^2 s / (2 D) in turns
    float kb2l2e;         // k b / 2 * log2(e)
    float scale;          // k b / (8 pi^2)
    float b;              // b
    float kh, invb;       // k / 2, 1 / b  (adjoint)
    float al2e;           // amplitude decay rate of air a (Np/m) * log2(e), 0 when lossless
    float pad1;
};
static_assert(sizeof(FreqConst) == 48, "three 16-byte words");

struct alignas(16) FwdParams {
    const float *recv;
    const int32_t *order;
    int64_t n_recv;
    const int32_t *n_seg_ptr;
    const float *rec;          // AoS records, kRecFloats per segment
    const float4 *crec;        // cull records: (o_hi, s0_hi), (t_hi, L_hi) per segment
    int nf;
    int uniform_b;             // all b equal: frequencies sorted by k, loop stops at first cull
    int tile_cull;             // skip segments that reach none of a warp's receivers
    float cutoff;
    float pre_alpha, pre_beta; // prefilter: keep iff alpha n^2 <= s^2 + beta
    float kmax_turns;          // largest f / c of the launch's frequencies, turns per metre
    int splits;
    int64_t n_items;           // CTA tiles x splits
    int *work_counter;         // zeroed before launch; CTAs take items from it
    const int32_t *tile_perm;  // dispatch rank -> CTA tile (heaviest first), or null
    // tile pre-cull: per CTA tile, the segments whose beams can reach its receivers
    const int32_t *list;       // segment indices, each tile's in segment order, or null
    const int64_t *list_off;   // per tile: first entry in list
    const int32_t *list_n;     // per tile: entries, or -1 (no list: stream every segment)
    // per 32-entry chunk of a tile's list (every list starts on a chunk boundary), one
    // word per warp tile w: bit b set if entry b of the chunk can reach warp tile w
    const uint32_t *list_words;
    float4 *partial;           // [splits][nf][n_recv]: re_hi, im_hi, re_lo, im_lo
    unsigned long long *stats; // counting mode when non-null: [1] prefiltered, [2] kept
    unsigned int *status;      // device status word (timeouts)
    // adjoint mode
    const float2 *grad_out;    // g = dL/dRe p + i dL/dIm p, [user frequency][n_recv]
    float *seg_G;              // per segment: sum over (r, f) of Re(conj(g) c~)
    float *seg_H;              // per (sorted frequency, segment): sum over r of Re(conj(g) dc~/db)
    int64_t seg_stride;        // stride of seg_H rows
    int fperm[GBT_MAX_FREQ];   // sorted frequency slot -> user frequency index
    // losses of porous surfaces (lossy instantiation): per user frequency f and segment j,
    // seg_rf[f * rf_stride + j] = (log2 |R|, arg R / 2 pi) of the path's reflection factor
    const float2 *seg_rf;
    int64_t rf_stride;
    // batched launch: per-instance parameters and the first global item of each
    const struct FwdParams *inst;
    const int64_t *inst_off;   // n_inst + 1 entries
    int n_inst;
    FreqConst fc[GBT_MAX_FREQ];
};

static_assert(sizeof(FwdParams) % 16 == 0, "instance parameters are copied as 16-byte words");

// Error-free transformations depend on every operation being rounded as written:
// nvcc contracts a product feeding an add into one FMA by default, which would
// round differently in each inlined copy.  The __f*_rn intrinsics are never
// contracted, so these sites use them wherever a rounding is relied upon.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Kahan's difference of products a*b - c*d, accurate to about one ulp.
__device__ __forceinline__ float dop(float a, float b, float c, float d)
{
    const float w = __fmul_rn(c, d);
    const float e = fmaf(-c, d, w);
    const float f = fmaf(a, b, -w);
    return f + e;
}

typedef unsigned long long f2x;   // two packed floats (lo = receiver 0, hi = receiver 1)
__device__ __forceinline__ f2x pk(float a, float b)
{
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2x v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c)
{
    f2x r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2x add2(f2x a, f2x b)
{
    f2x r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b)
{
    f2x r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b)
{
    f2x r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x neg2(f2x a) { return mul2(a, 0xbf800000bf800000ull); }
__device__ __forceinline__ f2x splat(float a) { return pk(a, a); }
// two_sum on both halves; the paired operations round each half exactly like the
// scalar ones, so both paths give identical results
__device__ __forceinline__ void two_sum2(f2x a, f2x b, f2x &s, f2x &e)
{
    s = add2(a, b);
    const f2x bv = sub2(s, a);
    e = add2(sub2(a, sub2(s, bv)), sub2(b, bv));
}
__device__ __forceinline__ f2x rint2(f2x a)
{
    float x, y;
    upk(a, x, y);
    return pk(rintf(x), rintf(y));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n"); }


__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
                 ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Bulk copy (TMA) of `bytes` contiguous bytes into shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Bounded wait: true when the phase of `parity` completed; false on abort or
// when the iteration limit ran out (then the device status word is flagged).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned int *status)
{
    for (long long it = 0; it < kSpinLimit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    atomicOr(status, STATUS_TIMEOUT);
    *abort_flag = 1;
    return false;
}

// One staged batch of a warp: the prefilter (hot) view relative to the warp
// tile's first receiver c and the exact-path view in the same frame.  With
// d = c - o (float-float) the exact view holds, per segment, A = d.t and
// S = s0 + A as float-float pairs, AL = A - L (the segment window), the
// compensated N = d x t and the direction as (hi, lo), so that for a receiver
// at x = c + x' the pair needs only x'.t and x' x t:
//   s_loc = A + x'.t,  s = S + x'.t,  n = N + x' x t.
struct StageSmem {
    float4 O[kBatch];               // o' = o - c, s0_hi (per-warp ball test)
    // prefilter constants, each duplicated into both halves of a float pair:
    // P[0] = t_z, -o'.t;  P[1..2] = 2a o'_x, 2a o'_y, 2a o'_z, beta - a |o'|^2;
    // P[3] = s0 + margin, L + margin;  P[4] = t_x, t_y (as D[0]: the prefilter reads its
    // own copy, which measured 6 % faster testing every pair than sharing D[0])
    float4 P[kBatch][5];
    // exact-path view, two values per word, each duplicated into both halves of a float
    // pair (a lane evaluating one segment for its two receivers loads its operands as
    // pairs); component-major, so lanes loading different segments hit different banks:
    // D[0] t_hi.x, t_hi.y | D[1] t_hi.z, S_hi | D[2] t_lo.x, t_lo.y | D[3] t_lo.z, S_lo
    // D[4] N.x, N.y | D[5] N.z, W Gamma_path | D[6] A_hi, A_lo | D[7] AL_hi, AL_lo
    float4 D[8][kBatch];
    int32_t seg[kBatch];            // global segment index of each staged record
};

// Losses of the staged batch (lossy instantiation): per frequency slot and staged
// segment, log2 |R| and arg R / 2 pi of its porous reflections' factor.
template <int NF>
struct LossSmem {
    float2 rf[NF][kBatch];
};

// Exact geometry of one (receiver, segment) pair in the warp tile's frame, in
// float-float: x' = (xh + xl) exactly; returns false when the pair falls outside
// the window.  `fast`: the warp item's choice of the FP32 local projection, within eps
// of x'.t; a pair within eps of an end of its window is decided and evaluated with the
// float-float projection instead, so the window test is as exact as on that path.  The
// paired twin in survivor_pair rounds each half identically, except that it switches a
// whole pair to the float-float projection when either half is near a window end (the
// other half's value then differs by at most the FP32 projection's error, and its window
// decision is the same).
template <int WINDOW>
__device__ __forceinline__ bool frame_geometry(float xh, float yh, float zh, float xl, float yl,
                                               float zl, const StageSmem &w, int j, bool fast,
                                               float eps, float &sh, float &sl, float &n2)
{
    const float4 d0 = w.D[0][j], d1 = w.D[1][j], d2 = w.D[2][j], d3 = w.D[3][j];
    const float4 d4 = w.D[4][j], d5 = w.D[5][j];
    const float4 T = make_float4(d0.x, d0.z, d1.x, d1.z), TL = make_float4(d2.x, d2.z, d3.x, d3.z);
    const float4 NN = make_float4(d4.x, d4.z, d5.x, d5.z);
    // u = x'.t as (U + ul)
    float U, ul;
    auto exact_u = [&]() {
        const float p0 = __fmul_rn(xh, T.x), p1 = __fmul_rn(yh, T.y), p2 = __fmul_rn(zh, T.z);
        const float r0 = fmaf(xh, TL.x, fmaf(xl, T.x, fmaf(xh, T.x, -p0)));
        const float r1 = fmaf(yh, TL.y, fmaf(yl, T.y, fmaf(yh, T.y, -p1)));
        const float r2 = fmaf(zh, TL.z, fmaf(zl, T.z, fmaf(zh, T.z, -p2)));
        float S1, E1, E2;
        two_sum(p0, p1, S1, E1);
        two_sum(S1, p2, U, E2);
        ul = __fadd_rn(__fadd_rn(E1, E2), __fadd_rn(__fadd_rn(r0, r1), r2));
    };
    if (fast) {
        U = fmaf(xh, T.x, fmaf(yh, T.y, __fmul_rn(zh, T.z)));
        ul = fmaf(xl, T.x, fmaf(yl, T.y, fmaf(zl, T.z, fmaf(xh, TL.x, fmaf(yh, TL.y, __fmul_rn(zh, TL.z))))));
    } else {
        exact_u();
    }
    if (WINDOW == GBT_WINDOW_SEGMENT) {
        const float4 d6 = w.D[6][j], d7 = w.D[7][j];
        float wa = __fadd_rn(__fadd_rn(d6.x, U), __fadd_rn(d6.z, ul));
        float wb = __fadd_rn(__fadd_rn(d7.x, U), __fadd_rn(d7.z, ul));
        if (fast && fminf(fabsf(wa), fabsf(wb)) <= eps) {
            fast = false;
            exact_u();
            wa = __fadd_rn(__fadd_rn(d6.x, U), __fadd_rn(d6.z, ul));
            wb = __fadd_rn(__fadd_rn(d7.x, U), __fadd_rn(d7.z, ul));
        }
        if (!(wa >= 0.0f)) return false;
        if (!(wb < 0.0f)) return false;
    }
    float e3;
    two_sum(T.w, U, sh, e3);
    sl = __fadd_rn(e3, __fadd_rn(ul, TL.w));
    if (WINDOW == GBT_WINDOW_LINE) {
        float ss = __fadd_rn(sh, sl);
        if (fast && fabsf(ss) <= eps) {
            fast = false;
            exact_u();
            two_sum(T.w, U, sh, e3);
            sl = __fadd_rn(e3, __fadd_rn(ul, TL.w));
            ss = __fadd_rn(sh, sl);
        }
        if (!(ss >= 0.0f)) return false;
    }
    // n = N + x' x t: the small terms first (float-float projection only), then the
    // main products
    float n0x = NN.x, n0y = NN.y, n0z = NN.z;
    if (!fast) {
        n0x = __fadd_rn(n0x, fmaf(yl, T.z, fmaf(-zl, T.y, fmaf(yh, TL.z, __fmul_rn(-zh, TL.y)))));
        n0y = __fadd_rn(n0y, fmaf(zl, T.x, fmaf(-xl, T.z, fmaf(zh, TL.x, __fmul_rn(-xh, TL.z)))));
        n0z = __fadd_rn(n0z, fmaf(xl, T.y, fmaf(-yl, T.x, fmaf(xh, TL.y, __fmul_rn(-yh, TL.x)))));
    }
    const float nx = fmaf(yh, T.z, fmaf(-zh, T.y, n0x));
    const float ny = fmaf(zh, T.x, fmaf(-xh, T.z, n0y));
    const float nz = fmaf(xh, T.y, fmaf(-yh, T.x, n0z));
    n2 = fmaf(nx, nx, fmaf(ny, ny, __fmul_rn(nz, nz)));
    return true;
}

// Adjoint terms of one beam: with c~ the contribution without W Gamma_path,
// G += Re(conj(g) c~) and H += Re(conj(g) dc~/db), where
// d log c / db = 1/b + i/E - k n^2 / (2 E^2), E = s - i b.  With losses c~ carries
// the porous reflections' factor (rf: log2 |R|, arg R in turns) and exp(-a s); neither
// depends on b, so the logarithmic derivative is the same.
template <bool LOSSY>
__device__ __forceinline__ void beam_adjoint(const FreqConst &q, float sh, float sl, float n2,
                                             float invD, float2 g, float &G, float &H,
                                             float2 rf = make_float2(0.f, 0.f))
{
    const float n2invD = n2 * invD;
    float ex = -q.kb2l2e * n2invD;
    if (LOSSY) ex = fmaf(-q.al2e, sh, ex + rf.x);
    const float ga = ex2_approx(ex);
    const float ph = __fmul_rn(q.K_hi, sh);       // rounded: pe below is its exact error
    const float pe = fmaf(q.K_hi, sh, -ph);
    const float corr = fmaf(q.K_hi, sl, fmaf(q.K_lo, sh, pe));
    float tau = __fsub_rn(ph, rintf(ph)) + corr;
    tau = fmaf(q.halfK * n2invD, sh, tau);
    if (LOSSY) tau += rf.y;
    tau = tau - rintf(tau);
    float sn, cs;
    __sincosf(6.283185307179586f * tau, &sn, &cs);
    const float gs = q.scale * ga * invD;
    const float cr = gs * fmaf(sh, cs, -q.b * sn);
    const float ci = gs * fmaf(sh, sn, q.b * cs);
    G = fmaf(g.x, cr, fmaf(g.y, ci, G));
    const float t = q.kh * n2 * invD * invD;                         // k n^2 / (2 D^2)
    const float dr = q.invb - q.b * invD - t * (sh * sh - q.b2);      // Re d log c / db
    const float di = sh * invD - t * (2.0f * sh * q.b);               // Im d log c / db
    H = fmaf(g.x, cr * dr - ci * di, fmaf(g.y, cr * di + ci * dr, H));
}

// Counting pass: the kept (pair, frequency) triples of one surviving pair, with
// the same geometry and cutoff arithmetic as the forward path.
template <int NF, int WINDOW>
__device__ __forceinline__ void survivor_count(const FwdParams &p, float xh, float yh, float zh,
                                               float xl, float yl, float zl, const StageSmem &w,
                                               int j, bool fast, float eps, uint32_t &kept)
{
    float sh, sl, n2;
    if (!frame_geometry<WINDOW>(xh, yh, zh, xl, yl, zl, w, j, fast, eps, sh, sl, n2)) return;
    if (p.uniform_b) {
        const float D = fmaf(sh, sh, p.fc[0].b2);
        const float r = n2 * rcp_approx(D);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (f >= p.nf) break;
            if (p.fc[f].kb2 * r > p.cutoff) break;
            ++kept;
        }
    } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (f >= p.nf) break;
            const float D = fmaf(sh, sh, p.fc[f].b2);
            if (p.fc[f].kb2 * n2 > p.cutoff * D) continue;
            ++kept;
        }
    }
}

// Two surviving pairs at once in paired FP32: receiver 0 of the lane with
// segment j0 and receiver 1 with segment j1 (a side without a survivor repeats
// the other side's segment and is masked out).  Every operation is the paired
// twin of one pair's evaluation (frame_geometry, then per frequency the Gaussian,
// the phase reduced in turns and the 1/E factor), so each half rounds as that
// evaluation would; only the MUFU operations run per half.  accx / accy
// hold the two receivers' real / imaginary sums per sorted frequency.
// Two staged words of segments j0 (lo half) and j1 (hi half) as float pairs; with one
// segment for both halves (SAME) the duplicated word is the pair itself.
template <bool SAME>
__device__ __forceinline__ void ld_pairs(const float4 &a, const float4 &b, f2x &u, f2x &v)
{
    if (SAME) {
        const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(&a);
        u = q.x;
        v = q.y;
    } else {
        const float4 qa = a, qb = b;
        u = pk(qa.x, qb.x);
        v = pk(qa.z, qb.z);
    }
}

template <int NF, int WINDOW, bool LOSSY, bool SAME = false>
__device__ __forceinline__ void survivor_pair(const FwdParams &p, f2x XH, f2x YH, f2x ZH,
                                              f2x XL, f2x YL, f2x ZL, f2x NXH, f2x NYH, f2x NZH,
                                              const StageSmem &w,
                                              const LossSmem<NF> *loss, int j0, int j1, bool h0,
                                              bool h1, bool fast, float eps, f2x (&accx)[NF],
                                              f2x (&accy)[NF])
{
    f2x THX, THY, THZ, SH, TLX, TLY, TLZ, SL, NX0, NY0, NZ0, AMP;
    ld_pairs<SAME>(w.D[0][j0], w.D[0][j1], THX, THY);
    ld_pairs<SAME>(w.D[1][j0], w.D[1][j1], THZ, SH);
    ld_pairs<SAME>(w.D[2][j0], w.D[2][j1], TLX, TLY);
    ld_pairs<SAME>(w.D[3][j0], w.D[3][j1], TLZ, SL);
    // u = x'.t as (U + ul): float-float, or (warp-uniform `fast`, compact warps at low
    // enough frequencies) the FP32 products with the lo parts' first-order terms, within
    // eps of x'.t.  A pair with a live half within eps of an end of its window takes the
    // float-float projection instead (`exact`), so every window decision is as exact as
    // on that path (frame_geometry does the same for one pair).
    f2x U, ul;
    f2x AH, AL, BH, BL;
    if (WINDOW == GBT_WINDOW_SEGMENT) {
        ld_pairs<SAME>(w.D[6][j0], w.D[6][j1], AH, AL);
        ld_pairs<SAME>(w.D[7][j0], w.D[7][j1], BH, BL);
    }
    bool exact = !fast;
    if (fast) {
        U = fma2(XH, THX, fma2(YH, THY, mul2(ZH, THZ)));
        ul = fma2(XL, THX, fma2(YL, THY, fma2(ZL, THZ, fma2(XH, TLX, fma2(YH, TLY, mul2(ZH, TLZ))))));
        float a0, a1, b0, b1;
        if (WINDOW == GBT_WINDOW_SEGMENT) {
            upk(add2(add2(AH, U), add2(AL, ul)), a0, a1);
            upk(add2(add2(BH, U), add2(BL, ul)), b0, b1);
        } else {
            upk(add2(add2(SH, U), add2(SL, ul)), a0, a1);   // s, near 0 exact as the sum
            b0 = a0;
            b1 = a1;
        }
        exact = (h0 && fminf(fabsf(a0), fabsf(b0)) <= eps) || (h1 && fminf(fabsf(a1), fabsf(b1)) <= eps);
    }
    if (exact) {
        const f2x p0 = mul2(XH, THX), p1 = mul2(YH, THY), p2 = mul2(ZH, THZ);
        const f2x r0 = fma2(XH, TLX, fma2(XL, THX, fma2(XH, THX, neg2(p0))));
        const f2x r1 = fma2(YH, TLY, fma2(YL, THY, fma2(YH, THY, neg2(p1))));
        const f2x r2 = fma2(ZH, TLZ, fma2(ZL, THZ, fma2(ZH, THZ, neg2(p2))));
        f2x S1, E1, E2;
        two_sum2(p0, p1, S1, E1);
        two_sum2(S1, p2, U, E2);
        ul = add2(add2(E1, E2), add2(add2(r0, r1), r2));
    }
    bool k0 = h0, k1 = h1;
    float u0, u1;
    if (WINDOW == GBT_WINDOW_SEGMENT) {
        upk(add2(add2(AH, U), add2(AL, ul)), u0, u1);
        k0 = k0 && u0 >= 0.0f;
        k1 = k1 && u1 >= 0.0f;
        upk(add2(add2(BH, U), add2(BL, ul)), u0, u1);
        k0 = k0 && u0 < 0.0f;
        k1 = k1 && u1 < 0.0f;
    }
    f2x sh, e3;
    two_sum2(SH, U, sh, e3);
    const f2x sl = add2(e3, add2(ul, SL));
    if (WINDOW == GBT_WINDOW_LINE) {
        upk(add2(sh, sl), u0, u1);
        k0 = k0 && u0 >= 0.0f;
        k1 = k1 && u1 >= 0.0f;
    }
    if (!(k0 || k1)) return;
    ld_pairs<SAME>(w.D[4][j0], w.D[4][j1], NX0, NY0);
    ld_pairs<SAME>(w.D[5][j0], w.D[5][j1], NZ0, AMP);
    // n = N + x' x t; the lo parts' products (about 1.3 ulp of |x'|) only where the
    // projection is float-float: on the FP32 path they are below its own rounding
    f2x n0x = NX0, n0y = NY0, n0z = NZ0;
    if (exact) {
        n0x = add2(n0x, fma2(YL, THZ, fma2(neg2(ZL), THY, fma2(YH, TLZ, mul2(neg2(ZH), TLY)))));
        n0y = add2(n0y, fma2(ZL, THX, fma2(neg2(XL), THZ, fma2(ZH, TLX, mul2(neg2(XH), TLZ)))));
        n0z = add2(n0z, fma2(XL, THY, fma2(neg2(YL), THX, fma2(XH, TLY, mul2(neg2(YH), TLX)))));
    }
    const f2x nx = fma2(YH, THZ, fma2(NZH, THY, n0x));
    const f2x ny = fma2(ZH, THX, fma2(NXH, THZ, n0y));
    const f2x nz = fma2(XH, THY, fma2(NYH, THX, n0z));
    const f2x n2 = fma2(nx, nx, fma2(ny, ny, mul2(nz, nz)));
    const f2x amp = AMP;
    float n20, n21;
    upk(n2, n20, n21);

    // one beam term on both halves, each half kept where its flag is set; with losses
    // the Gaussian exponent takes log2 |R| - a s log2(e) and the phase arg R / 2 pi
    auto beam = [&](const FreqConst &q, int f, f2x invD, bool kf0, bool kf1, f2x &bx, f2x &by) {
        const f2x n2invD = mul2(n2, invD);
        float e0, e1;
        f2x ex = mul2(splat(-q.kb2l2e), n2invD);
        f2x RPH = 0ull;
        if (LOSSY) {
            const float2 r0 = loss->rf[f][j0], r1 = loss->rf[f][j1];
            ex = fma2(splat(-q.al2e), sh, add2(ex, pk(r0.x, r1.x)));
            RPH = pk(r0.y, r1.y);
        }
        upk(ex, e0, e1);
        const f2x ga = pk(ex2_approx(e0), ex2_approx(e1));
        const f2x KH = splat(q.K_hi);
        const f2x nph = mul2(splat(-q.K_hi), sh);    // -K_hi sh, exactly
        const f2x pe = fma2(KH, sh, nph);
        const f2x corr = fma2(KH, sl, fma2(splat(q.K_lo), sh, pe));
        f2x tau = add2(sub2(rint2(nph), nph), corr);   // = ph - rint(ph)
        tau = fma2(mul2(splat(q.halfK), n2invD), sh, tau);
        if (LOSSY) tau = add2(tau, RPH);
        // |tau| < 2^22 turns (beyond it FP32 holds no phase): round by 1.5 x 2^23
        tau = sub2(tau, sub2(add2(tau, splat(12582912.0f)), splat(12582912.0f)));
        float t0, t1, s0, c0, s1, c1;
        upk(mul2(splat(6.283185307179586f), tau), t0, t1);
        __sincosf(t0, &s0, &c0);
        __sincosf(t1, &s1, &c1);
        const f2x SN = pk(s0, s1), CS = pk(c0, c1);
        const f2x gg = mul2(mul2(mul2(mul2(splat(q.scale), amp), ga), invD),
                            pk(kf0 ? 1.0f : 0.0f, kf1 ? 1.0f : 0.0f));
        const f2x B = splat(q.b);
        bx = fma2(gg, fma2(sh, CS, mul2(splat(-q.b), SN)), bx);
        by = fma2(gg, fma2(sh, SN, mul2(B, CS)), by);
    };
    if (p.uniform_b) {
        // one b for all frequencies, sorted by k: each half keeps a prefix
        float d0, d1;
        upk(fma2(sh, sh, splat(p.fc[0].b2)), d0, d1);
        const f2x invD = pk(rcp_approx(d0), rcp_approx(d1));
        float r0_, r1_;
        upk(mul2(n2, invD), r0_, r1_);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (f >= p.nf) break;
            const FreqConst &q = p.fc[f];
            k0 = k0 && !(q.kb2 * r0_ > p.cutoff);
            k1 = k1 && !(q.kb2 * r1_ > p.cutoff);
            if (!(k0 || k1)) break;
            beam(q, f, invD, k0, k1, accx[f], accy[f]);
        }
    } else {
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            if (f >= p.nf) break;
            const FreqConst &q = p.fc[f];
            float d0, d1;
            upk(fma2(sh, sh, splat(q.b2)), d0, d1);
            const bool kf0 = k0 && !(q.kb2 * n20 > p.cutoff * d0);
            const bool kf1 = k1 && !(q.kb2 * n21 > p.cutoff * d1);
            if (!(kf0 || kf1)) continue;
            beam(q, f, pk(rcp_approx(d0), rcp_approx(d1)), kf0, kf1, accx[f], accy[f]);
        }
    }
}

// Adjoint terms of one surviving pair added into G and H[f] (gk: this receiver's
// g per sorted frequency, stride kR * 32 float2).
template <int NF, int WINDOW, bool LOSSY>
__device__ __forceinline__ void survivor_adjoint(const FwdParams &p, float xh, float yh, float zh,
                                                 float xl, float yl, float zl, const StageSmem &w,
                                                 const LossSmem<NF> *loss, int j, bool fast,
                                                 float eps, const float2 *gk, float &G,
                                                 float (&H)[NF])
{
    float sh, sl, n2;
    if (!frame_geometry<WINDOW>(xh, yh, zh, xl, yl, zl, w, j, fast, eps, sh, sl, n2)) return;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (f >= p.nf) break;
        const FreqConst &q = p.fc[f];
        const float D = fmaf(sh, sh, q.b2);
        if (q.kb2 * n2 > p.cutoff * D) {
            if (p.uniform_b) break;
            continue;
        }
        beam_adjoint<LOSSY>(q, sh, sl, n2, rcp_approx(D), gk[f * (kR * 32)], G, H[f],
                            LOSSY ? loss->rf[f][j] : make_float2(0.f, 0.f));
    }
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Adds an FP32 partial sum into a float-float accumulator (hi, hi, lo, lo).
__device__ __forceinline__ void fold(float4 *acc, float2 &t)
{
    if (t.x != 0.0f || t.y != 0.0f) {
        float4 a = *acc;
        float s, e;
        two_sum(a.x, t.x, s, e);
        a.x = s;
        a.z += e;
        two_sum(a.y, t.y, s, e);
        a.y = s;
        a.w += e;
        *acc = a;
        t = make_float2(0.0f, 0.0f);
    }
}


// Conservative test: can the segment (origin (ox, oy, oz) relative to the frame
// of `sphere`, record words r0 / r1) keep any receiver inside the ball `sphere`
// (centre xyz, radius w)?  The distance from the segment line to a point is
// 1-Lipschitz, so shrinking the ball's centre distance by the radius bounds n
// from below and |s| from above over the whole ball; the radius carries slack
// for FP32 rounding at these magnitudes.
template <int WINDOW>
__device__ __forceinline__ bool ball_may_keep(const float4 &r0, const float4 &r1, float ox, float oy,
                                              float oz, const float4 &sphere, float alpha, float beta)
{
    const float dx = sphere.x - ox, dy = sphere.y - oy, dz = sphere.z - oz;
    const float sc = fmaf(dx, r1.x, fmaf(dy, r1.y, dz * r1.z));
    const float cxr = dy * r1.z - dz * r1.y, cyr = dz * r1.x - dx * r1.z, czr = dx * r1.y - dy * r1.x;
    // |d x t| from below: the approximate square root is within a few ulp, and the
    // factor takes it under the exact root
    float nc;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(nc) : "f"(fmaf(cxr, cxr, fmaf(cyr, cyr, czr * czr))));
    nc *= 0.999999f;
    const float R = sphere.w * 1.0001f + 0.05f + 1e-5f * (fabsf(ox) + fabsf(oy) + fabsf(oz));
    bool win;
    if (WINDOW == GBT_WINDOW_LINE) win = r0.w + sc + R >= -kWinMargin;
    else win = (sc + R >= -kWinMargin) && (sc - R <= r1.w + kWinMargin);
    const float sabs = fabsf(r0.w + sc) + R;
    const float nn = nc - R;
    return win && (nn <= 0.f || alpha * nn * nn <= fmaf(sabs, sabs, beta));
}

// Two values, each duplicated into both halves of a float pair.
__device__ __forceinline__ float4 dup2(float a, float b) { return make_float4(a, a, b, b); }

// Stage lane's raw record for the warp: the prefilter view relative to the frame
// c = (cx, cy, cz) (the warp tile's first receiver), the origin in that frame for the
// per-warp ball test and the direction.  A record past the segment count becomes one no
// receiver can keep.  Returns L_hi.
__device__ __forceinline__ float stage_batch(StageSmem &w, const float4 (&raw)[kRecFloats / 4],
                                             int lane, bool valid, int32_t seg, float cx,
                                             float cy, float cz, float alpha, float beta)
{
    const float4 r0 = raw[0], r1 = raw[1], r2 = raw[2];
    float4 *P = w.P[lane];
    w.seg[lane] = valid ? seg : -1;
    if (valid) {
        const float ox = (r0.x - cx) + r2.x, oy = (r0.y - cy) + r2.y, oz = (r0.z - cz) + r2.z;
        w.O[lane] = make_float4(ox, oy, oz, r0.w);
        const float ot = fmaf(ox, r1.x, fmaf(oy, r1.y, oz * r1.z));
        const float oo = fmaf(ox, ox, fmaf(oy, oy, oz * oz));
        const float a2 = 2.f * alpha;
        w.D[0][lane] = dup2(r1.x, r1.y);
        P[4] = dup2(r1.x, r1.y);
        P[0] = dup2(r1.z, -ot);
        P[1] = dup2(a2 * ox, a2 * oy);
        P[2] = dup2(a2 * oz, fmaf(-alpha, oo, beta));
        P[3] = dup2(r0.w + kWinMargin, r1.w + kWinMargin);
    } else {
        // far behind its own start
        w.O[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        w.D[0][lane] = dup2(0.f, 0.f);
        P[4] = dup2(0.f, 0.f);
        P[0] = dup2(0.f, -1e15f);
        P[1] = dup2(0.f, 0.f);
        P[2] = dup2(0.f, 0.f);
        P[3] = dup2(0.f, 0.f);
    }
    return valid ? r1.w : 0.f;
}

// Stage lane's raw record's exact-path view in the warp's frame: float-float
// d = c - o, A = d.t, S = s0 + A, AL = A - L and the compensated N = d x t, with the
// direction as (hi, lo) and the amplitude; finite values past the segment count.
__device__ __forceinline__ void stage_exact(StageSmem &w, const float4 (&raw)[kRecFloats / 4],
                                            int lane, bool valid, float cx, float cy, float cz)
{
    const float4 r0 = raw[0], r1 = raw[1], r2 = raw[2], r3 = raw[3], r4 = raw[4];
    if (valid) {
        // d = c - o as (dh + dl)
        float dxh, dxe, dyh, dye, dzh, dze;
        two_sum(cx, -r0.x, dxh, dxe);
        two_sum(cy, -r0.y, dyh, dye);
        two_sum(cz, -r0.z, dzh, dze);
        const float dxl = __fsub_rn(dxe, r2.x), dyl = __fsub_rn(dye, r2.y), dzl = __fsub_rn(dze, r2.z);
        // A = d.t, float-float
        const float q0 = __fmul_rn(dxh, r1.x), q1 = __fmul_rn(dyh, r1.y), q2 = __fmul_rn(dzh, r1.z);
        const float e0 = fmaf(dxh, r3.x, fmaf(dxl, r1.x, fmaf(dxh, r1.x, -q0)));
        const float e1 = fmaf(dyh, r3.y, fmaf(dyl, r1.y, fmaf(dyh, r1.y, -q1)));
        const float e2 = fmaf(dzh, r3.z, fmaf(dzl, r1.z, fmaf(dzh, r1.z, -q2)));
        float S1, E1, Ah, E2;
        two_sum(q0, q1, S1, E1);
        two_sum(S1, q2, Ah, E2);
        const float Al = __fadd_rn(__fadd_rn(E1, E2), __fadd_rn(__fadd_rn(e0, e1), e2));
        // S = s0 + A, AL = A - L
        float Sh, es, ALh, ea;
        two_sum(r0.w, Ah, Sh, es);
        const float Sl = __fadd_rn(es, __fadd_rn(Al, r2.w));
        two_sum(Ah, -r1.w, ALh, ea);
        const float ALl = __fadd_rn(ea, __fsub_rn(Al, r3.w));
        // N = d x t, compensated
        const float nx = dop(dyh, r1.z, dzh, r1.y) +
                         fmaf(dyh, r3.z, fmaf(-dzh, r3.y, fmaf(dyl, r1.z, -dzl * r1.y)));
        const float ny = dop(dzh, r1.x, dxh, r1.z) +
                         fmaf(dzh, r3.x, fmaf(-dxh, r3.z, fmaf(dzl, r1.x, -dxl * r1.z)));
        const float nz = dop(dxh, r1.y, dyh, r1.x) +
                         fmaf(dxh, r3.y, fmaf(-dyh, r3.x, fmaf(dxl, r1.y, -dyl * r1.x)));
        w.D[1][lane] = dup2(r1.z, Sh);
        w.D[2][lane] = dup2(r3.x, r3.y);
        w.D[3][lane] = dup2(r3.z, Sl);
        w.D[4][lane] = dup2(nx, ny);
        w.D[5][lane] = dup2(nz, r4.x);
        w.D[6][lane] = dup2(Ah, Al);
        w.D[7][lane] = dup2(ALh, ALl);
    } else {
        w.D[1][lane] = dup2(0.f, -1e15f);
        w.D[2][lane] = dup2(0.f, 0.f);
        w.D[3][lane] = dup2(0.f, 0.f);
        w.D[4][lane] = dup2(0.f, 0.f);
        w.D[5][lane] = dup2(0.f, 0.f);
        w.D[6][lane] = dup2(-1e15f, 0.f);
        w.D[7][lane] = dup2(-1e15f, 0.f);
    }
}

template <int NF>
struct AdjSmem {
    float2 g[NF][kR][32];      // the warp's receivers' g, per sorted frequency
};
// Per-warp shared memory of the pair kernel: two raw record buffers (bulk-copy
// or cp.async targets), the staged batch, and the completion barriers of the
// bulk copies.
struct WarpBuf {
    float4 raw[kWRaw][kBatch][kRecFloats / 4];
    StageSmem stg;
    unsigned long long bar[kWRaw];
    int32_t queue[kBatch];           // list positions of the next batch for this warp tile
    int abort_flag, pad[3];
};

template <int NF, int MODE, bool BATCHED, bool LOSSY = false>
struct PairCfg {
    static constexpr size_t kAdj = MODE == kBwd ? sizeof(AdjSmem<NF>) : 0;
    static constexpr size_t kInst = BATCHED ? sizeof(FwdParams) : 0;
    static constexpr size_t kLoss = LOSSY ? sizeof(LossSmem<NF>) : 0;
    static constexpr size_t kPerWarp = (sizeof(WarpBuf) + kAdj + kInst + kLoss + 127) / 128 * 128;
    // as many warps as fit in the shared memory budget, at most kWarpsFwd
    static constexpr int kFit = (int)(kSmemBudget / kPerWarp);
    static constexpr int kWarps = kFit < kWarpsFwd ? kFit : kWarpsFwd;
    static constexpr size_t kSmem = kWarps * kPerWarp;
};

// Persistent pair kernel.  Every warp works on its own: it takes (warp tile of
// 64 receivers, segment split) items from a global queue (CTA tiles of 960
// heaviest first), streams the item's record batches into its own double buffer
// (one bulk copy per batch for consecutive segments, one 16-byte cp.async per
// lane and word for a tile's list), stages each batch relative to its first
// receiver, and runs the prefilter and the exact path for its receivers.  No
// warp ever waits for another, so warps whose receivers meet more surviving
// pairs cost only themselves.  The FP32 sums fold into the item's float-float
// partials (global, resident in L2) every kFoldEvery batches.
template <int NF, int WINDOW, int MODE, bool BATCHED, bool LOSSY = false>
__global__ void __maxnreg__(128) gbs_fwd_kernel(const __grid_constant__ FwdParams prm)
{
    using Cfg = PairCfg<NF, MODE, BATCHED, LOSSY>;
    static_assert(!(LOSSY && BATCHED), "batches with losses run the single-sum kernel");
    constexpr bool STATS = MODE == kStats;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *const mine = smem_raw + (size_t)warp * Cfg::kPerWarp;
    WarpBuf &B = *reinterpret_cast<WarpBuf *>(mine);
    AdjSmem<NF> &adj = *reinterpret_cast<AdjSmem<NF> *>(mine + sizeof(WarpBuf));
    FwdParams &inst = *reinterpret_cast<FwdParams *>(mine + sizeof(WarpBuf) + Cfg::kAdj);
    LossSmem<NF> *const loss =
        reinterpret_cast<LossSmem<NF> *>(mine + sizeof(WarpBuf) + Cfg::kAdj + Cfg::kInst);

    if (lane == 0) {
        for (int i = 0; i < kWRaw; ++i) mbar_init(smem_addr(&B.bar[i]), 1);
        B.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncwarp();
    volatile int *abort_flag = &B.abort_flag;
    uint32_t n_pre = 0, n_kept = 0;
    unsigned long long n_test = 0;
    uint32_t ph = 0;   // bit i: parity of the next completion of bar[i]

    for (;;) {
        int64_t it = 0;
        if (lane == 0) it = atomicAdd(prm.work_counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (BATCHED) {
            if (it < prm.n_items) {
                int lo = 0, hi = prm.n_inst - 1;      // last instance with inst_off <= it
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (prm.inst_off[mid] <= it) lo = mid;
                    else hi = mid - 1;
                }
                it -= prm.inst_off[lo];
                const int4 *src = reinterpret_cast<const int4 *>(prm.inst + lo);
                int4 *dst = reinterpret_cast<int4 *>(&inst);
                for (int q = lane; q < (int)(sizeof(FwdParams) / 16); q += 32) dst[q] = src[q];
                __syncwarp();
            } else {
                break;
            }
        }
        const FwdParams &p = BATCHED ? inst : prm;
        if ((!BATCHED && it >= p.n_items) || *abort_flag) break;

        // item -> (CTA tile by dispatch rank, split, warp tile within the CTA tile)
        const int64_t per_tile = (int64_t)kTileWarps * p.splits;
        const int64_t tile_rank = it / per_tile;
        const int64_t rem = it - tile_rank * per_tile;
        const int split = (int)(rem / kTileWarps);
        const int wl = (int)(rem - (int64_t)split * kTileWarps);
        const int64_t tile = p.tile_perm ? (int64_t)p.tile_perm[tile_rank] : tile_rank;
        const int64_t wbase = tile * kCtaRecv + (int64_t)wl * kWarpRecv;
        if (wbase >= p.n_recv) continue;
        // the segments this item streams: the CTA tile's list, or every segment
        const int32_t *lst = nullptr;
        int64_t n_seg = *p.n_seg_ptr;
        if (p.list) {
            const int32_t ln = p.list_n[tile];
            if (ln >= 0) {
                lst = p.list + p.list_off[tile];
                n_seg = ln;
            }
        }
        const int64_t n_batches = (n_seg + kBatch - 1) / kBatch;
        const uint32_t nb = split < n_batches ? (uint32_t)((n_batches - 1 - split) / p.splits + 1) : 0u;
        const float alpha = p.pre_alpha, beta = p.pre_beta;
        // frame of the staged batches: the warp tile's first receiver
        const int64_t c_idx = p.order ? p.order[wbase] : wbase;
        const float cx = p.recv[3 * c_idx], cy = p.recv[3 * c_idx + 1], cz = p.recv[3 * c_idx + 2];

        // receiver k of the lane at x = c + x', x' = (xp + xl) exactly
        float xa[kR], ya[kR], za[kR], xp[kR], yp[kR], zp[kR], xl[kR], yl[kR], zl[kR], xx[kR];
        int32_t ridx[kR];
        uint32_t valid = 0;
        float4 *const part_base = p.partial + (int64_t)split * p.nf * p.n_recv;
#pragma unroll
        for (int k = 0; k < kR; ++k) {
            // lane holds receivers lane and lane + 32 of the warp tile: the two halves
            // of its Morton patch, so a beam edge splits work evenly over lanes
            const int64_t r = wbase + (int64_t)k * 32 + lane;
            xa[k] = ya[k] = za[k] = xp[k] = yp[k] = zp[k] = xl[k] = yl[k] = zl[k] = xx[k] = 0.0f;
            ridx[k] = -1;
            if (r < p.n_recv) {
                const int64_t o = p.order ? p.order[r] : r;
                xa[k] = p.recv[3 * o]; ya[k] = p.recv[3 * o + 1]; za[k] = p.recv[3 * o + 2];
                two_sum(xa[k], -cx, xp[k], xl[k]);
                two_sum(ya[k], -cy, yp[k], yl[k]);
                two_sum(za[k], -cz, zp[k], zl[k]);
                xx[k] = fmaf(xp[k], xp[k], fmaf(yp[k], yp[k], zp[k] * zp[k]));
                valid |= 1u << k;
                ridx[k] = (int32_t)o;
            }
            if (MODE == kBwd) {
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    adj.g[f][k][lane] = (f < p.nf && ridx[k] >= 0)
                                            ? p.grad_out[(int64_t)p.fperm[f] * p.n_recv + ridx[k]]
                                            : make_float2(0.f, 0.f);
            } else if (MODE == kFwd) {
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    if (f < p.nf && ridx[k] >= 0)
                        part_base[(int64_t)f * p.n_recv + ridx[k]] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        // bounding ball of the warp tile's receivers (relative to its first receiver)
        float4 sphere = make_float4(0.f, 0.f, 0.f, 0.f);
        if (p.tile_cull) {
            float sx = 0.f, sy = 0.f, sz = 0.f, nv = 0.f;
#pragma unroll
            for (int k = 0; k < kR; ++k)
                if ((valid >> k) & 1u) { sx += xp[k]; sy += yp[k]; sz += zp[k]; nv += 1.f; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
                sz += __shfl_xor_sync(0xffffffffu, sz, o);
                nv += __shfl_xor_sync(0xffffffffu, nv, o);
            }
            if (nv > 0.f) { sx /= nv; sy /= nv; sz /= nv; }
            float r2 = 0.f;
#pragma unroll
            for (int k = 0; k < kR; ++k)
                if ((valid >> k) & 1u) {
                    const float ex = xp[k] - sx, ey = yp[k] - sy, ez = zp[k] - sz;
                    r2 = fmaxf(r2, fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
            sphere = make_float4(sx, sy, sz, sqrtf(r2));
        }
        // the FP32 local projection when the warp is compact enough for its frequencies
        float xmax2 = fmaxf((valid & 1u) ? xx[0] : 0.f, (valid & 2u) ? xx[1] : 0.f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) xmax2 = fmaxf(xmax2, __shfl_xor_sync(0xffffffffu, xmax2, o));
        const bool fast_u = sqrtf(xmax2) * p.kmax_turns <= kFastTurns;
        // its error bound: the three-term FP32 dot product with |t| = 1 is within about
        // 3 x 2^-24 max|x'| of x'.t; eps is over five times that
        const float eps_u = 1e-6f * sqrtf(xmax2);
        static_assert(kR == 2, "the paired prefilter handles two receivers per lane");
        const f2x X2 = pk(xp[0], xp[1]), Y2 = pk(yp[0], yp[1]), Z2 = pk(zp[0], zp[1]);
        const f2x NAXX = pk(-alpha * xx[0], -alpha * xx[1]);
        const f2x AL2 = pk(alpha, alpha);
        const f2x MG2 = pk(kWinMargin, kWinMargin);
        // per-batch FP32 sums of the lane's two receivers, paired (re, im)
        f2x accx[NF], accy[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) accx[f] = accy[f] = 0ull;
        const f2x XL2 = pk(xl[0], xl[1]), YL2 = pk(yl[0], yl[1]), ZL2 = pk(zl[0], zl[1]);
        const f2x NX2 = neg2(X2), NY2 = neg2(Y2), NZ2 = neg2(Z2);
        auto fold_all = [&]() {
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if (f < p.nf) {
                    float x0, x1, y0, y1;
                    upk(accx[f], x0, x1);
                    upk(accy[f], y0, y1);
                    float2 t0 = make_float2(x0, y0), t1 = make_float2(x1, y1);
                    if (ridx[0] >= 0) fold(part_base + (int64_t)f * p.n_recv + ridx[0], t0);
                    if (ridx[1] >= 0) fold(part_base + (int64_t)f * p.n_recv + ridx[1], t1);
                }
                accx[f] = accy[f] = 0ull;
            }
        };

        // Batches of the item, double-buffered: raw buffer k % 2 receives batch k.  Consecutive
        // segments: batch k is split + k * splits, one bulk copy (lane 0) on the buffer's
        // mbarrier.  A tile list: the item takes the list's 32-entry chunks split, split +
        // splits, ..., reads this warp tile's word of 32 such chunks at once (one per lane),
        // queues the set bits' list positions in order, gathers the entries of each full
        // batch, and every lane copies its own record with 16-byte async copies (one commit
        // group per batch, empty past the end).
        // Per buffer: records in the batch, and this lane's segment index (or -1).
        int nrec0 = 0, nrec1 = 0;
        int32_t seg0 = -1, seg1 = -1;
        const int64_t n_chunks = (n_seg + kBatch - 1) / kBatch;
        const uint32_t *lw =
            lst ? p.list_words + (p.list_off[tile] / kBatch) * kChunkWords + wl : nullptr;
        int64_t wnext = split;   // list: lane 0's chunk of the next window
        int64_t wchunk = 0;      // list: this lane's chunk in the current window
        uint32_t word = 0u;      // list: its entries for this warp tile not yet queued
        auto next_list_batch = [&](int32_t &pos) -> int {
            int n = 0;
            for (;;) {
                if (!__any_sync(0xffffffffu, word != 0u)) {
                    if (wnext >= n_chunks) break;
                    wchunk = wnext + (int64_t)lane * p.splits;
                    word = wchunk < n_chunks ? lw[wchunk * kChunkWords] : 0u;
                    wnext += (int64_t)kBatch * p.splits;
                    continue;
                }
                // lanes in chunk order, bits in entry order
                const int cnt = __popc(word);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int total = __shfl_sync(0xffffffffu, incl, 31);
                int slot = n + incl - cnt;
                while (word != 0u && slot < kBatch) {
                    B.queue[slot++] = (int32_t)(wchunk * kBatch + __ffs(word) - 1);
                    word &= word - 1u;
                }
                n = min(n + total, kBatch);
                if (n == kBatch) break;
            }
            __syncwarp();
            pos = lane < n ? B.queue[lane] : -1;
            __syncwarp();
            return n;
        };
        auto issue = [&](uint32_t k) {   // all lanes, k in increasing order
            const int buf = (int)(k & 1u);
            int n = 0;
            int32_t idx = -1;
            if (lst) {
                int32_t pos;
                n = next_list_batch(pos);
                idx = pos >= 0 ? lst[pos] : -1;
                if (idx >= 0) {
                    const float4 *src =
                        reinterpret_cast<const float4 *>(p.rec + (int64_t)idx * kRecFloats);
#pragma unroll
                    for (int c = 0; c < kRecFloats / 4; ++c) cp_async16(&B.raw[buf][lane][c], src + c, 16);
                }
                cp_async_commit();
            } else if (k < nb) {
                const int64_t b = split + (int64_t)k * p.splits;
                n = (int)min((int64_t)kBatch, n_seg - b * kBatch);
                idx = lane < n ? (int32_t)(b * kBatch + lane) : -1;
                if (lane == 0) {
                    const uint32_t bytes = (uint32_t)n * kRecFloats * 4;
                    mbar_arrive_expect_tx(smem_addr(&B.bar[buf]), bytes);
                    bulk_g2s(smem_addr(&B.raw[buf][0][0]), p.rec + b * kBatch * kRecFloats, bytes,
                             smem_addr(&B.bar[buf]));
                }
            }
            if (buf) { nrec1 = n; seg1 = idx; } else { nrec0 = n; seg0 = idx; }
        };
        issue(0);
        issue(1);
        uint32_t waited = 0;   // bulk batches whose copy has landed
        bool dirty = false;    // survivors since the last fold
        for (uint32_t kb_ = 0;; ++kb_) {
            const int buf = (int)(kb_ & 1u);
            const int nrec = buf ? nrec1 : nrec0;
            if (nrec <= 0) break;
            const int32_t my_seg = buf ? seg1 : seg0;
            if (lst) {
                cp_async_wait1();   // this lane's copies of batch kb_
            } else {
                bool ok = mbar_wait(smem_addr(&B.bar[buf]), (ph >> buf) & 1u, abort_flag, p.status);
                if (!__all_sync(0xffffffffu, ok)) break;
                ph ^= 1u << buf;
                waited = kb_ + 1;
            }
            const bool seg_ok = lane < nrec;
            StageSmem &w = B.stg;
            const float my_len = stage_batch(w, B.raw[buf][lane], lane, seg_ok, my_seg, cx, cy, cz,
                                             alpha, beta);
            // The exact view: with the pre-cull at once (nearly every batch has survivors);
            // testing every pair only after the prefilter, and only for a batch in which the
            // warp has a survivor (most such batches have none), before raw[buf] is reused.
            if (lst) stage_exact(w, B.raw[buf][lane], lane, seg_ok, cx, cy, cz);
            if (LOSSY && MODE != kStats) {
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    loss->rf[f][lane] = (seg_ok && f < p.nf)
                                            ? p.seg_rf[(int64_t)p.fperm[f] * p.rf_stride + my_seg]
                                            : make_float2(0.f, 0.f);
            }
            uint32_t tmask = 0u;
            if (p.tile_cull) {
                // this lane's segment against the warp tile's ball (own lane's staging only)
                const float4 O = w.O[lane];
                const float4 *R1 = &B.raw[buf][lane][1];   // t_hi, L_hi of the raw record
                // a list entry carrying this warp tile's bit already passed the same test
                // against the warp tile's ball when the lists were built
                const bool pass = seg_ok && (lst != nullptr ||
                                  ball_may_keep<WINDOW>(O, make_float4(R1->x, R1->y, R1->z, my_len),
                                                        O.x, O.y, O.z, sphere, alpha, beta));
                tmask = __ballot_sync(0xffffffffu, pass);
            }
            if (lst) {
                __syncwarp();    // the batch is staged and raw[buf] is free again
                issue(kb_ + 2);
            }

            // ---- prefilter: one keep bit per (receiver, segment); segment jj at bit 31 - jj.
            // Both receivers of the lane go through paired FP32 instructions:
            //   s_loc = x'.t - o'.t,  sm = s_loc + s0 + margin,
            //   g = sm^2 + beta - alpha |x' - o'|^2 + alpha s_loc^2  (= q - alpha n^2),
            // keep iff g >= 0 and the window test holds.
            uint32_t m[kR];
#pragma unroll
            for (int k = 0; k < kR; ++k) m[k] = 0u;
            auto pair_bits = [&](int jj, uint32_t &kb0, uint32_t &kb1) {
                const float4 *P = w.P[jj];
                const float4 p0 = P[4], p1 = P[0], p2 = P[1], p3 = P[2], p4 = P[3];
                const f2x TX = pk(p0.x, p0.y), TY = pk(p0.z, p0.w), TZ = pk(p1.x, p1.y);
                const f2x OT = pk(p1.z, p1.w);
                const f2x OX = pk(p2.x, p2.y), OY = pk(p2.z, p2.w), OZ = pk(p3.x, p3.y);
                const f2x C7 = pk(p3.z, p3.w), S0 = pk(p4.x, p4.y);
                const f2x sl = fma2(X2, TX, fma2(Y2, TY, fma2(Z2, TZ, OT)));
                const f2x sm2 = add2(sl, S0);
                const f2x nd = fma2(X2, OX, fma2(Y2, OY, fma2(Z2, OZ, add2(NAXX, C7))));
                const f2x gg = fma2(mul2(sl, AL2), sl, fma2(sm2, sm2, nd));
                float g0, g1, s0_, s1_;
                upk(gg, g0, g1);
                if (WINDOW == GBT_WINDOW_LINE) {
                    upk(sm2, s0_, s1_);
                    kb0 = ~(__float_as_uint(g0) | __float_as_uint(s0_));
                    kb1 = ~(__float_as_uint(g1) | __float_as_uint(s1_));
                } else {
                    const f2x a = add2(sl, MG2);
                    const f2x bb = sub2(sl, pk(p4.z, p4.w));
                    float a0, a1, b0_, b1_;
                    upk(a, a0, a1);
                    upk(bb, b0_, b1_);
                    kb0 = ~(__float_as_uint(g0) | __float_as_uint(a0)) & __float_as_uint(b0_);
                    kb1 = ~(__float_as_uint(g1) | __float_as_uint(a1)) & __float_as_uint(b1_);
                }
            };
            if (MODE == kFwd && lst) {
                // With the pre-cull most tested pairs survive the exact test, so the
                // prefilter is skipped: every lane takes each segment that reaches the
                // warp tile's ball, in segment order, for both of its receivers.  The
                // exact path rejects whatever the prefilter would have, so the kept terms,
                // their arithmetic and their order per receiver are unchanged.
                uint32_t T = tmask;
                dirty |= T != 0u;
                while (T) {
                    const int jj = __ffs(T) - 1;
                    T &= T - 1;
                    survivor_pair<NF, WINDOW, LOSSY, true>(p, X2, Y2, Z2, XL2, YL2, ZL2, NX2, NY2, NZ2, w, loss, jj,
                                                           jj, (valid & 1u) != 0u, (valid & 2u) != 0u,
                                                           fast_u, eps_u, accx, accy);
                }
            } else if (p.tile_cull) {
                // only the segments that can reach this warp tile's receivers
                uint32_t T = tmask;
                if (STATS) n_test += __popc(T) * __popc(valid);
                while (T) {
                    const int jj = __ffs(T) - 1;
                    T &= T - 1;
                    uint32_t kb0, kb1;
                    pair_bits(jj, kb0, kb1);
                    m[0] |= (kb0 >> 31) << (31 - jj);
                    m[1] |= (kb1 >> 31) << (31 - jj);
                }
            } else {
                if (STATS) n_test += (uint32_t)nrec * __popc(valid);
#pragma unroll 4
                for (int jj = 0; jj < kBatch; ++jj) {
                    uint32_t kb0, kb1;
                    pair_bits(jj, kb0, kb1);
                    m[0] = __funnelshift_l(kb0, m[0], 1);
                    m[1] = __funnelshift_l(kb1, m[1], 1);
                }
            }
            if (!lst) {
                if (__any_sync(0xffffffffu, (((valid & 1u) ? m[0] : 0u) | ((valid & 2u) ? m[1] : 0u)) != 0u))
                    stage_exact(w, B.raw[buf][lane], lane, seg_ok, cx, cy, cz);
                __syncwarp();    // the batch is staged and raw[buf] is free again
                issue(kb_ + 2);
            }
            // ---- survivors, in segment order per receiver
            if (MODE == kFwd && lst) {
                // evaluated above
            } else if (MODE == kFwd) {
                // the two receivers' survivors side by side, each in segment order
                uint32_t mm0 = (valid & 1u) ? m[0] : 0u, mm1 = (valid & 2u) ? m[1] : 0u;
                while (mm0 | mm1) {
                    const bool h0 = mm0 != 0u, h1 = mm1 != 0u;
                    int j0 = __clz(mm0), j1 = __clz(mm1);
                    if (h0) mm0 ^= 0x80000000u >> j0;
                    if (h1) mm1 ^= 0x80000000u >> j1;
                    if (!h0) j0 = j1;
                    if (!h1) j1 = j0;
                    survivor_pair<NF, WINDOW, LOSSY>(p, X2, Y2, Z2, XL2, YL2, ZL2, NX2, NY2, NZ2, w, loss, j0, j1, h0,
                                                     h1, fast_u, eps_u, accx, accy);
                }
            } else if (MODE == kBwd) {
                // segment by segment: the lanes holding a survivor of segment jj add their
                // receivers' terms, the warp sums them, and one lane adds the sums to the
                // segment's global G and H (no shared-memory atomics between lanes)
                const uint32_t mm0 = (valid & 1u) ? m[0] : 0u, mm1 = (valid & 2u) ? m[1] : 0u;
                uint32_t any = __reduce_or_sync(0xffffffffu, mm0 | mm1);
                while (any) {
                    const int jj = __clz(any);
                    any ^= 0x80000000u >> jj;
                    float G = 0.f, H[NF];
#pragma unroll
                    for (int f = 0; f < NF; ++f) H[f] = 0.f;
                    if ((mm0 << jj) >> 31)
                        survivor_adjoint<NF, WINDOW, LOSSY>(p, xp[0], yp[0], zp[0], xl[0], yl[0],
                                                            zl[0], w, loss, jj, fast_u, eps_u,
                                                            &adj.g[0][0][lane],
                                                            G, H);
                    if ((mm1 << jj) >> 31)
                        survivor_adjoint<NF, WINDOW, LOSSY>(p, xp[1], yp[1], zp[1], xl[1], yl[1],
                                                            zl[1], w, loss, jj, fast_u, eps_u,
                                                            &adj.g[0][1][lane],
                                                            G, H);
                    G = warp_sum(G);
#pragma unroll
                    for (int f = 0; f < NF; ++f)
                        if (f < p.nf) H[f] = warp_sum(H[f]);
                    const int32_t jg = w.seg[jj];
                    if (lane == 0 && jg >= 0) {
                        if (G != 0.f) atomicAdd(&p.seg_G[jg], G);
#pragma unroll
                        for (int f = 0; f < NF; ++f)
                            if (f < p.nf && H[f] != 0.f) atomicAdd(&p.seg_H[(int64_t)f * p.seg_stride + jg], H[f]);
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < kR; ++k) {
                    uint32_t mm = ((valid >> k) & 1u) ? m[k] : 0u;
                    if (STATS) n_pre += __popc(mm);
                    while (mm) {
                        const int jj = __clz(mm);
                        mm ^= 0x80000000u >> jj;
                        survivor_count<NF, WINDOW>(p, xp[k], yp[k], zp[k], xl[k], yl[k], zl[k], w, jj,
                                                   fast_u, eps_u, n_kept);
                    }
                }
            }
            if (MODE == kFwd) {
                dirty |= (m[0] | m[1]) != 0u;
                if ((kb_ % kFoldEvery) == kFoldEvery - 1 && dirty) {
                    dirty = false;
                    fold_all();
                }
            }
            __syncwarp();        // before the next batch is staged over this one
        }
        if (lst) {
            cp_async_wait0();    // every gather of this item has landed
        } else if (*abort_flag && lane == 0) {
            // a wait gave up: let the bulk copies still in flight land before leaving
            const uint32_t issued = min(nb, waited + 2u);
            for (uint32_t k = waited; k < issued; ++k) {
                const int bf = (int)(k & 1u);
                for (long long i2 = 0; i2 < kSpinLimit; ++i2)
                    if (mbar_try_wait(smem_addr(&B.bar[bf]), (ph >> bf) & 1u)) break;
                ph ^= 1u << bf;
            }
        }
        if (MODE == kFwd) fold_all();
    }
    if (STATS) {
        atomicAdd(&prm.stats[1], (unsigned long long)n_pre);
        atomicAdd(&prm.stats[2], (unsigned long long)n_kept);
        atomicAdd(&prm.stats[3], n_test);
    }
}

// ------------------------------------------------------------- prepass --

struct PrepParams {
    const int32_t *n_seg_ptr;
    const double *o, *t, *L, *s0;
    const int32_t *ray, *depth, *bmat;
    const float *gamma;
    const float *weight;       // per global ray, or nullptr -> the fan's own weight
    FanDev fan;
    int64_t n_fan;
    int n_materials;
    float *rec;
    float4 *crec;              // cull records (origin, s0, direction, length), 32 B each
    // F64 path records (nullptr when not needed)
    double *amp64;
    unsigned int *status;
    // losses: per-material flow resistivity (kPa s m^-2, <= 0 hard) or nullptr, the
    // primitives that end the segments, the scene's triangles (unit normal at 9..11)
    const float *sigma;
    const int32_t *hit;
    const double *tri;
    int64_t n_tri;
    int nf;
    double freq[GBT_MAX_FREQ];
    float2 *seg_rf;            // [f][rf_stride] (log2 |R|, arg R / 2 pi), or nullptr
    double2 *seg_r64;          // [f][rf_stride] R for the F64 path, or nullptr
    int64_t rf_stride;
};

__device__ __forceinline__ void split_ff(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// Cosine of the angle of incidence at the reflection that starts segment j (depth >= 1):
// |t_j . n| with n the unit normal of the primitive that ended segment j - 1 (ground:
// +z); a mirror reflection keeps |d . n|.  An unknown primitive is flagged.
__device__ __forceinline__ double incidence_cos(const PrepParams &p, int64_t j)
{
    const int prim = p.hit[j - 1];
    double nx = 0.0, ny = 0.0, nz = 1.0;
    if (prim >= 1 && prim <= p.n_tri) {
        const double *n = p.tri + 12 * (int64_t)(prim - 1) + 9;
        nx = n[0]; ny = n[1]; nz = n[2];
    } else if (prim != 0) {
        atomicOr(p.status, STATUS_BAD_INPUT);
    }
    return fabs(p.t[3 * j] * nx + p.t[3 * j + 1] * ny + p.t[3 * j + 2] * nz);
}

// Plane-wave reflection factor of a porous, locally reacting surface of flow resistivity
// sigma (kPa s m^-2) at frequency f for incidence cos(theta) = c: the Delany-Bazley
// normalised impedance Z = 1 + 9.08 (f/sigma)^-0.75 + i 11.9 (f/sigma)^-0.73
// (exp(-i omega t)) in R = (Z c - 1) / (Z c + 1).
__device__ __forceinline__ double2 porous_reflection(double f, double sigma, double c)
{
    const double x = f / sigma;
    const double zr = 1.0 + 9.08 * pow(x, -0.75), zi = 11.9 * pow(x, -0.73);
    const double ar = zr * c - 1.0, ai = zi * c, br = zr * c + 1.0, bi = zi * c;
    const double inv = 1.0 / (br * br + bi * bi);
    return make_double2((ar * br + ai * bi) * inv, (ai * br - ar * bi) * inv);
}

__global__ void prepass_kernel(PrepParams p)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = *p.n_seg_ptr;
    if (j >= n) return;
    // Gamma_path: product of gamma over the reflections before this segment
    double g = 1.0;
    const int dep = p.depth[j];
    for (int q = 1; q <= dep; ++q) {
        const int m = p.bmat[j - dep + q];
        if (m < 0 || m >= p.n_materials) {
            atomicOr(p.status, STATUS_BOUNDS);
            continue;
        }
        g *= (double)p.gamma[m];
    }
    const double w = p.weight ? (double)p.weight[p.ray[j]] : fan_weight(p.fan, p.n_fan, p.ray[j]);
    const double amp = w * g;
    float4 *R = reinterpret_cast<float4 *>(p.rec + j * kRecFloats);
    float oh[3], ol[3], th[3], tl[3], s0h, s0l, Lh, Ll;
    for (int a = 0; a < 3; ++a) {
        split_ff(p.o[3 * j + a], oh[a], ol[a]);
        split_ff(p.t[3 * j + a], th[a], tl[a]);
    }
    split_ff(p.s0[j], s0h, s0l);
    split_ff(p.L[j], Lh, Ll);
    R[0] = make_float4(oh[0], oh[1], oh[2], s0h);     // R_OXH .. R_S0H
    R[1] = make_float4(th[0], th[1], th[2], Lh);      // R_TXH .. R_LH
    R[2] = make_float4(ol[0], ol[1], ol[2], s0l);     // R_OXL .. R_S0L
    R[3] = make_float4(tl[0], tl[1], tl[2], Ll);      // R_TXL .. R_LL
    R[4] = make_float4((float)amp, 0.f, 0.f, 0.f);    // R_AMP
    p.crec[2 * j] = R[0];
    p.crec[2 * j + 1] = R[1];
    if (p.amp64) p.amp64[j] = amp;
    if (p.seg_rf || p.seg_r64) {
        // per frequency: the product of the porous reflections' factors before segment j
        for (int f = 0; f < p.nf; ++f) {
            double rr = 1.0, ri = 0.0;
            if (p.sigma) {
                for (int q = 1; q <= dep; ++q) {
                    const int64_t jq = j - dep + q;
                    const int m = p.bmat[jq];
                    if (m < 0 || m >= p.n_materials) continue;     // flagged above
                    const double sg = (double)p.sigma[m];
                    if (!(sg > 0.0)) continue;                      // hard surface
                    const double2 r = porous_reflection(p.freq[f], sg, incidence_cos(p, jq));
                    const double nr = rr * r.x - ri * r.y;
                    ri = rr * r.y + ri * r.x;
                    rr = nr;
                }
            }
            const int64_t k = (int64_t)f * p.rf_stride + j;
            if (p.seg_rf)
                p.seg_rf[k] = make_float2((float)(0.5 * log2(rr * rr + ri * ri)),
                                          (float)(atan2(ri, rr) * (0.5 / kPi)));
            if (p.seg_r64) p.seg_r64[k] = make_double2(rr, ri);
        }
    }
}

// ------------------------------------------------------ FP64 variant --

constexpr int kThreads64 = 128;
constexpr int kTS64 = 64;

struct F64Params {
    const float *recv;
    const int32_t *order;
    int64_t n_recv;
    const int32_t *n_seg_ptr;
    const double *o, *t, *L, *s0, *amp;
    int nf;
    double cutoff;
    double k[GBT_MAX_FREQ], b[GBT_MAX_FREQ];
    int splits;
    double2 *partial;          // [splits][nf][n_recv]
    double absorb[GBT_MAX_FREQ];   // amplitude decay rate of air per frequency (Np/m)
    const double2 *r64;        // [f][r64_stride] porous reflections' factor, or nullptr
    int64_t r64_stride;
};

// Every step in FP64.  The cull k n^2 b / (2 D) <= C is tested as k b n^2 <= 2 C D
// (no division), first for the union over the frequencies (the smallest k b against the
// largest b^2) so that a pair every frequency culls costs no per-frequency work; the
// accumulators of NF frequency slots stay in registers.
template <int WINDOW, int NF>
__global__ void __launch_bounds__(kThreads64) gbs_fwd_f64_kernel(const F64Params p)
{
    __shared__ double so[kTS64][3], stt[kTS64][3], sL[kTS64], s0s[kTS64], sa[kTS64];
    const int64_t r = (int64_t)blockIdx.x * kThreads64 + threadIdx.x;
    const int split = blockIdx.y;
    const int64_t n_seg = *p.n_seg_ptr;
    const int64_t seg_begin = split * n_seg / p.splits;
    const int64_t seg_end = (split + 1) * n_seg / p.splits;
    const bool valid = r < p.n_recv;
    const int64_t ri = valid ? (p.order ? p.order[r] : r) : 0;
    const double x = valid ? (double)p.recv[3 * ri] : 0.0;
    const double y = valid ? (double)p.recv[3 * ri + 1] : 0.0;
    const double z = valid ? (double)p.recv[3 * ri + 2] : 0.0;
    double kb[NF], b2[NF];
    double kbmin = 1e300, b2max = 0.0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        kb[f] = f < p.nf ? p.k[f] * p.b[f] : 1e300;
        b2[f] = f < p.nf ? p.b[f] * p.b[f] : 0.0;
        kbmin = fmin(kbmin, kb[f]);
        b2max = fmax(b2max, b2[f]);
    }
    const double c2 = 2.0 * p.cutoff;
    double sr[NF], cr[NF], si[NF], ci[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) sr[f] = cr[f] = si[f] = ci[f] = 0.0;
    for (int64_t t0 = seg_begin; t0 < seg_end; t0 += kTS64) {
        __syncthreads();
        for (int q = threadIdx.x; q < kTS64; q += kThreads64) {
            const int64_t j = t0 + q;
            if (j < seg_end) {
                so[q][0] = p.o[3 * j]; so[q][1] = p.o[3 * j + 1]; so[q][2] = p.o[3 * j + 2];
                stt[q][0] = p.t[3 * j]; stt[q][1] = p.t[3 * j + 1]; stt[q][2] = p.t[3 * j + 2];
                sL[q] = p.L[j]; s0s[q] = p.s0[j]; sa[q] = p.amp[j];
            }
        }
        __syncthreads();
        const int nt = (int)min((int64_t)kTS64, seg_end - t0);
        if (!valid) continue;
        for (int q = 0; q < nt; ++q) {
            const double dx = x - so[q][0], dy = y - so[q][1], dz = z - so[q][2];
            const double tx = stt[q][0], ty = stt[q][1], tz = stt[q][2];
            const double sl = dx * tx + dy * ty + dz * tz;
            const double s = s0s[q] + sl;
            if (WINDOW == GBT_WINDOW_SEGMENT) {
                if (!(sl >= 0.0 && sl < sL[q])) continue;
            } else {
                if (!(s >= 0.0)) continue;
            }
            const double cx = dy * tz - dz * ty, cy = dz * tx - dx * tz, cz = dx * ty - dy * tx;
            const double n2 = cx * cx + cy * cy + cz * cz;
            const double ss = s * s;
            // union over the frequencies: culled for every f (with a relative margin far
            // above FP64 rounding, so no pair a frequency keeps is skipped)
            if (kbmin * n2 > c2 * (ss + b2max) * (1.0 + 1e-12)) continue;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                if (f >= p.nf) break;
                const double k = p.k[f], b = p.b[f];
                const double D = ss + b2[f];
                if (kb[f] * n2 > c2 * D) continue;
                // c = amp * (k b / 8 pi^2) / E * exp(i k s + i k n^2 / (2E)), E = s - i b
                const double invD = 1.0 / D;
                const double re_exp = -0.5 * kb[f] * n2 * invD - p.absorb[f] * s;
                const double ph = k * s + 0.5 * k * n2 * s * invD;
                const double a = sa[q] * (kb[f] / (8.0 * kPi * kPi)) * exp(re_exp) * invD;
                double sn, cs;
                sincos(ph, &sn, &cs);
                double vr = a * (s * cs - b * sn), vi = a * (s * sn + b * cs);
                if (p.r64) {
                    const double2 R = p.r64[(int64_t)f * p.r64_stride + t0 + q];
                    const double ur = vr * R.x - vi * R.y;
                    vi = vr * R.y + vi * R.x;
                    vr = ur;
                }
                // Neumaier accumulation
                double t1 = sr[f] + vr;
                cr[f] += fabs(sr[f]) >= fabs(vr) ? (sr[f] - t1) + vr : (vr - t1) + sr[f];
                sr[f] = t1;
                double t2 = si[f] + vi;
                ci[f] += fabs(si[f]) >= fabs(vi) ? (si[f] - t2) + vi : (vi - t2) + si[f];
                si[f] = t2;
            }
        }
    }
    if (!valid) return;
#pragma unroll
    for (int f = 0; f < NF; ++f)
        if (f < p.nf)
            p.partial[((int64_t)split * p.nf + f) * p.n_recv + ri] =
                make_double2(sr[f] + cr[f], si[f] + ci[f]);
}

template <int WINDOW>
void launch_f64(const F64Params &q, dim3 grid, cudaStream_t s)
{
    if (q.nf <= 1) gbs_fwd_f64_kernel<WINDOW, 1><<<grid, kThreads64, 0, s>>>(q);
    else if (q.nf <= 2) gbs_fwd_f64_kernel<WINDOW, 2><<<grid, kThreads64, 0, s>>>(q);
    else if (q.nf <= 4) gbs_fwd_f64_kernel<WINDOW, 4><<<grid, kThreads64, 0, s>>>(q);
    else if (q.nf <= 8) gbs_fwd_f64_kernel<WINDOW, 8><<<grid, kThreads64, 0, s>>>(q);
    else gbs_fwd_f64_kernel<WINDOW, GBT_MAX_FREQ><<<grid, kThreads64, 0, s>>>(q);
}

// ------------------------------------------------------------ adjoint --

// Per ray: the weight gradient sum_j Gamma_path_j G_j, the material gradient
// sum over bounces of W (product of the other bounces' gamma) G_j, and the beam
// parameter gradient sum_j W Gamma_path_j H_jf.  Products of the other
// bounces are formed directly, so gamma = 0 needs no special case.
struct RayGradParams {
    int64_t n_rays, ray_begin;
    const int32_t *ray_off, *bmat;
    const float *gamma, *weight;
    FanDev fan;
    int64_t n_fan;
    const float *seg_G, *seg_H;
    int64_t seg_stride;
    int nf, n_materials;
    float *grad_w;             // n_fan entries (this range written), or nullptr
    double *acc;               // [n_materials] gamma, then [nf] b (sorted slots)
    unsigned int *status;
};

constexpr int kMaxDepth = 65;

__global__ void ray_grad_kernel(RayGradParams p)
{
    extern __shared__ double sacc[];
    const int nacc = p.n_materials + p.nf;
    for (int k = threadIdx.x; k < nacc; k += blockDim.x) sacc[k] = 0.0;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < p.n_rays) {
        const int64_t a = p.ray_off[i];
        const int cnt = (int)(p.ray_off[i + 1] - a);
        const double W = p.weight ? (double)p.weight[p.ray_begin + i]
                                  : fan_weight(p.fan, p.n_fan, p.ray_begin + i);
        double gams[kMaxDepth];
        int mats[kMaxDepth];
        double gp = 1.0, gw = 0.0;
        for (int d = 0; d < cnt && d < kMaxDepth; ++d) {
            const int64_t j = a + d;
            if (d >= 1) {
                int m = p.bmat[j];
                if (m < 0 || m >= p.n_materials) {
                    atomicOr(p.status, STATUS_BOUNDS);
                    m = 0;
                }
                mats[d] = m;
                gams[d] = (double)p.gamma[m];
                gp *= gams[d];
            }
            const double G = (double)p.seg_G[j];
            gw += gp * G;
            if (G != 0.0) {
                for (int q = 1; q <= d; ++q) {
                    double others = 1.0;
                    for (int q2 = 1; q2 <= d; ++q2)
                        if (q2 != q) others *= gams[q2];
                    atomicAdd(&sacc[mats[q]], W * others * G);
                }
            }
            for (int f = 0; f < p.nf; ++f) {
                const double H = (double)p.seg_H[f * p.seg_stride + j];
                if (H != 0.0) atomicAdd(&sacc[p.n_materials + f], W * gp * H);
            }
        }
        if (p.grad_w) p.grad_w[p.ray_begin + i] = (float)gw;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nacc; k += blockDim.x)
        if (sacc[k] != 0.0) atomicAdd(&p.acc[k], sacc[k]);
}

struct GradOutParams {
    const double *acc;
    int n_materials, nf;
    int fperm[GBT_MAX_FREQ];
    float *grad_gamma;
    double *grad_b;
};

__global__ void grad_out_kernel(GradOutParams p)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < p.n_materials) p.grad_gamma[k] = (float)p.acc[k];
    else if (k < p.n_materials + p.nf && p.grad_b)
        p.grad_b[p.fperm[k - p.n_materials]] = p.acc[k];
}

// ------------------------------------------------------------- reduce --

// ---- dispatch order of the CTA tiles: heaviest first
// Items of one tile cost about the same (their batches interleave over the whole
// segment list), but tiles differ by the number of beams that reach them.  A
// sampled count of segments whose Gaussian can reach each tile's bounding ball
// ranks the tiles so the persistent CTAs take the heavy ones first and the queue
// drains with light items (longest processing time first).  The order only
// changes which CTA computes an item, never the arithmetic of any sum.
constexpr int kWeightSamples = 1 << 15;        // sampled segments per estimate
constexpr int64_t kMaxOrderedTiles = 1 << 14;  // beyond this the rank pass is skipped

// A ball with its share of the list test's slack, and a segment's share (seg_reaches_ball).
__device__ __forceinline__ float4 reach_ball(const float4 &b)
{
    return make_float4(b.x, b.y, b.z,
                       fmaf(b.w, 1.0001f, 0.05f) + 1e-5f * (fabsf(b.x) + fabsf(b.y) + fabsf(b.z)));
}
__device__ __forceinline__ float segment_slack(const float4 &r0)
{
    return 1e-5f * (fabsf(r0.x) + fabsf(r0.y) + fabsf(r0.z));
}

// Also each tile's reach ball (the list passes' form, with the ball's share of the slack).
__global__ void tile_ball_kernel(const float *recv, const int32_t *order, int64_t n_recv,
                                 float4 *ball, unsigned int *weight, float4 *rball)
{
    __shared__ float red[4][8];
    const int64_t base = (int64_t)blockIdx.x * kCtaRecv;
    const int n = (int)(n_recv - base < (int64_t)kCtaRecv ? n_recv - base : (int64_t)kCtaRecv);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int64_t o = order ? order[base + j] : base + j;
        sx += recv[3 * o]; sy += recv[3 * o + 1]; sz += recv[3 * o + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    if (lane == 0) { red[0][wid] = sx; red[1][wid] = sy; red[2][wid] = sz; }
    __syncthreads();
    sx = sy = sz = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { sx += red[0][k]; sy += red[1][k]; sz += red[2][k]; }
    const float cx = sx / (float)n, cy = sy / (float)n, cz = sz / (float)n;
    float r2 = 0.f;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int64_t o = order ? order[base + j] : base + j;
        const float dx = recv[3 * o] - cx, dy = recv[3 * o + 1] - cy, dz = recv[3 * o + 2] - cz;
        r2 = fmaxf(r2, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    }
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    __syncthreads();
    if (lane == 0) red[3][wid] = r2;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r2 = fmaxf(r2, red[3][k]);
        ball[blockIdx.x] = make_float4(cx, cy, cz, sqrtf(r2));
        rball[blockIdx.x] = reach_ball(ball[blockIdx.x]);
        weight[blockIdx.x] = 0u;
    }
}

// Bounding ball of each warp tile (64 receivers), one warp per warp tile.
__global__ void warp_ball_kernel(const float *recv, const int32_t *order, int64_t n_recv,
                                 int64_t n_wtiles, float4 *wball)
{
    const int64_t wt = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (wt >= n_wtiles) return;
    float x[2] = {0.f, 0.f}, y[2] = {0.f, 0.f}, z[2] = {0.f, 0.f};
    float sx = 0.f, sy = 0.f, sz = 0.f, nv = 0.f;
    bool ok[2];
    for (int k = 0; k < 2; ++k) {
        const int64_t r = wt * kWarpRecv + k * 32 + lane;
        ok[k] = r < n_recv;
        if (ok[k]) {
            const int64_t o = order ? order[r] : r;
            x[k] = recv[3 * o]; y[k] = recv[3 * o + 1]; z[k] = recv[3 * o + 2];
            sx += x[k]; sy += y[k]; sz += z[k]; nv += 1.f;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
    }
    if (nv > 0.f) { sx /= nv; sy /= nv; sz /= nv; }
    float r2 = 0.f;
    for (int k = 0; k < 2; ++k)
        if (ok[k]) {
            const float dx = x[k] - sx, dy = y[k] - sy, dz = z[k] - sz;
            r2 = fmaxf(r2, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
    for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    if (lane == 0) wball[wt] = make_float4(sx, sy, sz, sqrtf(r2));
}

template <int WINDOW>
__global__ void tile_weight_kernel(const float4 *crec, const int32_t *n_seg_ptr, const float4 *ball,
                                   int64_t n_tiles, float alpha, float beta, unsigned int *weight)
{
    const int64_t ns = *n_seg_ptr;
    const int64_t stride = ns > kWeightSamples ? (ns + kWeightSamples - 1) / kWeightSamples : 1;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * stride;
    const bool ok = j < ns;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    if (ok) {
        r0 = crec[2 * j];
        r1 = crec[2 * j + 1];
    }
    for (int64_t t = 0; t < n_tiles; ++t) {
        const float4 b = ball[t];
        bool pass = false;
        if (ok)
            pass = ball_may_keep<WINDOW>(r0, r1, r0.x - b.x, r0.y - b.y, r0.z - b.z,
                                         make_float4(0.f, 0.f, 0.f, b.w), alpha, beta);
        const unsigned int m = __ballot_sync(0xffffffffu, pass);
        if ((threadIdx.x & 31) == 0 && m) atomicAdd(&weight[t], (unsigned int)__popc(m));
    }
}

// perm[rank] = tile, ranks by weight descending, ties by tile index (a permutation)
__global__ void tile_rank_kernel(const unsigned int *weight, int64_t n_tiles, int32_t *perm)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const unsigned int wt = weight[t];
    int64_t rank = 0;
    for (int64_t u = 0; u < n_tiles; ++u) {
        const unsigned int wu = weight[u];
        rank += (wu > wt) || (wu == wt && u < t);
    }
    perm[rank] = (int32_t)t;
}

// ---- tile pre-cull: per CTA tile, the list of segments that can reach it
// Two passes over (chunk of 1024 segments) x (tile) with the ball test of the
// pre-cull: counts, then the indices, each tile's list in segment order (so the
// sums keep their order and stay deterministic).  Tiles take consecutive ranges
// of the list buffer lightest first; a tile that does not fit streams every
// segment, which gives the same field.
constexpr int kListChunk = 1024;

// The list passes' form of ball_may_keep, with its slack split between the ball and the
// segment: a reach ball (centre, W) with W = r 1.0001 + 0.05 + 1e-5 (|cx| + |cy| + |cz|),
// and the segment's 1e-5 (|ox| + |oy| + |oz|).  Their sum bounds the slack of
// ball_may_keep (|o - c| <= |o| + |c|), so the test is at least as conservative and
// costs each (segment, ball) pair a single add for it.  From a segment's cull record
// (its origin rounded to FP32, which the slack of 5 cm far exceeds).
// A segment's terms of the test, formed once for all the balls it meets: with d = c - o,
// d.t = c.t - o.t and d x t = c x t - o x t, whose extra rounding (a few ulp of |c| and
// |o|) the slack's 1e-5 (|o| + |c|) far exceeds.
struct SegCull {
    float tx, ty, tz, len, s0;   // direction, length, start
    float ot, ox, oy, oz;        // o.t and o x t
    float slack;                 // the segment's share of the slack
};
__device__ __forceinline__ SegCull seg_cull(const float4 &r0, const float4 &r1)
{
    SegCull g;
    g.tx = r1.x; g.ty = r1.y; g.tz = r1.z; g.len = r1.w; g.s0 = r0.w;
    g.ot = fmaf(r0.x, r1.x, fmaf(r0.y, r1.y, r0.z * r1.z));
    g.ox = fmaf(r0.y, r1.z, -r0.z * r1.y);
    g.oy = fmaf(r0.z, r1.x, -r0.x * r1.z);
    g.oz = fmaf(r0.x, r1.y, -r0.y * r1.x);
    g.slack = segment_slack(r0);
    return g;
}
template <int WINDOW>
__device__ __forceinline__ bool seg_reaches_ball(const SegCull &g, const float4 &rb, float alpha,
                                                 float beta)
{
    const float sc = fmaf(rb.x, g.tx, fmaf(rb.y, g.ty, fmaf(rb.z, g.tz, -g.ot)));
    const float cxr = fmaf(rb.y, g.tz, fmaf(-rb.z, g.ty, -g.ox));
    const float cyr = fmaf(rb.z, g.tx, fmaf(-rb.x, g.tz, -g.oy));
    const float czr = fmaf(rb.x, g.ty, fmaf(-rb.y, g.tx, -g.oz));
    float nc;   // |d x t| from below (see ball_may_keep)
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(nc) : "f"(fmaf(cxr, cxr, fmaf(cyr, cyr, czr * czr))));
    nc *= 0.999999f;
    const float R = rb.w + g.slack;
    bool win;
    if (WINDOW == GBT_WINDOW_LINE) win = g.s0 + sc + R >= -kWinMargin;
    else win = (sc + R >= -kWinMargin) && (sc - R <= g.len + kWinMargin);
    const float sabs = fabsf(g.s0 + sc) + R;
    const float nn = nc - R;
    return win && (nn <= 0.f || alpha * nn * nn <= fmaf(sabs, sabs, beta));
}

template <int WINDOW>
__global__ void __launch_bounds__(kListChunk) list_count_kernel(
    const float4 *crec, const int32_t *n_seg_ptr, const float4 *rball, int64_t n_tiles,
    int64_t n_chunks, float alpha, float beta, int32_t *counts, uint32_t *bits)
{
    // block (c, g): chunk c against the 32-tile groups g, g + G, ... (G = gridDim.y); lane
    // k of each warp keeps tile k's ballot of the group, so the group ends with one count
    // and one ballot store per lane
    extern __shared__ int32_t cnt_s[];
    const int64_t G = gridDim.y, g = blockIdx.y;
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x) cnt_s[t] = 0;
    __syncthreads();
    const int64_t ns = *n_seg_ptr;
    const int64_t c = blockIdx.x;
    if (c * kListChunk < ns) {
        const int64_t j = c * kListChunk + threadIdx.x;
        const bool ok = j < ns;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        if (ok) {
            r0 = crec[2 * j];
            r1 = crec[2 * j + 1];
        }
        const SegCull sg = seg_cull(r0, r1);
        const int lane = threadIdx.x & 31;
        for (int64_t t0 = g * 32; t0 < n_tiles; t0 += G * 32) {
            const int nt = (int)min((int64_t)32, n_tiles - t0);
            uint32_t mine = 0u;
            for (int k = 0; k < nt; ++k) {
                const bool pass = ok && seg_reaches_ball<WINDOW>(sg, rball[t0 + k], alpha, beta);
                const uint32_t m = __ballot_sync(0xffffffffu, pass);
                if (lane == k) mine = m;
            }
            if (lane < nt) {
                if (mine) atomicAdd(&cnt_s[t0 + lane], (int32_t)__popc(mine));
                if (bits) bits[(t0 + lane) * n_chunks * 32 + c * 32 + (threadIdx.x >> 5)] = mine;
            }
        }
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x)
        if ((t / 32) % G == g) counts[t * n_chunks + c] = cnt_s[t];
}

// Exclusive scan of 1024 values held one per thread; returns the block total.
__device__ __forceinline__ int64_t block_scan_1024(int64_t v, int64_t &excl, int64_t *ws)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t x = ws[lane];
        int64_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        ws[lane] = xi - x;
        if (lane == 31) ws[32] = xi;
    }
    __syncthreads();
    excl = incl - v + ws[wid];
    const int64_t total = ws[32];
    __syncthreads();
    return total;
}

// One block per tile: chunk counts -> exclusive offsets within the tile; the tile's total.
__global__ void __launch_bounds__(1024) list_scan_chunks_kernel(int32_t *counts, int64_t n_chunks,
                                                                unsigned int *total)
{
    __shared__ int64_t ws[33];
    int32_t *row = counts + (int64_t)blockIdx.x * n_chunks;
    int64_t carry = 0;
    for (int64_t base = 0; base < n_chunks; base += 1024) {
        const int64_t c = base + threadIdx.x;
        const int64_t v = c < n_chunks ? row[c] : 0;
        int64_t excl;
        const int64_t tot = block_scan_1024(v, excl, ws);
        if (c < n_chunks) row[c] = (int32_t)(carry + excl);
        carry += tot;
    }
    if (threadIdx.x == 0) total[blockIdx.x] = (unsigned int)carry;
}

// Per 32-entry chunk of a tile list, one word per warp tile of the CTA tile: bit b set
// if entry b can reach the warp tile's ball.  Each warp takes whole chunks (blocks
// (g, t) stride over tile t's chunks) and writes the chunk's 16 words in one store.
template <int WINDOW>
__global__ void list_words_kernel(const float4 *crec, const float4 *wball, int64_t n_wtiles,
                                  float alpha, float beta, const int64_t *list_off,
                                  const int32_t *list_n, const int32_t *list, uint32_t *list_words)
{
    static_assert(kTileWarps <= kChunkWords, "one word per warp tile");
    __shared__ float4 sball[kTileWarps];
    const int64_t t = blockIdx.y;
    const int32_t n = list_n[t];
    if (n <= 0) return;                    // uniform over the block
    const int nw = (int)min((int64_t)kTileWarps, n_wtiles - t * kTileWarps);
    if (threadIdx.x < nw) sball[threadIdx.x] = reach_ball(wball[t * kTileWarps + threadIdx.x]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t off = list_off[t];       // a multiple of 32
    uint32_t *words = list_words + (off / 32) * kChunkWords;
    const int64_t n_ch = ((int64_t)n + 31) / 32;
    const int64_t wpb = blockDim.x / 32;
    for (int64_t ch = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); ch < n_ch;
         ch += (int64_t)gridDim.x * wpb) {
        const int64_t i = ch * 32 + lane;
        const bool in = i < n;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
        if (in) {
            const int64_t jseg = list[off + i];
            r0 = crec[2 * jseg];
            r1 = crec[2 * jseg + 1];
        }
        const SegCull sg = seg_cull(r0, r1);
        uint32_t mine = 0u;
        for (int w = 0; w < nw; ++w) {
            const uint32_t m = __ballot_sync(
                0xffffffffu, in && seg_reaches_ball<WINDOW>(sg, sball[w], alpha, beta));
            if (lane == w) mine = m;
        }
        if (lane < kChunkWords) words[ch * kChunkWords + lane] = mine;
    }
}

// One block: list ranges, tiles lightest first (perm lists them heaviest first), each
// starting on a 32-entry chunk boundary.
__global__ void __launch_bounds__(1024) list_layout_kernel(const unsigned int *total,
                                                           const int32_t *perm, int64_t n_tiles,
                                                           int64_t cap, int64_t *list_off,
                                                           int32_t *list_n)
{
    __shared__ int64_t ws[33];
    const int64_t per = (n_tiles + 1023) / 1024;
    const int64_t i0 = (int64_t)threadIdx.x * per;
    auto tile_at = [&](int64_t i) {   // i-th lightest tile
        const int64_t r = n_tiles - 1 - i;
        return perm ? (int64_t)perm[r] : r;
    };
    auto padded = [](int64_t n) { return (n + 31) / 32 * 32; };   // whole 32-entry chunks
    int64_t sum = 0;
    for (int64_t i = i0; i < i0 + per && i < n_tiles; ++i) sum += padded(total[tile_at(i)]);
    int64_t off;
    block_scan_1024(sum, off, ws);
    for (int64_t i = i0; i < i0 + per && i < n_tiles; ++i) {
        const int64_t t = tile_at(i);
        const int64_t n = total[t];
        list_off[t] = off;
        list_n[t] = off + padded(n) <= cap ? (int32_t)n : -1;
        off += padded(n);
    }
}

template <int WINDOW>
__global__ void __launch_bounds__(kListChunk) list_write_kernel(
    const float4 *crec, const int32_t *n_seg_ptr, const float4 *rball, int64_t n_tiles,
    int64_t n_chunks, float alpha, float beta, const int32_t *chunk_off, const int64_t *list_off,
    const int32_t *list_n, int32_t *list)
{
    __shared__ int32_t wsum[32];
    const int64_t ns = *n_seg_ptr;
    const int64_t c = blockIdx.x;
    if (c * kListChunk >= ns) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t j = c * kListChunk + threadIdx.x;
    const bool ok = j < ns;
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0;
    if (ok) {
        r0 = crec[2 * j];
        r1 = crec[2 * j + 1];
    }
    const SegCull sg = seg_cull(r0, r1);
    for (int64_t t = 0; t < n_tiles; ++t) {
        if (list_n[t] < 0) continue;
        const bool pass = ok && seg_reaches_ball<WINDOW>(sg, rball[t], alpha, beta);
        const unsigned int m = __ballot_sync(0xffffffffu, pass);
        if (lane == 0) wsum[wid] = __popc(m);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < wid; ++w) before += wsum[w];
        if (pass)
            list[list_off[t] + chunk_off[t * n_chunks + c] + before +
                 __popc(m & ((1u << lane) - 1u))] = (int32_t)j;
        __syncthreads();
    }
}

// The same lists from the ballots the counting pass stored (one 32-bit word per tile and
// warp of 32 segments): no ball test is repeated.  Each warp reads its word of 32 tiles at
// once (one per lane; most are zero), and for each non-zero one finds its place within
// the chunk from the earlier warps' words, so there is no block barrier per tile.  Entry
// order is the same (chunk, then warp, then lane).
__global__ void __launch_bounds__(kListChunk) list_write_bits_kernel(
    const int32_t *n_seg_ptr, int64_t n_tiles, int64_t n_chunks, const uint32_t *bits,
    const int32_t *chunk_off, const int64_t *list_off, const int32_t *list_n, int32_t *list)
{
    const int64_t ns = *n_seg_ptr;
    const int64_t c = blockIdx.x;
    if (c * kListChunk >= ns) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t j = c * kListChunk + threadIdx.x;
    const int64_t row_stride = n_chunks * 32;
    for (int64_t t0 = (int64_t)blockIdx.y * 32; t0 < n_tiles; t0 += (int64_t)gridDim.y * 32) {
        const int64_t tl = t0 + lane;
        uint32_t mw = 0u;
        if (tl < n_tiles && list_n[tl] >= 0) mw = bits[tl * row_stride + c * 32 + wid];
        uint32_t nz = __ballot_sync(0xffffffffu, mw != 0u);
        while (nz) {
            const int k = __ffs(nz) - 1;
            nz &= nz - 1u;
            const int64_t t = t0 + k;
            const uint32_t m = __shfl_sync(0xffffffffu, mw, k);
            const uint32_t *row = bits + t * row_stride + c * 32;
            int before = lane < wid ? __popc(row[lane]) : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
            if ((m >> lane) & 1u)
                list[list_off[t] + chunk_off[t * n_chunks + c] + before +
                     __popc(m & ((1u << lane) - 1u))] = (int32_t)j;
        }
    }
}

// Time synthesis: out[n, r] (+)= Re sum_f ph[n, f] p[f, r], ph[n, f] = A_f exp(-i omega_f t_n).
// Each block forms the phasors of its kSynthTile samples in shared memory: the phase in
// turns, f t0 + n (f dt), reduced to [0, 1) in FP64, then sine and cosine of the reduced
// turn in FP32 (sincospif, about one ulp: the phasors are FP32 numbers either way).
// Threads run over groups of four adjacent receivers (one 16-byte streaming store per
// sample), each holding its receivers' fields in registers; NF is the exact frequency
// count.  Bound by writing n_t * n_recv floats.
constexpr int kSynthTile = 32;
constexpr int kSynthRecv = 4;                   // receivers per thread

struct SynthParams {
    const float2 *p;           // [nf][n_recv] fields
    int64_t n_recv, n_t;
    double freq[GBT_MAX_FREQ], amp_re[GBT_MAX_FREQ], amp_im[GBT_MAX_FREQ];
    double t0, dt;
    float *out;                // [n_t][n_recv]
    int accumulate;
};

template <int NF>
__global__ void __launch_bounds__(256) synth_kernel(const SynthParams p)
{
    __shared__ float2 sph[kSynthTile][NF];
    const int64_t n0 = (int64_t)blockIdx.y * kSynthTile;
    for (int i = threadIdx.x; i < kSynthTile * NF; i += blockDim.x) {
        const int a = i / NF, f = i - a * NF;
        double turns = fma((double)(n0 + a), p.freq[f] * p.dt, p.freq[f] * p.t0);
        turns -= floor(turns);
        float sn, cs;
        sincospif(2.0f * (float)turns, &sn, &cs);
        // A (cos - i sin)
        sph[a][f] = make_float2((float)(p.amp_re[f] * cs + p.amp_im[f] * sn),
                                (float)(p.amp_im[f] * cs - p.amp_re[f] * sn));
    }
    __syncthreads();
    const int64_t r = kSynthRecv * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    if (r >= p.n_recv) return;
    const int nr = (int)min((int64_t)kSynthRecv, p.n_recv - r);
    float2 pr[kSynthRecv][NF];
#pragma unroll
    for (int k = 0; k < kSynthRecv; ++k)
#pragma unroll
        for (int f = 0; f < NF; ++f)
            pr[k][f] = k < nr ? p.p[(int64_t)f * p.n_recv + r + k] : make_float2(0.f, 0.f);
    const int na = (int)min((int64_t)kSynthTile, p.n_t - n0);
    float *o = p.out + n0 * p.n_recv + r;
    // 16-byte stores need a row length divisible by four (every row then starts aligned)
    const bool vec = nr == kSynthRecv && !p.accumulate && (p.n_recv & 3) == 0 &&
                     ((uintptr_t)p.out & 15u) == 0;
    for (int a = 0; a < na; ++a) {
        float acc[kSynthRecv];
#pragma unroll
        for (int k = 0; k < kSynthRecv; ++k) acc[k] = 0.f;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const float2 q = sph[a][f];
#pragma unroll
            for (int k = 0; k < kSynthRecv; ++k)
                acc[k] = fmaf(q.x, pr[k][f].x, fmaf(-q.y, pr[k][f].y, acc[k]));
        }
        float *row = o + a * p.n_recv;
        if (vec) {
            __stcs(reinterpret_cast<float4 *>(row), make_float4(acc[0], acc[1], acc[2], acc[3]));
        } else {
            for (int k = 0; k < nr; ++k) row[k] = p.accumulate ? row[k] + acc[k] : acc[k];
        }
    }
}

struct ReduceParams {
    int64_t n;                 // nf * n_recv
    int64_t n_recv;
    int perm[GBT_MAX_FREQ];    // partial frequency slot -> output frequency
    int splits;
    const float4 *p32;
    const double2 *p64;
    float2 *out;
    int accumulate;
};

__global__ void reduce_kernel(ReduceParams p)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    // splits in order (the sums are the same whatever the unrolling); unrolled so the
    // independent loads are in flight together
    const int64_t f = i / p.n_recv, r = i - f * p.n_recv;
    const int64_t oi = (int64_t)p.perm[f] * p.n_recv + r;
    if (p.p32) {
        // float-float partials (hi, running FP32 sum of errors) merged into a float-float
        // total with error-free FP32 sums: about 44 bits, far beyond the complex64 output,
        // and no FP64 arithmetic (GB300 issues FP64 at a small fraction of the FP32 rate)
        const float4 *src = p.p32 + i;
        float rh = 0.0f, rl = 0.0f, ih = 0.0f, il = 0.0f;
#pragma unroll 8
        for (int s = 0; s < p.splits; ++s) {
            const float4 v = __ldcs(src + (int64_t)s * p.n);
            float t, e;
            two_sum(rh, v.x, t, e);
            rh = t;
            rl = __fadd_rn(rl, __fadd_rn(e, v.z));
            two_sum(ih, v.y, t, e);
            ih = t;
            il = __fadd_rn(il, __fadd_rn(e, v.w));
        }
        if (p.accumulate) {
            const float2 o = p.out[oi];
            float t, e;
            two_sum(rh, o.x, t, e);
            rh = t;
            rl = __fadd_rn(rl, e);
            two_sum(ih, o.y, t, e);
            ih = t;
            il = __fadd_rn(il, e);
        }
        p.out[oi] = make_float2(__fadd_rn(rh, rl), __fadd_rn(ih, il));
        return;
    }
    double re = 0.0, im = 0.0;
    {
        const double2 *src = p.p64 + i;
#pragma unroll 8
        for (int s = 0; s < p.splits; ++s) {
            const double2 v = src[(int64_t)s * p.n];
            re += v.x;
            im += v.y;
        }
    }
    if (p.accumulate) {
        const float2 o = p.out[oi];
        re += (double)o.x;
        im += (double)o.y;
    }
    p.out[oi] = make_float2((float)re, (float)im);
}

// ------------------------------------------------------ receiver order --

__device__ __forceinline__ unsigned int ordered_bits(float f)
{
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(unsigned int u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void bbox_kernel(const float *recv, int64_t n, unsigned int *bb)
{
    __shared__ unsigned int lo[3], hi[3];
    if (threadIdx.x < 3) { lo[threadIdx.x] = 0xffffffffu; hi[threadIdx.x] = 0u; }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            unsigned int u = ordered_bits(recv[3 * i + a]);
            atomicMin(&lo[a], u);
            atomicMax(&hi[a], u);
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&bb[threadIdx.x], lo[threadIdx.x]);
        atomicMax(&bb[3 + threadIdx.x], hi[threadIdx.x]);
    }
}

__device__ __forceinline__ unsigned int spread10(unsigned int v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void morton_kernel(const float *recv, int64_t n, int64_t npad, const unsigned int *bb,
                              unsigned long long *keys)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    if (i >= n) { keys[i] = ~0ull; return; }
    unsigned int code = 0;
    for (int a = 0; a < 3; ++a) {
        const float lo = from_ordered(bb[a]), hi = from_ordered(bb[3 + a]);
        const float span = hi - lo;
        float u = span > 0.f ? (recv[3 * i + a] - lo) / span : 0.f;
        unsigned int q = (unsigned int)fminf(fmaxf(u * 1023.0f, 0.0f), 1023.0f);
        code |= spread10(q) << a;
    }
    keys[i] = ((unsigned long long)code << 32) | (unsigned long long)i;
}

__global__ void bitonic_step(unsigned long long *keys, int64_t npad, int64_t j, int64_t k)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    const int64_t l = i ^ j;
    if (l > i) {
        const unsigned long long a = keys[i], b = keys[l];
        const bool up = (i & k) == 0;
        if ((a > b) == up) { keys[i] = b; keys[l] = a; }
    }
}

// ---- stable LSD radix sort of the (Morton code, index) keys on the code's 30 bits,
// 8 bits per pass: the same order as sorting the whole keys, in O(n) per pass
constexpr int kRadixBlock = 1024;   // keys per block, one per thread
constexpr int kRadixBuckets = 256;

__device__ __forceinline__ unsigned int radix_digit(unsigned long long key, int shift)
{
    return (unsigned int)(key >> (32 + shift)) & (kRadixBuckets - 1);
}

// counts[d * nblocks + block]: keys of the block with digit d
__global__ void __launch_bounds__(kRadixBlock) radix_count_kernel(const unsigned long long *keys,
                                                                  int64_t n, int shift,
                                                                  uint32_t *counts, int64_t nblocks)
{
    __shared__ uint32_t c[kRadixBuckets];
    if (threadIdx.x < kRadixBuckets) c[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kRadixBlock + threadIdx.x;
    if (i < n) atomicAdd(&c[radix_digit(keys[i], shift)], 1u);
    __syncthreads();
    if (threadIdx.x < kRadixBuckets) counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = c[threadIdx.x];
}

// One block: exclusive scan of the counts in place (digit-major, then block).
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t *counts, int64_t total)
{
    __shared__ int64_t ws[33];
    int64_t carry = 0;
    for (int64_t base = 0; base < total; base += 1024) {
        const int64_t c = base + threadIdx.x;
        const int64_t v = c < total ? counts[c] : 0;
        int64_t excl;
        const int64_t tot = block_scan_1024(v, excl, ws);
        if (c < total) counts[c] = (uint32_t)(carry + excl);
        carry += tot;
    }
}

// Stable scatter: rank within the warp from the lanes holding the same digit, then the
// counts of earlier warps of the block, then the scanned offset of (digit, block).
__global__ void __launch_bounds__(kRadixBlock) radix_scatter_kernel(const unsigned long long *in,
                                                                    unsigned long long *out,
                                                                    int64_t n, int shift,
                                                                    const uint32_t *offs,
                                                                    int64_t nblocks)
{
    __shared__ uint32_t wc[kRadixBlock / 32][kRadixBuckets];
    for (int q = threadIdx.x; q < (kRadixBlock / 32) * kRadixBuckets; q += kRadixBlock)
        (&wc[0][0])[q] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kRadixBlock + threadIdx.x;
    const bool ok = i < n;
    const unsigned long long key = ok ? in[i] : 0ull;
    const unsigned int d = ok ? radix_digit(key, shift) : (unsigned int)kRadixBuckets;
    const unsigned int same = __match_any_sync(0xffffffffu, d);
    const unsigned int rank = __popc(same & ((1u << lane) - 1u));
    if (ok && rank == 0) wc[wid][d] = __popc(same);
    __syncthreads();
    if (threadIdx.x < kRadixBuckets) {
        uint32_t run = 0u;
        for (int w = 0; w < kRadixBlock / 32; ++w) {
            const uint32_t c = wc[w][threadIdx.x];
            wc[w][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    if (ok) out[offs[(int64_t)d * nblocks + blockIdx.x] + wc[wid][d] + rank] = key;
}

__global__ void extract_order(const unsigned long long *keys, int64_t n, int32_t *order)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) order[i] = (int32_t)(keys[i] & 0xffffffffull);
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The 32-byte cull records follow the 80-byte records in a sum's record region.
float4 *cull_records(const float *rec, int64_t capacity)
{
    return reinterpret_cast<float4 *>(
        reinterpret_cast<char *>(const_cast<float *>(rec)) +
        align_up((size_t)kRecFloats * (size_t)capacity * sizeof(float), 256));
}

template <int NF, int WINDOW, int MODE, bool BATCHED = false, bool LOSSY = false>
void launch_fwd_t(const FwdParams &p, cudaStream_t s, bool timed)
{
    constexpr bool STATS = MODE != kFwd;
    using Cfg = PairCfg<NF, MODE, BATCHED, LOSSY>;
    const size_t smem = Cfg::kSmem;
    const int threads = 32 * Cfg::kWarps;
    GBT_CUDA(cudaFuncSetAttribute(gbs_fwd_kernel<NF, WINDOW, MODE, BATCHED, LOSSY>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GBT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, gbs_fwd_kernel<NF, WINDOW, MODE, BATCHED, LOSSY>, threads, smem));
    if (per_sm < 1) fail(GBT_ERR_UNSUPPORTED, "GBS kernel does not fit on one SM");
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((p.n_items + Cfg::kWarps - 1) / Cfg::kWarps,
                             (int64_t)std::max(per_sm, 1) * num_sms()));
    GBT_CUDA(cudaMemsetAsync(p.work_counter, 0, sizeof(int), s));
    if (MODE != kStats && timed) timing_begin(s);
    gbs_fwd_kernel<NF, WINDOW, MODE, BATCHED, LOSSY><<<grid, threads, smem, s>>>(p);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
    if (MODE != kStats && timed) timing_end(s);
    (void)STATS;
}

template <int NF, int WINDOW>
void launch_fwd(const FwdParams &p, cudaStream_t s, bool timed)
{
    if (p.grad_out) launch_fwd_t<NF, WINDOW, kBwd>(p, s, timed);
    else if (p.stats) launch_fwd_t<NF, WINDOW, kStats>(p, s, timed);
    else launch_fwd_t<NF, WINDOW, kFwd>(p, s, timed);
}

// With losses (seg_rf set) the forward and adjoint launches take the lossy kernel,
// instantiated for 1, 2, 4 and 8 frequency slots; counting needs no losses.
template <int NF, int WINDOW>
void launch_fwd_lossy(const FwdParams &p, cudaStream_t s, bool timed)
{
    if (p.grad_out) launch_fwd_t<NF, WINDOW, kBwd, false, true>(p, s, timed);
    else launch_fwd_t<NF, WINDOW, kFwd, false, true>(p, s, timed);
}

template <int WINDOW>
void launch_fwd_nf(const FwdParams &p, cudaStream_t s, bool timed = true)
{
    if (p.seg_rf && !p.stats) {
        if (p.nf <= 1) launch_fwd_lossy<1, WINDOW>(p, s, timed);
        else if (p.nf <= 2) launch_fwd_lossy<2, WINDOW>(p, s, timed);
        else if (p.nf <= 4) launch_fwd_lossy<4, WINDOW>(p, s, timed);
        else if (p.nf <= 8) launch_fwd_lossy<8, WINDOW>(p, s, timed);
        else fail(GBT_ERR_UNSUPPORTED, "pair kernel launched with more than 8 frequencies");
        return;
    }
    if (p.nf <= 1) launch_fwd<1, WINDOW>(p, s, timed);
    else if (p.nf <= 2) launch_fwd<2, WINDOW>(p, s, timed);
    else if (p.nf <= 4) launch_fwd<4, WINDOW>(p, s, timed);
    else if (p.nf <= 6) launch_fwd<6, WINDOW>(p, s, timed);
    else if (p.nf <= 8) launch_fwd<8, WINDOW>(p, s, timed);
    else fail(GBT_ERR_UNSUPPORTED, "pair kernel launched with more than 8 frequencies");
}

// Frequency processing order: when every b is equal, sorted by k so that the kept
// frequencies of a pair form a prefix (wider beams first); otherwise as given.
// perm[slot] = user frequency index.  Returns whether b is uniform.
bool freq_order(const gbt_sum_args &a, int (&perm)[GBT_MAX_FREQ])
{
    for (int f = 0; f < GBT_MAX_FREQ; ++f) perm[f] = f;
    bool uniform = true;
    for (int f = 1; f < a.n_freq; ++f) uniform = uniform && a.beam_b[f] == a.beam_b[0];
    if (uniform)
        std::stable_sort(perm, perm + a.n_freq,
                         [&](int x, int y) { return a.freq_hz[x] < a.freq_hz[y]; });
    return uniform;
}

// Frequencies go through the pair kernel in groups of at most kGroupFreq slots of
// the processing order; the kernel is instantiated for up to that many.
constexpr int kGroupFreq = 8;

// Kernel parameters shared by the forward, counting and adjoint launches, for the
// frequency group that starts at processing slot g0 (fperm maps the group's slots to
// user frequency indices).
FwdParams make_pair_params(const TraceDev &td, const SceneDev &sd, const gbt_sum_args &a,
                           const float *rec, int g0 = 0)
{
    FwdParams q{};
    q.recv = a.recv; q.order = a.recv_order; q.n_recv = a.n_recv;
    q.n_seg_ptr = td.ray_off + td.n_rays;
    q.rec = rec;
    q.crec = cull_records(rec, td.capacity);
    q.nf = std::min(kGroupFreq, a.n_freq - g0);
    q.cutoff = (float)a.cutoff;
    q.tile_cull = a.tile_cull ? 1 : 0;
    int perm[GBT_MAX_FREQ];
    q.uniform_b = freq_order(a, perm) ? 1 : 0;
    double amin = 1e300, bmax = 0.0, kmax = 0.0;
    for (int f = 0; f < GBT_MAX_FREQ; ++f) q.fperm[f] = f;
    for (int f = 0; f < q.nf; ++f) {
        const int g = perm[g0 + f];
        q.fperm[f] = g;
        const double K = a.freq_hz[g] / sd.c;       // turns per metre
        const double k = 2.0 * kPi * K;
        const double b = a.beam_b[g];
        FreqConst &c = q.fc[f];
        c.K_hi = (float)K;
        c.K_lo = (float)(K - (double)c.K_hi);
        c.halfK = (float)(0.5 * K);
        c.kb2 = (float)(0.5 * k * b);
        c.kb2l2e = (float)(0.5 * k * b * 1.4426950408889634);
        c.b = (float)b;
        c.b2 = (float)(b * b);
        c.scale = (float)(k * b / (8.0 * kPi * kPi));
        c.kh = (float)(0.5 * k);
        c.invb = (float)(1.0 / b);
        c.al2e = (float)(a.absorption[g] * 1.4426950408889634);
        amin = std::min(amin, 0.5 * k * b);
        bmax = std::max(bmax, b * b);
        kmax = std::max(kmax, K);
    }
    q.kmax_turns = (float)kmax;
    q.pre_alpha = (float)(amin / (a.cutoff + 1.0));
    q.pre_beta = (float)bmax;
    q.status = status_word();
    return q;
}

}  // namespace

bool has_losses(const gbt_sum_args &a)
{
    if (a.flow_resistivity) return true;
    for (int f = 0; f < a.n_freq; ++f)
        if (a.absorption[f] != 0.0) return true;
    return false;
}

// Per (frequency, segment) loss factors of a sum: (log2 |R|, arg R / 2 pi) floats for the
// F32 path, complex doubles for the F64 path; none without losses.
static size_t loss_bytes(const TraceDev &td, const gbt_sum_args &a)
{
    if (!has_losses(a)) return 0;
    const size_t per = a.precision == GBT_PRECISION_F64 ? sizeof(double2) : sizeof(float2);
    return align_up((size_t)a.n_freq * (size_t)td.capacity * per, 256);
}

int choose_splits(const TraceDev &td, const gbt_sum_args &a)
{
    if (a.seg_split > 0) return a.seg_split;
    const int64_t nseg_est = td.n_seg_host >= 0 ? td.n_seg_host : td.capacity;
    if (a.precision == GBT_PRECISION_F64) {
        const int64_t tiles = (a.n_recv + kThreads64 - 1) / kThreads64;
        int64_t s = (4 * (int64_t)num_sms() + tiles - 1) / (tiles > 0 ? tiles : 1);
        s = std::max<int64_t>(1, std::min<int64_t>(s, (nseg_est + kTS64 - 1) / kTS64));
        return (int)std::min<int64_t>(s, 4096);
    }
    // items are (warp tile, split): about 16 per resident warp, 32 with the pre-cull (its
    // item costs vary more), so that the last items to finish are short ones
    const int64_t wtiles = std::max<int64_t>(1, (a.n_recv + kCtaRecv - 1) / kCtaRecv) * kTileWarps;
    const int64_t warps = (int64_t)num_sms() * kWarpsFwd;
    const int64_t per_warp = a.tile_cull ? 32 : 16;
    int64_t s = (per_warp * warps + wtiles - 1) / wtiles;
    s = std::max<int64_t>(1, std::min<int64_t>(s, (nseg_est + kBatch - 1) / kBatch));
    // partial sums stay under ~1 GiB
    const int64_t per_split = (int64_t)a.n_freq * std::max<int64_t>(a.n_recv, 1) * 16;
    s = std::min<int64_t>(s, std::max<int64_t>(1, (1LL << 30) / per_split));
    return (int)std::min<int64_t>(s, 4096);
}

static int64_t cta_tiles(int64_t n_recv) { return (n_recv + kCtaRecv - 1) / kCtaRecv; }

// Tile workspace: balls, weights and the dispatch permutation (heaviest tiles
// first), plus, with the tile pre-cull, the per-tile segment lists.
struct TileWs {
    float4 *ball = nullptr;
    float4 *rball = nullptr;       // the balls with their share of the list test's slack
    unsigned int *weight = nullptr;
    int32_t *perm = nullptr;
    int32_t *counts = nullptr;     // [tiles][chunks]: counts, then offsets within the tile
    int64_t *list_off = nullptr;
    int32_t *list_n = nullptr;
    int32_t *list = nullptr;
    uint32_t *words = nullptr;     // per 32-entry list chunk: one word per warp tile
    float4 *wball = nullptr;       // per warp tile: bounding ball
    uint32_t *bits = nullptr;      // [tiles][chunks * 32]: the counting pass's ballots, or null
    int64_t tiles = 0, chunks = 0, cap = 0, wtiles = 0;
    bool order = false, lists = false;
    size_t bytes = 0;              // workspace the layout needs
};

std::atomic<int64_t> g_list_cap_limit{0};   // set_list_capacity (0: the default)

static TileWs tile_ws_layout(void *ws, int64_t n_recv, int64_t seg_capacity, bool tile_cull)
{
    TileWs t;
    t.tiles = cta_tiles(n_recv);
    t.order = t.tiles >= 2 && t.tiles <= kMaxOrderedTiles;
    t.lists = tile_cull && t.tiles >= 1 && t.tiles <= kMaxOrderedTiles && seg_capacity > 0;
    if (!t.order && !t.lists) return t;
    t.chunks = t.lists ? (seg_capacity + kListChunk - 1) / kListChunk : 0;
    // room for an eighth of all (tile, segment) pairs, at least 16M entries
    const int64_t all = t.tiles * seg_capacity;
    // (a multiple of 32: every tile's list starts on a 32-entry chunk boundary)
    t.cap = t.lists ? std::min<int64_t>(all, std::max<int64_t>(int64_t(1) << 24, all / 8)) : 0;
    const int64_t limit = g_list_cap_limit.load();
    if (limit > 0) t.cap = std::min(t.cap, limit);
    t.cap = (t.cap + 31) / 32 * 32;
    t.wtiles = (n_recv + kWarpRecv - 1) / kWarpRecv;
    char *w = static_cast<char *>(ws);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *r = w ? w + off : nullptr;
        off += align_up(bytes, 256);
        return r;
    };
    t.ball = reinterpret_cast<float4 *>(take((size_t)t.tiles * sizeof(float4)));
    t.rball = reinterpret_cast<float4 *>(take((size_t)t.tiles * sizeof(float4)));
    t.weight = reinterpret_cast<unsigned int *>(take((size_t)t.tiles * sizeof(unsigned int)));
    t.perm = reinterpret_cast<int32_t *>(take((size_t)t.tiles * sizeof(int32_t)));
    if (t.lists) {
        t.counts = reinterpret_cast<int32_t *>(take((size_t)(t.tiles * t.chunks) * sizeof(int32_t)));
        t.list_off = reinterpret_cast<int64_t *>(take((size_t)t.tiles * sizeof(int64_t)));
        t.list_n = reinterpret_cast<int32_t *>(take((size_t)t.tiles * sizeof(int32_t)));
        t.list = reinterpret_cast<int32_t *>(take((size_t)t.cap * sizeof(int32_t)));
        t.words = reinterpret_cast<uint32_t *>(take((size_t)(t.cap / 32) * kChunkWords * sizeof(uint32_t)));
        t.wball = reinterpret_cast<float4 *>(take((size_t)t.wtiles * sizeof(float4)));
        // the ballots, unless they would take more than 4 GiB (then the write pass repeats
        // the ball tests)
        const size_t bb = (size_t)t.tiles * (size_t)t.chunks * 32 * sizeof(uint32_t);
        if (bb <= (size_t(1) << 32)) t.bits = reinterpret_cast<uint32_t *>(take(bb));
    }
    t.bytes = off;
    return t;
}

static size_t tile_ws_bytes(int64_t n_recv, int64_t seg_capacity, bool tile_cull)
{
    return tile_ws_layout(nullptr, n_recv, seg_capacity, tile_cull).bytes;
}

// Launches the tile preparation for q's receivers and records (the records must
// be written earlier on s) and points q at its results: the dispatch order and,
// with the pre-cull, the segment lists.  Weights are the exact list sizes when
// the lists are built, else a sampled count.
static void tile_prep_launch(FwdParams &q, int window, const TileWs &t, cudaStream_t s)
{
    if (!t.order && !t.lists) return;
    const int64_t T = t.tiles;
    int64_t n = 0;
    tile_ball_kernel<<<(unsigned)T, 256, 0, s>>>(q.recv, q.order, q.n_recv, t.ball, t.weight, t.rball);
    ++n;
    // tile groups of the chunk-major list passes (each block walks 1 / tg of the tiles):
    // one, since more re-read the chunk's records for every group (measured on the city:
    // 8 groups took list_count 1.77 -> 2.19 ms and list_write_bits 1.58 -> 1.75 ms)
    const unsigned tg = 1;
    if (t.lists) {
        const size_t sm = (size_t)T * sizeof(int32_t);
        if (window == GBT_WINDOW_LINE) {
            GBT_CUDA(cudaFuncSetAttribute(list_count_kernel<GBT_WINDOW_LINE>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            list_count_kernel<GBT_WINDOW_LINE><<<dim3((unsigned)t.chunks, tg), kListChunk, sm, s>>>(
                q.crec, q.n_seg_ptr, t.rball, T, t.chunks, q.pre_alpha, q.pre_beta, t.counts, t.bits);
        } else {
            GBT_CUDA(cudaFuncSetAttribute(list_count_kernel<GBT_WINDOW_SEGMENT>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            list_count_kernel<GBT_WINDOW_SEGMENT><<<dim3((unsigned)t.chunks, tg), kListChunk, sm, s>>>(
                q.crec, q.n_seg_ptr, t.rball, T, t.chunks, q.pre_alpha, q.pre_beta, t.counts, t.bits);
        }
        list_scan_chunks_kernel<<<(unsigned)T, 1024, 0, s>>>(t.counts, t.chunks, t.weight);
        n += 2;
    } else {
        if (window == GBT_WINDOW_LINE)
            tile_weight_kernel<GBT_WINDOW_LINE><<<kWeightSamples / 256, 256, 0, s>>>(
                q.crec, q.n_seg_ptr, t.ball, T, q.pre_alpha, q.pre_beta, t.weight);
        else
            tile_weight_kernel<GBT_WINDOW_SEGMENT><<<kWeightSamples / 256, 256, 0, s>>>(
                q.crec, q.n_seg_ptr, t.ball, T, q.pre_alpha, q.pre_beta, t.weight);
        ++n;
    }
    if (t.order) {
        tile_rank_kernel<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(t.weight, T, t.perm);
        ++n;
        q.tile_perm = t.perm;
    }
    if (t.lists) {
        list_layout_kernel<<<1, 1024, 0, s>>>(t.weight, t.order ? t.perm : nullptr, T, t.cap,
                                              t.list_off, t.list_n);
        warp_ball_kernel<<<(unsigned)((t.wtiles + 7) / 8), 256, 0, s>>>(q.recv, q.order, q.n_recv,
                                                                         t.wtiles, t.wball);
        const dim3 mgrid(128, (unsigned)T);     // many blocks per tile: the gathers overlap
        if (window == GBT_WINDOW_LINE) {
            if (t.bits)
                list_write_bits_kernel<<<dim3((unsigned)t.chunks, tg), kListChunk, 0, s>>>(
                    q.n_seg_ptr, T, t.chunks, t.bits, t.counts, t.list_off, t.list_n, t.list);
            else
                list_write_kernel<GBT_WINDOW_LINE><<<(unsigned)t.chunks, kListChunk, 0, s>>>(
                    q.crec, q.n_seg_ptr, t.rball, T, t.chunks, q.pre_alpha, q.pre_beta, t.counts,
                    t.list_off, t.list_n, t.list);
            list_words_kernel<GBT_WINDOW_LINE><<<mgrid, 256, 0, s>>>(
                q.crec, t.wball, t.wtiles, q.pre_alpha, q.pre_beta, t.list_off, t.list_n, t.list, t.words);
        } else {
            if (t.bits)
                list_write_bits_kernel<<<dim3((unsigned)t.chunks, tg), kListChunk, 0, s>>>(
                    q.n_seg_ptr, T, t.chunks, t.bits, t.counts, t.list_off, t.list_n, t.list);
            else
                list_write_kernel<GBT_WINDOW_SEGMENT><<<(unsigned)t.chunks, kListChunk, 0, s>>>(
                    q.crec, q.n_seg_ptr, t.rball, T, t.chunks, q.pre_alpha, q.pre_beta, t.counts,
                    t.list_off, t.list_n, t.list);
            list_words_kernel<GBT_WINDOW_SEGMENT><<<mgrid, 256, 0, s>>>(
                q.crec, t.wball, t.wtiles, q.pre_alpha, q.pre_beta, t.list_off, t.list_n, t.list, t.words);
        }
        n += 4;
        q.list = t.list;
        q.list_off = t.list_off;
        q.list_n = t.list_n;
        q.list_words = t.words;
    }
    GBT_CUDA(cudaGetLastError());
    note_launches(n);
}

// Kernel records: the 80-byte records, then the 32-byte cull records of the list and
// dispatch-order kernels (sector aligned, a fraction of the size, so they stay in L2).
static size_t records_bytes(const TraceDev &td)
{
    return align_up((size_t)kRecFloats * (size_t)td.capacity * sizeof(float), 256) +
           align_up((size_t)td.capacity * 2 * sizeof(float4), 256);
}


// Prepass of a trace's segments into kernel records (and FP64 amplitudes when amp64 is
// set), with the sum's reflection coefficients and ray weights.
static void prepass_launch(const TraceDev &td, const SceneDev &sd, const gbt_sum_args &a,
                           float *rec, double *amp64, cudaStream_t s, void *loss = nullptr)
{
    if (td.capacity == 0) return;
    PrepParams pp{};
    pp.n_seg_ptr = td.ray_off + td.n_rays;
    pp.o = td.o; pp.t = td.t; pp.L = td.L; pp.s0 = td.s0;
    pp.ray = td.ray; pp.depth = td.depth; pp.bmat = td.bmat;
    pp.gamma = a.gamma;
    pp.weight = a.ray_weight;
    pp.fan = td.fan;
    pp.n_fan = td.n_fan;
    pp.n_materials = sd.n_materials;
    pp.rec = rec;
    pp.crec = cull_records(rec, td.capacity);
    pp.amp64 = amp64;
    pp.status = status_word();
    if (loss) {
        pp.sigma = a.flow_resistivity;
        pp.hit = td.hit;
        pp.tri = sd.tri;
        pp.n_tri = sd.n_tri;
        pp.nf = a.n_freq;
        for (int f = 0; f < a.n_freq; ++f) pp.freq[f] = a.freq_hz[f];
        pp.rf_stride = td.capacity;
        if (a.precision == GBT_PRECISION_F64) pp.seg_r64 = static_cast<double2 *>(loss);
        else pp.seg_rf = static_cast<float2 *>(loss);
    }
    prepass_kernel<<<(unsigned)((td.capacity + 255) / 256), 256, 0, s>>>(pp);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}

size_t sum_workspace_bytes(const TraceDev &td, const gbt_sum_args &a, int splits)
{
    size_t b = records_bytes(td);
    b += align_up((size_t)td.capacity * sizeof(double), 256);               // amp64
    b += 256;                                                               // work counter
    const size_t part = (size_t)splits * a.n_freq * (size_t)a.n_recv;
    b += align_up(part * (a.precision == GBT_PRECISION_F64 ? sizeof(double2) : sizeof(float4)),
                  256);
    if (a.precision != GBT_PRECISION_F64) b += tile_ws_bytes(a.n_recv, td.capacity, a.tile_cull != 0);
    b += loss_bytes(td, a);
    return b;
}

void sum_launch(const TraceDev &td, const SceneDev &sd, const gbt_sum_args &a, int splits,
                void *work, cudaStream_t s, unsigned long long *stats)
{
    char *w = static_cast<char *>(work);
    float *rec = reinterpret_cast<float *>(w);
    w += records_bytes(td);
    double *amp64 = reinterpret_cast<double *>(w);
    w += align_up((size_t)td.capacity * sizeof(double), 256);
    int *counter = reinterpret_cast<int *>(w);
    w += 256;
    void *partial = w;
    w += align_up((size_t)splits * a.n_freq * (size_t)a.n_recv *
                      (a.precision == GBT_PRECISION_F64 ? sizeof(double2) : sizeof(float4)),
                  256);
    void *order_ws = w;
    if (a.precision != GBT_PRECISION_F64) w += tile_ws_bytes(a.n_recv, td.capacity, a.tile_cull != 0);
    void *loss = loss_bytes(td, a) ? static_cast<void *>(w) : nullptr;
    const int32_t *n_seg_ptr = td.ray_off + td.n_rays;

    prepass_launch(td, sd, a, rec, amp64, s, loss);

    if (a.n_recv <= 0) return;
    ReduceParams rp{};
    rp.n_recv = a.n_recv;
    rp.out = reinterpret_cast<float2 *>(a.out);
    rp.accumulate = a.accumulate;
    rp.splits = splits;
    auto reduce = [&]() {
        reduce_kernel<<<(unsigned)((rp.n + 255) / 256), 256, 0, s>>>(rp);
        note_launches(1);
        GBT_CUDA(cudaGetLastError());
    };
    if (a.precision == GBT_PRECISION_F64) {
        F64Params q{};
        q.recv = a.recv; q.order = a.recv_order; q.n_recv = a.n_recv;
        q.n_seg_ptr = n_seg_ptr;
        q.o = td.o; q.t = td.t; q.L = td.L; q.s0 = td.s0; q.amp = amp64;
        q.nf = a.n_freq;
        q.cutoff = a.cutoff;
        for (int f = 0; f < a.n_freq; ++f) {
            q.k[f] = 2.0 * kPi * a.freq_hz[f] / sd.c;
            q.b[f] = a.beam_b[f];
        }
        q.splits = splits;
        q.partial = reinterpret_cast<double2 *>(partial);
        for (int f = 0; f < a.n_freq; ++f) q.absorb[f] = a.absorption[f];
        q.r64 = static_cast<const double2 *>(loss);
        q.r64_stride = td.capacity;
        dim3 grid((unsigned)((a.n_recv + kThreads64 - 1) / kThreads64), (unsigned)splits);
        if (a.window == GBT_WINDOW_LINE) launch_f64<GBT_WINDOW_LINE>(q, grid, s);
        else launch_f64<GBT_WINDOW_SEGMENT>(q, grid, s);
        note_launches(1);
        GBT_CUDA(cudaGetLastError());
        rp.n = (int64_t)a.n_freq * a.n_recv;
        for (int f = 0; f < GBT_MAX_FREQ; ++f) rp.perm[f] = f;
        rp.p64 = reinterpret_cast<double2 *>(partial);
        reduce();
        return;
    }
    // F32: one pair launch and one merge per group of at most 8 frequencies, each
    // group with its own partials (split-major within the group) and output rows
    for (int g0 = 0; g0 < a.n_freq; g0 += kGroupFreq) {
        FwdParams q = make_pair_params(td, sd, a, rec, g0);
        q.splits = splits;
        q.partial = reinterpret_cast<float4 *>(partial) + (int64_t)splits * g0 * a.n_recv;
        q.stats = stats;
        q.seg_rf = static_cast<const float2 *>(loss);
        q.rf_stride = td.capacity;
        q.n_items = cta_tiles(a.n_recv) * kTileWarps * splits;
        q.work_counter = counter;
        tile_prep_launch(q, a.window, tile_ws_layout(order_ws, a.n_recv, td.capacity, a.tile_cull != 0), s);
        if (a.window == GBT_WINDOW_LINE) launch_fwd_nf<GBT_WINDOW_LINE>(q, s);
        else launch_fwd_nf<GBT_WINDOW_SEGMENT>(q, s);
        if (stats) continue;
        rp.n = (int64_t)q.nf * a.n_recv;
        for (int f = 0; f < GBT_MAX_FREQ; ++f) rp.perm[f] = q.fperm[f];
        rp.p32 = q.partial;
        reduce();
    }
}

void synth_launch(const float *p, int nf, int64_t n_recv, const double *freq_hz,
                  const double *amp, double t0, double dt, int64_t n_t, float *out,
                  int accumulate, cudaStream_t s)
{
    if (n_recv <= 0 || n_t <= 0) return;
    SynthParams sp{};
    sp.p = reinterpret_cast<const float2 *>(p);
    sp.n_recv = n_recv;
    sp.n_t = n_t;
    for (int f = 0; f < nf; ++f) {
        sp.freq[f] = freq_hz[f];
        sp.amp_re[f] = amp[2 * f];
        sp.amp_im[f] = amp[2 * f + 1];
    }
    sp.t0 = t0;
    sp.dt = dt;
    sp.out = out;
    sp.accumulate = accumulate;
    const int64_t per_block = 256 * kSynthRecv;
    const dim3 grid((unsigned)((n_recv + per_block - 1) / per_block),
                    (unsigned)((n_t + kSynthTile - 1) / kSynthTile));
    switch (nf) {
#define GBT_SYNTH(NFV) \
    case NFV: synth_kernel<NFV><<<grid, 256, 0, s>>>(sp); break;
        GBT_SYNTH(1) GBT_SYNTH(2) GBT_SYNTH(3) GBT_SYNTH(4) GBT_SYNTH(5) GBT_SYNTH(6)
        GBT_SYNTH(7) GBT_SYNTH(8) GBT_SYNTH(9) GBT_SYNTH(10) GBT_SYNTH(11) GBT_SYNTH(12)
        GBT_SYNTH(13) GBT_SYNTH(14) GBT_SYNTH(15) GBT_SYNTH(16)
#undef GBT_SYNTH
    default: fail(GBT_ERR_INVALID_ARG, "synthesis takes 1 .. 16 frequencies");
    }
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}

size_t recv_order_scratch_bytes(int64_t n)
{
    const int64_t nblocks = (n + kRadixBlock - 1) / kRadixBlock;
    return 2 * align_up((size_t)n * sizeof(unsigned long long), 256) +
           align_up((size_t)kRadixBuckets * nblocks * sizeof(uint32_t), 256) + 256;
}

void recv_order_launch(const float *recv, int64_t n, int32_t *order, void *scratch, cudaStream_t s)
{
    if (n <= 0) return;
    const int64_t nblocks = (n + kRadixBlock - 1) / kRadixBlock;
    char *w = static_cast<char *>(scratch);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(w);
    w += align_up((size_t)n * sizeof(unsigned long long), 256);
    unsigned long long *tmp = reinterpret_cast<unsigned long long *>(w);
    w += align_up((size_t)n * sizeof(unsigned long long), 256);
    uint32_t *counts = reinterpret_cast<uint32_t *>(w);
    w += align_up((size_t)kRadixBuckets * nblocks * sizeof(uint32_t), 256);
    unsigned int *bb = reinterpret_cast<unsigned int *>(w);
    GBT_CUDA(cudaMemsetAsync(bb, 0xff, 3 * sizeof(unsigned int), s));
    GBT_CUDA(cudaMemsetAsync(bb + 3, 0x00, 3 * sizeof(unsigned int), s));
    bbox_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(recv, n, bb);
    note_launches(1);
    morton_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(recv, n, n, bb, keys);
    note_launches(1);
    for (int shift = 0; shift < 30; shift += 8) {   // 30-bit codes: four passes
        radix_count_kernel<<<(unsigned)nblocks, kRadixBlock, 0, s>>>(keys, n, shift, counts, nblocks);
        radix_scan_kernel<<<1, 1024, 0, s>>>(counts, (int64_t)kRadixBuckets * nblocks);
        radix_scatter_kernel<<<(unsigned)nblocks, kRadixBlock, 0, s>>>(keys, tmp, n, shift, counts,
                                                                         nblocks);
        note_launches(3);
        std::swap(keys, tmp);
    }
    extract_order<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, order);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}


// ------------------------------------------------------------ adjoint --

static size_t bwd_layout(const TraceDev &td, const gbt_sum_args &a, const SceneDev *sd,
                         size_t *off)
{
    // records | amp64 | counter | seg_G | seg_H | acc | tile order | losses
    size_t b = 0;
    off[0] = b; b += records_bytes(td);
    off[1] = b; b += align_up((size_t)td.capacity * sizeof(double), 256);
    off[2] = b; b += 256;
    off[3] = b; b += align_up((size_t)td.capacity * sizeof(float), 256);
    off[4] = b; b += align_up((size_t)a.n_freq * td.capacity * sizeof(float), 256);
    off[5] = b; b += align_up((size_t)((sd ? sd->n_materials : 1024) + GBT_MAX_FREQ) * sizeof(double), 256);
    off[6] = b; b += tile_ws_bytes(a.n_recv, td.capacity, a.tile_cull != 0);
    off[7] = b; b += loss_bytes(td, a);
    return b;
}

size_t bwd_workspace_bytes(const TraceDev &td, const gbt_sum_args &a)
{
    size_t off[8];
    return bwd_layout(td, a, &td.scene->d, off);
}

void bwd_launch(const TraceDev &td, const SceneDev &sd, const gbt_sum_args &a,
                const float *grad_out, float *grad_gamma, float *grad_w, double *grad_b,
                void *work, cudaStream_t s)
{
    size_t off[8];
    bwd_layout(td, a, &sd, off);
    char *w = static_cast<char *>(work);
    float *rec = reinterpret_cast<float *>(w + off[0]);
    double *amp64 = reinterpret_cast<double *>(w + off[1]);
    int *counter = reinterpret_cast<int *>(w + off[2]);
    float *seg_G = reinterpret_cast<float *>(w + off[3]);
    float *seg_H = reinterpret_cast<float *>(w + off[4]);
    double *acc = reinterpret_cast<double *>(w + off[5]);

    GBT_CUDA(cudaMemsetAsync(seg_G, 0, (size_t)td.capacity * sizeof(float), s));
    GBT_CUDA(cudaMemsetAsync(seg_H, 0, (size_t)a.n_freq * td.capacity * sizeof(float), s));
    GBT_CUDA(cudaMemsetAsync(acc, 0, (size_t)(sd.n_materials + GBT_MAX_FREQ) * sizeof(double), s));
    if (grad_w) GBT_CUDA(cudaMemsetAsync(grad_w, 0, (size_t)td.n_fan * sizeof(float), s));

    void *loss = loss_bytes(td, a) ? static_cast<void *>(w + off[7]) : nullptr;
    prepass_launch(td, sd, a, rec, amp64, s, loss);
    // per frequency group: seg_G gathers every frequency's terms, seg_H the group's rows
    // (processing slots g0 .. g0 + nf - 1)
    if (a.n_recv > 0) {
        const int splits = choose_splits(td, a);
        for (int g0 = 0; g0 < a.n_freq; g0 += kGroupFreq) {
            FwdParams q = make_pair_params(td, sd, a, rec, g0);
            q.splits = splits;
            q.n_items = cta_tiles(a.n_recv) * kTileWarps * splits;
            q.work_counter = counter;
            q.grad_out = reinterpret_cast<const float2 *>(grad_out);
            q.seg_G = seg_G;
            q.seg_H = seg_H + (int64_t)g0 * td.capacity;
            q.seg_stride = td.capacity;
            q.seg_rf = static_cast<const float2 *>(loss);
            q.rf_stride = td.capacity;
            tile_prep_launch(q, a.window, tile_ws_layout(w + off[6], a.n_recv, td.capacity, a.tile_cull != 0), s);
            if (a.window == GBT_WINDOW_LINE) launch_fwd_nf<GBT_WINDOW_LINE>(q, s);
            else launch_fwd_nf<GBT_WINDOW_SEGMENT>(q, s);
        }
    }
    int fperm[GBT_MAX_FREQ];
    freq_order(a, fperm);
    RayGradParams r{};
    r.n_rays = td.n_rays;
    r.ray_begin = td.ray_begin;
    r.ray_off = td.ray_off;
    r.bmat = td.bmat;
    r.gamma = a.gamma;
    r.weight = a.ray_weight;
    r.fan = td.fan;
    r.n_fan = td.n_fan;
    r.seg_G = seg_G;
    r.seg_H = seg_H;
    r.seg_stride = td.capacity;
    r.nf = a.n_freq;
    r.n_materials = sd.n_materials;
    r.grad_w = grad_w;
    r.acc = acc;
    r.status = status_word();
    const size_t sh = (size_t)(sd.n_materials + a.n_freq) * sizeof(double);
    ray_grad_kernel<<<(unsigned)((td.n_rays + 127) / 128), 128, sh, s>>>(r);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
    GradOutParams g{};
    g.acc = acc;
    g.n_materials = sd.n_materials;
    g.nf = a.n_freq;
    for (int f = 0; f < GBT_MAX_FREQ; ++f) g.fperm[f] = fperm[f];
    g.grad_gamma = grad_gamma;
    g.grad_b = grad_b;
    const int nk = sd.n_materials + a.n_freq;
    grad_out_kernel<<<(unsigned)((nk + 127) / 128), 128, 0, s>>>(g);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------ batched --

// Many (trace, sum arguments) instances in one persistent launch: one global
// work counter over the items of all instances (instances ordered by cost,
// longest first), each CTA loading the item's instance parameters.
template <int NF, int WINDOW>
int batched_prepare()
{
    using Cfg = PairCfg<NF, kFwd, true>;
    const size_t smem = Cfg::kSmem;
    GBT_CUDA(cudaFuncSetAttribute(gbs_fwd_kernel<NF, WINDOW, kFwd, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GBT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, gbs_fwd_kernel<NF, WINDOW, kFwd, true>, 32 * Cfg::kWarps, smem));
    if (per_sm < 1) fail(GBT_ERR_UNSUPPORTED, "GBS kernel does not fit on one SM");
    return per_sm;
}

template <int NF, int WINDOW>
void batched_launch(const FwdParams &prm, int grid, cudaStream_t s)
{
    GBT_CUDA(cudaMemsetAsync(prm.work_counter, 0, sizeof(int), s));
    using Cfg = PairCfg<NF, kFwd, true>;
    gbs_fwd_kernel<NF, WINDOW, kFwd, true><<<grid, 32 * Cfg::kWarps, Cfg::kSmem, s>>>(prm);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}

typedef int (*BatchedPrepFn)();
enum { kFused = 0, kConcurrent = 1 };      // how a batch executes
constexpr int kBranches = 4;               // branch streams of a concurrent batch
typedef void (*BatchedLaunchFn)(const FwdParams &, int, cudaStream_t);

struct BatchImpl {
    std::vector<const gbt_trace_t *> traces;
    std::vector<gbt_sum_args> args;
    std::vector<int> order;            // instance processing order (cost, descending)
    std::vector<int64_t> n_seg, cost;
    std::vector<int> splits;
    std::vector<size_t> rec_off, part_off, ord_off, loss_off;
    std::vector<FwdParams> table;      // in processing order
    std::vector<int64_t> inst_off;
    void *work = nullptr;
    size_t work_bytes = 0;
    int *counter = nullptr;
    FwdParams *d_table = nullptr;
    int64_t *d_off = nullptr;
    int grid = 1;
    int nf_max = 1, window = 0;
    BatchedLaunchFn launch = nullptr;
    bool use_graph = false;
    cudaStream_t capture_stream = nullptr;   // private stream the graph is recorded on
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_kernels = 0;               // kernel nodes of the recorded graph
    cudaEvent_t used = nullptr;              // after the latest submit
    // kConcurrent: each instance runs the single-instance pair kernel (parameters
    // in constant space) on one of a few branch streams forked from the submit
    // stream, so one instance's draining tail overlaps the next one's start
    int mode = kFused;
    std::vector<cudaStream_t> branch;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
};

static void batch_plan(BatchImpl &B, double items_per_slot)
{
    // splits per instance: items proportional to the instance's cost
    const int64_t slots = (int64_t)B.grid;
    double total = 0.0;
    for (int64_t c : B.cost) total += (double)std::max<int64_t>(c, 1);
    const int n = (int)B.args.size();
    B.splits.assign(n, 1);
    for (int i = 0; i < n; ++i) {
        const gbt_sum_args &a = B.args[i];
        const int64_t tiles = std::max<int64_t>(1, (a.n_recv + kCtaRecv - 1) / kCtaRecv);
        const double want = items_per_slot * slots * (double)std::max<int64_t>(B.cost[i], 1) / total;
        int64_t sp = (int64_t)std::ceil(want / (double)tiles);
        const int64_t nb = std::max<int64_t>(1, (B.n_seg[i] + kBatch - 1) / kBatch);
        sp = std::max<int64_t>(1, std::min<int64_t>(sp, nb));
        const int64_t per_split = (int64_t)a.n_freq * std::max<int64_t>(a.n_recv, 1) * 16;
        sp = std::min<int64_t>(sp, std::max<int64_t>(1, (1LL << 30) / per_split));
        B.splits[i] = (int)std::min<int64_t>(sp, 4096);
    }
}

// Concurrent batches split each instance as a single sum would.
static void batch_plan_concurrent(BatchImpl &B)
{
    const int n = (int)B.args.size();
    B.splits.assign(n, 1);
    for (int i = 0; i < n; ++i) B.splits[i] = choose_splits(B.traces[i]->d, B.args[i]);
}

static void batch_layout(BatchImpl &B, cudaStream_t s)
{
    const int n = (int)B.args.size();
    B.rec_off.assign(n, 0);
    B.part_off.assign(n, 0);
    B.ord_off.assign(n, 0);
    B.loss_off.assign(n, 0);
    size_t b = 0;
    for (int i = 0; i < n; ++i) {
        B.rec_off[i] = b;
        b += records_bytes(B.traces[i]->d);
        B.part_off[i] = b;
        b += align_up((size_t)B.splits[i] * B.args[i].n_freq * (size_t)B.args[i].n_recv *
                          sizeof(float4), 256);
        B.ord_off[i] = b;
        b += tile_ws_bytes(B.args[i].n_recv, B.traces[i]->d.capacity, B.args[i].tile_cull != 0);
        B.loss_off[i] = b;
        b += loss_bytes(B.traces[i]->d, B.args[i]);
    }
    const size_t cnt = align_up((size_t)n * sizeof(int), 256);    // one work counter per instance
    const size_t tab = align_up((size_t)n * sizeof(FwdParams), 256);
    const size_t off = align_up((size_t)(n + 1) * sizeof(int64_t), 256);
    const size_t need = b + cnt + tab + off;
    if (need > B.work_bytes) {
        if (B.work) dfree(B.work, s);
        B.work = dalloc(need, s);
        B.work_bytes = need;
    }
    char *w = static_cast<char *>(B.work);
    B.counter = reinterpret_cast<int *>(w + b);
    B.d_table = reinterpret_cast<FwdParams *>(w + b + cnt);
    B.d_off = reinterpret_cast<int64_t *>(w + b + cnt + tab);

    B.table.clear();
    B.inst_off.assign(1, 0);
    for (int k = 0; k < n; ++k) {
        const int i = B.order[k];
        const TraceDev &td = B.traces[i]->d;
        const gbt_sum_args &a = B.args[i];
        float *rec = reinterpret_cast<float *>(w + B.rec_off[i]);
        FwdParams q = make_pair_params(td, td.scene->d, a, rec);
        q.splits = B.splits[i];
        q.n_items = cta_tiles(a.n_recv) * kTileWarps * q.splits;
        q.partial = reinterpret_cast<float4 *>(w + B.part_off[i]);
        q.work_counter = B.mode == kConcurrent ? B.counter + k : B.counter;
        if (has_losses(a)) {
            q.seg_rf = reinterpret_cast<const float2 *>(w + B.loss_off[i]);
            q.rf_stride = td.capacity;
        }
        {
            const TileWs t = tile_ws_layout(w + B.ord_off[i], a.n_recv, td.capacity, a.tile_cull != 0);
            q.tile_perm = t.order ? t.perm : nullptr;
            q.list = t.lists ? t.list : nullptr;
            q.list_off = t.lists ? t.list_off : nullptr;
            q.list_n = t.lists ? t.list_n : nullptr;
            q.list_words = t.lists ? t.words : nullptr;
        }
        B.table.push_back(q);
        B.inst_off.push_back(B.inst_off.back() + q.n_items);
    }
    GBT_CUDA(cudaMemcpyAsync(B.d_table, B.table.data(), (size_t)n * sizeof(FwdParams),
                             cudaMemcpyHostToDevice, s));
    GBT_CUDA(cudaMemcpyAsync(B.d_off, B.inst_off.data(), (size_t)(n + 1) * sizeof(int64_t),
                             cudaMemcpyHostToDevice, s));
    GBT_CUDA(cudaStreamSynchronize(s));
}

static void batch_prepass(BatchImpl &B, int i, cudaStream_t s)
{
    const TraceDev &td = B.traces[i]->d;
    char *w = static_cast<char *>(B.work);
    prepass_launch(td, td.scene->d, B.args[i], reinterpret_cast<float *>(w + B.rec_off[i]), nullptr,
                   s, has_losses(B.args[i]) ? static_cast<void *>(w + B.loss_off[i]) : nullptr);
}

// Merge of instance i (processing index k) into its output.
static void batch_reduce(BatchImpl &B, int k, cudaStream_t s)
{
    const int i = B.order[k];
    const gbt_sum_args &a = B.args[i];
    if (a.n_recv == 0) return;
    ReduceParams rp{};
    rp.n = (int64_t)a.n_freq * a.n_recv;
    rp.n_recv = a.n_recv;
    for (int f = 0; f < GBT_MAX_FREQ; ++f) rp.perm[f] = B.table[k].fperm[f];
    rp.splits = B.splits[i];
    rp.p32 = reinterpret_cast<float4 *>(static_cast<char *>(B.work) + B.part_off[i]);
    rp.p64 = nullptr;
    rp.out = reinterpret_cast<float2 *>(a.out);
    rp.accumulate = a.accumulate;
    reduce_kernel<<<(unsigned)((rp.n + 255) / 256), 256, 0, s>>>(rp);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}

// Concurrent form: instances (longest first) dealt round-robin to branch streams
// forked from s and joined back into it; on each branch an instance's prepass,
// tile order, pair kernel and merge follow one another.
static void batch_record_concurrent(BatchImpl &B, cudaStream_t s)
{
    const int n = (int)B.args.size();
    const int nb = std::max(1, std::min(n, kBranches));
    if (B.branch.empty()) {
        B.branch.assign(nb, nullptr);
        B.join.assign(nb, nullptr);
        for (int j = 0; j < nb; ++j) {
            GBT_CUDA(cudaStreamCreateWithFlags(&B.branch[j], cudaStreamNonBlocking));
            GBT_CUDA(cudaEventCreateWithFlags(&B.join[j], cudaEventDisableTiming));
        }
        GBT_CUDA(cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming));
    }
    GBT_CUDA(cudaEventRecord(B.fork, s));
    for (int j = 0; j < nb; ++j) GBT_CUDA(cudaStreamWaitEvent(B.branch[j], B.fork, 0));
    char *w = static_cast<char *>(B.work);
    for (int k = 0; k < n; ++k) {
        const int i = B.order[k];
        cudaStream_t bs = B.branch[k % nb];
        batch_prepass(B, i, bs);
        if (B.args[i].n_recv == 0) continue;
        const FwdParams &q = B.table[k];
        {
            FwdParams qq = q;
            tile_prep_launch(qq, B.window,
                             tile_ws_layout(w + B.ord_off[i], B.args[i].n_recv,
                                            B.traces[i]->d.capacity, B.args[i].tile_cull != 0), bs);
        }
        if (B.window == GBT_WINDOW_LINE) launch_fwd_nf<GBT_WINDOW_LINE>(q, bs, false);
        else launch_fwd_nf<GBT_WINDOW_SEGMENT>(q, bs, false);
        batch_reduce(B, k, bs);
    }
    for (int j = 0; j < nb; ++j) {
        GBT_CUDA(cudaEventRecord(B.join[j], B.branch[j]));
        GBT_CUDA(cudaStreamWaitEvent(s, B.join[j], 0));
    }
}

static void batch_record(BatchImpl &B, cudaStream_t s)
{
    if (B.mode == kConcurrent) {
        batch_record_concurrent(B, s);
        return;
    }
    const int n = (int)B.args.size();
    char *w = static_cast<char *>(B.work);
    for (int i = 0; i < n; ++i) batch_prepass(B, i, s);
    for (int k = 0; k < n; ++k) {
        const int i = B.order[k];
        FwdParams qq = B.table[k];
        tile_prep_launch(qq, B.window,
                         tile_ws_layout(w + B.ord_off[i], B.args[i].n_recv, B.traces[i]->d.capacity,
                                        B.args[i].tile_cull != 0), s);
    }
    FwdParams prm = B.table[0];
    prm.inst = B.d_table;
    prm.inst_off = B.d_off;
    prm.n_inst = n;
    prm.n_items = B.inst_off.back();
    prm.work_counter = B.counter;
    B.launch(prm, B.grid, s);
    for (int k = 0; k < n; ++k) batch_reduce(B, k, s);
}

BatchImpl *batch_create(const gbt_batch_desc &d, cudaStream_t s)
{
    BatchImpl *B = new BatchImpl();
    try {
        // an instance with more than kGroupFreq frequencies becomes one instance per group of
        // consecutive frequencies, each writing its own rows of the caller's output
        for (int i = 0; i < d.n_instances; ++i) {
            const gbt_sum_args &a = d.args[i];
            for (int g0 = 0; g0 < a.n_freq; g0 += kGroupFreq) {
                gbt_sum_args sa = a;
                sa.n_freq = std::min(kGroupFreq, a.n_freq - g0);
                for (int f = 0; f < GBT_MAX_FREQ; ++f) {
                    sa.freq_hz[f] = f < sa.n_freq ? a.freq_hz[g0 + f] : 0.0;
                    sa.beam_b[f] = f < sa.n_freq ? a.beam_b[g0 + f] : 0.0;
                }
                sa.out = a.out + (size_t)g0 * (size_t)a.n_recv * 2;
                B->traces.push_back(d.traces[i]);
                B->args.push_back(sa);
            }
        }
        const int n = (int)B->args.size();
        B->use_graph = d.use_graph != 0;
        B->window = B->args[0].window;
        bool lossy = false;
        for (int i = 0; i < n; ++i) {
            GBT_REQUIRE(B->args[i].window == B->window, "batch instances must share one window");
            GBT_REQUIRE(B->args[i].precision == GBT_PRECISION_F32, "batches are F32 only");
            B->nf_max = std::max(B->nf_max, (int)B->args[i].n_freq);
            lossy = lossy || has_losses(B->args[i]);
        }
        if (lossy && d.form == GBT_BATCH_FUSED)
            fail(GBT_ERR_UNSUPPORTED, "the fused batch form has no losses: use GBT_BATCH_CONCURRENT");
        status_word();   // allocate before any capture
        // segment counts of every trace (each read once its trace is complete)
        B->n_seg.resize(n);
        B->cost.resize(n);
        for (int i = 0; i < n; ++i) {
            const TraceDev &td = B->traces[i]->d;
            const int32_t ns = read_device_i32(td.ray_off + td.n_rays, td.used);
            B->n_seg[i] = ns;
            B->cost[i] = (int64_t)ns * B->args[i].n_recv * B->args[i].n_freq;
        }
        B->order.resize(n);
        for (int i = 0; i < n; ++i) B->order[i] = i;
        std::stable_sort(B->order.begin(), B->order.end(),
                         [&](int x, int y) { return B->cost[x] > B->cost[y]; });
        int per_sm = 1;
        BatchedPrepFn prep = nullptr;
        const int nf = B->nf_max <= 1 ? 1 : B->nf_max <= 2 ? 2 : B->nf_max <= 4 ? 4 : 8;
#define GBT_PICK(NFV)                                                                     \
    if (nf == NFV) {                                                                      \
        prep = B->window == GBT_WINDOW_LINE ? batched_prepare<NFV, GBT_WINDOW_LINE>       \
                                            : batched_prepare<NFV, GBT_WINDOW_SEGMENT>;   \
        B->launch = B->window == GBT_WINDOW_LINE ? batched_launch<NFV, GBT_WINDOW_LINE>   \
                                                 : batched_launch<NFV, GBT_WINDOW_SEGMENT>; \
    }
        GBT_PICK(1) GBT_PICK(2) GBT_PICK(4) GBT_PICK(8)
#undef GBT_PICK
        per_sm = prep();
        B->grid = per_sm * num_sms();
        // candidates: the concurrent form, then the fused launch at a few work
        // granularities (items per resident CTA); 0 items marks the concurrent form
        auto plan = [&](double ips) {
            B->mode = ips > 0.0 ? kFused : kConcurrent;
            if (ips > 0.0) batch_plan(*B, ips);
            else batch_plan_concurrent(*B);
            batch_layout(*B, s);
        };
        // the fused form's default granularity when it is not tuned
        double best_ips = d.form == GBT_BATCH_FUSED ? 32.0 : 0.0;
        std::vector<double> cands;
        if (d.form != GBT_BATCH_FUSED) cands.push_back(0.0);
        if (d.form != GBT_BATCH_CONCURRENT && !lossy)
            for (double v : {4.0, 8.0, 16.0, 32.0}) cands.push_back(v);
        if (d.autotune && cands.size() > 1) {
            float best = 1e30f;
            cudaEvent_t e0, e1;
            GBT_CUDA(cudaEventCreate(&e0));
            GBT_CUDA(cudaEventCreate(&e1));
            try {
                for (double ips : cands) {
                    plan(ips);
                    batch_record(*B, s);   // warm
                    GBT_CUDA(cudaEventRecord(e0, s));
                    batch_record(*B, s);
                    GBT_CUDA(cudaEventRecord(e1, s));
                    GBT_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    GBT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < best) { best = ms; best_ips = ips; }
                }
            } catch (...) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                throw;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        plan(best_ips);
    } catch (...) {
        batch_destroy(B);
        throw;
    }
    return B;
}

static void batch_mark_used(BatchImpl *B, cudaStream_t s)
{
    mark_used(B->used, s);
    for (const gbt_trace_t *t : B->traces) mark_trace_used(t, s);
}

void batch_submit(BatchImpl *B, cudaStream_t s)
{
    if (!B->use_graph) {
        batch_record(*B, s);
        batch_mark_used(B, s);
        return;
    }
    if (!B->exec) {
        // record on a private stream (the caller's may be the legacy default stream,
        // which cannot be captured); the graph is then launched on the caller's stream
        if (!B->capture_stream)
            GBT_CUDA(cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking));
        cudaStream_t cs = B->capture_stream;
        GBT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            batch_record(*B, cs);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        GBT_CUDA(cudaStreamEndCapture(cs, &B->graph));
        GBT_CUDA(cudaGraphInstantiate(&B->exec, B->graph, 0));
        // the launches were counted while recording; later replays add the graph's kernels
        size_t nn = 0;
        GBT_CUDA(cudaGraphGetNodes(B->graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn) GBT_CUDA(cudaGraphGetNodes(B->graph, nodes.data(), &nn));
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            GBT_CUDA(cudaGraphNodeGetType(nd, &t));
            if (t == cudaGraphNodeTypeKernel) ++B->graph_kernels;
        }
    } else {
        note_launches(B->graph_kernels);
    }
    GBT_CUDA(cudaGraphLaunch(B->exec, s));
    batch_mark_used(B, s);
}

void batch_destroy(BatchImpl *B)
{
    if (!B) return;
    // the batch's workspace is freed behind its latest submit; graphs, streams and
    // events may be destroyed while work they launched is still pending
    cudaStream_t q = nullptr;
    try {
        q = after_last_use(B->used);
    } catch (...) {
        cudaDeviceSynchronize();
    }
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->capture_stream) cudaStreamDestroy(B->capture_stream);
    for (cudaStream_t b : B->branch) if (b) cudaStreamDestroy(b);
    for (cudaEvent_t e : B->join) if (e) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->work) dfree(B->work, q);
    if (B->used) cudaEventDestroy(B->used);
    delete B;
}

// ---------------------------------------------------- bounded-wait self test --

// Waits on an mbarrier phase that nothing completes, with the same bounded
// try-wait loop the pair kernel uses; when the limit runs out it flags
// STATUS_TIMEOUT and returns, leaving the context usable.
__global__ void selftest_wait_kernel(long long spins, unsigned int *status)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x != 0) return;
    mbar_init(smem_addr(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    for (long long it = 0; it < spins; ++it)
        if (mbar_try_wait(smem_addr(&bar), 0u)) return;
    atomicOr(status, STATUS_TIMEOUT);
}

void selftest_timeout_launch(long long spins, cudaStream_t s)
{
    selftest_wait_kernel<<<1, 32, 0, s>>>(spins, status_word());
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}

// ------------------------------------------------- receiver order, no allocation --
//
// Some callers cannot allocate device memory at the point where they need a
// receiver order: a host application that owns every device allocation and
// forbids libraries from calling the CUDA allocator, or a latency-critical
// loop (a real-time auralisation thread, for example) that must not call an
// allocator because an allocation may block or fail under memory pressure.
// For them the sort's scratch lives in a fixed device array below.  The array
// is part of the library image: every GPU that loads the library holds it
// (8 MiB + 256 bytes) until the process exits.  Its contents persist between
// calls, so everything that must start at zero is cleared on each call, and
// calls that overlap on the GPU share (and race on) the array.
constexpr int64_t kNoAllocMaxRecv = 1 << 20;
static __device__ __align__(256) unsigned char
    g_order_scratch[kNoAllocMaxRecv * sizeof(unsigned long long) + 256];

namespace {
std::mutex g_order_scratch_mu;
void *g_order_scratch_dev[64] = {};
}  // namespace

void recv_order_noalloc_launch(const float *recv, int64_t n, int32_t *order, cudaStream_t s)
{
    if (n > kNoAllocMaxRecv)
        fail(GBT_ERR_INVALID_ARG, "gbt_recv_order_noalloc handles at most 1048576 receivers (got " +
                                      std::to_string(n) + ")");
    if (n <= 0) return;
    int dev = 0;
    GBT_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(GBT_ERR_UNSUPPORTED, "device index >= 64");
    void *base = nullptr;
    {
        // set-up, once per device, with that device current: the host-side name of
        // the array is not a device address, so ask the runtime for the address
        std::lock_guard<std::mutex> lk(g_order_scratch_mu);
        if (!g_order_scratch_dev[dev]) {
            void *ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_order_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                fail(GBT_ERR_CUDA, std::string("cudaGetSymbolAddress(order scratch): ") +
                                       cudaGetErrorString(e));
            }
            g_order_scratch_dev[dev] = ptr;
        }
        base = g_order_scratch_dev[dev];
    }
    int64_t npad = 1;
    while (npad < n) npad <<= 1;
    unsigned long long *keys = static_cast<unsigned long long *>(base);
    unsigned int *bb = reinterpret_cast<unsigned int *>(
        static_cast<char *>(base) + align_up((size_t)npad * sizeof(unsigned long long), 256));
    GBT_CUDA(cudaMemsetAsync(bb, 0xff, 3 * sizeof(unsigned int), s));
    GBT_CUDA(cudaMemsetAsync(bb + 3, 0x00, 3 * sizeof(unsigned int), s));
    bbox_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(recv, n, bb);
    note_launches(1);
    const unsigned g = (unsigned)((npad + 255) / 256);
    morton_kernel<<<g, 256, 0, s>>>(recv, n, npad, bb, keys);
    note_launches(1);
    for (int64_t k = 2; k <= npad; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            bitonic_step<<<g, 256, 0, s>>>(keys, npad, j, k);
            note_launches(1);
        }
    extract_order<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, order);
    note_launches(1);
    GBT_CUDA(cudaGetLastError());
}

void set_list_capacity(int64_t entries) { g_list_cap_limit.store(entries); }

}  // namespace gbt
