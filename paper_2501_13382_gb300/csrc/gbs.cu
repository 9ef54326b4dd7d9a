// gbs.cu -- Gaussian beam summation (Eq. 3 with the beam of Eq. 1 / Eq. 2)
// for every (receiver, segment, frequency) triple.
//
// GB300 design (FP32 path):
//  * Receivers are processed in a spatially coherent order (Morton order of
//    their positions), 512 per CTA (256 threads x 2), held in registers both
//    absolute (for the exact path) and relative to the CTA's first receiver
//    (for the prefilter, which keeps every quantity small and the expansion
//    |x - o|^2 = |x'|^2 - 2 x'.o' + |o'|^2 well conditioned).
//  * Segments stream through shared memory in tiles of 128; each CTA covers
//    one receiver tile and one of `splits` contiguous segment ranges, so the
//    grid fills all SMs whatever the receiver count.
//  * Prefilter (every pair, frequency independent): s_loc, s, n^2 and the
//    union of the per-frequency Gaussian cutoffs, conservative by one unit of
//    the exponent and 1 cm of window, 13-15 FP32/ALU instructions per pair.
//    The keep bit goes into a 32-bit mask per receiver (one funnel shift),
//    so no divergent branch sits in the pair loop.
//  * Survivors (typically 0.1-5 % of pairs) are then visited in segment order
//    by scanning the mask, and evaluated exactly: float-float differences and
//    dot products give s to ~1e-12 relative; the phase k s is reduced modulo
//    one turn in float-float before the FP32 MUFU sin/cos; n^2 comes from a
//    compensated cross product.  Per-tile FP32 partial sums are folded into
//    float-float accumulators in shared memory, and the segment ranges are
//    merged in FP64 in a fixed order by a second kernel (deterministic).
#include <math.h>

#include "gbt_internal.h"

namespace gbt {
namespace {

constexpr int kThreads = 256;
constexpr int kR = 2;                       // receivers per thread
constexpr int kTileRecv = kThreads * kR;    // receivers per CTA
constexpr int kTS = 128;                    // segments per shared-memory tile
constexpr float kWinMargin = 0.01f;         // prefilter window slack (m)
constexpr int kMaxNF = 8;

struct FreqConst {
    float K_hi, K_lo;     // f / c in turns per metre, float-float
    float halfK;          // K / 2: second phase term K n^2 s / (2 D) in turns
    float kb2;            // k b / 2  (Gaussian exponent factor)
    float kb2l2e;         // k b / 2 * log2(e)
    float b, b2;          // b, b^2
    float scale;          // k b / (8 pi^2)
};

struct FwdParams {
    const float *recv;
    const int32_t *order;
    int64_t n_recv;
    const int32_t *n_seg_ptr;
    const float *rec;          // SoA records, field f at rec + f * stride
    int64_t stride;
    int nf;
    float cutoff;
    float pre_alpha, pre_beta; // prefilter: keep iff alpha n^2 <= s^2 + beta
    int splits;
    int n_items;               // receiver tiles x splits
    int *work_counter;         // zeroed before launch; CTAs take items from it
    float4 *partial;           // [splits][nf][n_recv]: re_hi, im_hi, re_lo, im_lo
    unsigned long long *stats; // counting mode when non-null: [1] prefiltered, [2] kept
    FreqConst fc[GBT_MAX_FREQ];
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bv = s - a;
    e = (a - (s - bv)) + (b - bv);
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
    float w = c * d;
    float e = fmaf(-c, d, w);
    float f = fmaf(a, b, -w);
    return f + e;
}

struct ColdSmem {
    float f[14][kTS];   // oxh oyh ozh oxl oyl ozl txl tyl tzl s0h s0l Lh Ll amp
};
enum { C_OXH = 0, C_OYH, C_OZH, C_OXL, C_OYL, C_OZL, C_TXL, C_TYL, C_TZL, C_S0H, C_S0L,
       C_LH, C_LL, C_AMP };

template <int NF>
struct FwdSmem {
    float4 A[kTS];            // tx, ty, tz, -o'.t
    float4 B[kTS];            // -2o'x, -2o'y, -2o'z, |o'|^2
    float2 Cw[kTS];           // s0 + margin, L + margin
    ColdSmem cold;
    float4 acc[NF][kR][kThreads];   // float-float accumulators per (f, receiver)
};

// Exact geometry of one (receiver, segment) pair in float-float; returns false
// when the pair falls outside the window.
template <int WINDOW>
__device__ __forceinline__ bool exact_geometry(float x, float y, float z, const ColdSmem &c,
                                               const float4 &A, int j, float &sh, float &sl,
                                               float &n2)
{
    const float oxh = c.f[C_OXH][j], oyh = c.f[C_OYH][j], ozh = c.f[C_OZH][j];
    const float thx = A.x, thy = A.y, thz = A.z;
    const float tlx = c.f[C_TXL][j], tly = c.f[C_TYL][j], tlz = c.f[C_TZL][j];
    // delta = x - o as (a + e)
    float ax, ex, ay, ey, az, ez;
    two_sum(x, -oxh, ax, ex);
    two_sum(y, -oyh, ay, ey);
    two_sum(z, -ozh, az, ez);
    ex -= c.f[C_OXL][j];
    ey -= c.f[C_OYL][j];
    ez -= c.f[C_OZL][j];
    // s_loc = delta . t
    float p0 = ax * thx, p1 = ay * thy, p2 = az * thz;
    float r0 = fmaf(ax, tlx, fmaf(ex, thx, fmaf(ax, thx, -p0)));
    float r1 = fmaf(ay, tly, fmaf(ey, thy, fmaf(ay, thy, -p1)));
    float r2 = fmaf(az, tlz, fmaf(ez, thz, fmaf(az, thz, -p2)));
    float S1, E1, S, E2;
    two_sum(p0, p1, S1, E1);
    two_sum(S1, p2, S, E2);
    const float lo = (E1 + E2) + (r0 + r1 + r2);
    if (WINDOW == GBT_WINDOW_SEGMENT) {
        if (!(S + lo >= 0.0f)) return false;
        if (!((S - c.f[C_LH][j]) + (lo - c.f[C_LL][j]) < 0.0f)) return false;
    }
    float e3;
    two_sum(c.f[C_S0H][j], S, sh, e3);
    sl = e3 + (lo + c.f[C_S0L][j]);
    if (WINDOW == GBT_WINDOW_LINE) {
        if (!(sh + sl >= 0.0f)) return false;
    }
    // n = delta x t, compensated
    float nx = dop(ay, thz, az, thy) + fmaf(ay, tlz, fmaf(-az, tly, fmaf(ey, thz, -ez * thy)));
    float ny = dop(az, thx, ax, thz) + fmaf(az, tlx, fmaf(-ax, tlz, fmaf(ez, thx, -ex * thz)));
    float nz = dop(ax, thy, ay, thx) + fmaf(ax, tly, fmaf(-ay, tlx, fmaf(ex, thy, -ey * thx)));
    n2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
    return true;
}

template <int NF, int WINDOW>
__device__ __forceinline__ void survivor(const FwdParams &p, float x, float y, float z,
                                         const ColdSmem &c, const float4 &A, int j,
                                         float2 (&tmp)[NF], uint32_t &kept)
{
    float sh, sl, n2;
    if (!exact_geometry<WINDOW>(x, y, z, c, A, j, sh, sl, n2)) return;
    const float amp = c.f[C_AMP][j];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (f >= p.nf) break;
        const FreqConst &q = p.fc[f];
        const float D = fmaf(sh, sh, q.b2);
        if (q.kb2 * n2 > p.cutoff * D) continue;          // Gaussian cutoff
        if (p.stats) {
            ++kept;
            continue;
        }
        const float invD = rcp_approx(D);
        const float n2invD = n2 * invD;
        const float ga = ex2_approx(-q.kb2l2e * n2invD);  // exp(-k b n^2 / (2 D))
        // phase in turns: frac(K s) in float-float, plus K n^2 s / (2 D)
        const float ph = q.K_hi * sh;
        const float pe = fmaf(q.K_hi, sh, -ph);
        const float corr = fmaf(q.K_hi, sl, fmaf(q.K_lo, sh, pe));
        float tau = (ph - rintf(ph)) + corr;
        tau = fmaf(q.halfK * n2invD, sh, tau);
        tau = tau - rintf(tau);
        float sn, cs;
        __sincosf(6.283185307179586f * tau, &sn, &cs);
        const float g = q.scale * amp * ga * invD;      // (s + i b) / D = 1 / E
        tmp[f].x = fmaf(g, fmaf(sh, cs, -q.b * sn), tmp[f].x);
        tmp[f].y = fmaf(g, fmaf(sh, sn, q.b * cs), tmp[f].y);
    }
}

template <int NF>
__device__ __forceinline__ void fold(float4 &acc, float2 &t)
{
    if (t.x != 0.0f || t.y != 0.0f) {
        float s, e;
        two_sum(acc.x, t.x, s, e);
        acc.x = s;
        acc.z += e;
        two_sum(acc.y, t.y, s, e);
        acc.y = s;
        acc.w += e;
        t = make_float2(0.0f, 0.0f);
    }
}

template <int NF, int WINDOW>
__global__ void __launch_bounds__(kThreads, 2) gbs_fwd_kernel(const FwdParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FwdSmem<NF> &sm = *reinterpret_cast<FwdSmem<NF> *>(smem_raw);
    __shared__ int s_item;

    const int tid = threadIdx.x;
    const int64_t n_seg = *p.n_seg_ptr;
    const int64_t n_seg_tiles = (n_seg + kTS - 1) / kTS;
    const float alpha = p.pre_alpha, beta = p.pre_beta;
    uint32_t n_pre = 0, n_kept = 0;

    // Persistent CTAs: each item is (receiver tile, split); split s covers the
    // segment tiles s, s + splits, s + 2 splits, ... so every item sees a mix of
    // ray directions and the work per item is even.
    for (;;) {
        if (tid == 0) s_item = atomicAdd(p.work_counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= p.n_items) break;
        const int64_t tile_base = (int64_t)(item / p.splits) * kTileRecv;
        const int split = item % p.splits;

        // tile centre: the tile's first receiver
        const int64_t c_idx = p.order ? p.order[tile_base] : tile_base;
        const float cx = p.recv[3 * c_idx], cy = p.recv[3 * c_idx + 1], cz = p.recv[3 * c_idx + 2];

        float xa[kR], ya[kR], za[kR], xp[kR], yp[kR], zp[kR], xx[kR];
        int64_t ridx[kR];
        uint32_t valid = 0;
#pragma unroll
        for (int k = 0; k < kR; ++k) {
            const int64_t r = tile_base + (int64_t)tid * kR + k;
            ridx[k] = -1;
            xa[k] = ya[k] = za[k] = xp[k] = yp[k] = zp[k] = xx[k] = 0.0f;
            if (r < p.n_recv) {
                const int64_t o = p.order ? p.order[r] : r;
                ridx[k] = o;
                xa[k] = p.recv[3 * o]; ya[k] = p.recv[3 * o + 1]; za[k] = p.recv[3 * o + 2];
                xp[k] = xa[k] - cx; yp[k] = ya[k] - cy; zp[k] = za[k] - cz;
                xx[k] = fmaf(xp[k], xp[k], fmaf(yp[k], yp[k], zp[k] * zp[k]));
                valid |= 1u << k;
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int k = 0; k < kR; ++k) sm.acc[f][k][tid] = make_float4(0.f, 0.f, 0.f, 0.f);

        float2 tmp[kR][NF];
#pragma unroll
        for (int k = 0; k < kR; ++k)
#pragma unroll
            for (int f = 0; f < NF; ++f) tmp[k][f] = make_float2(0.f, 0.f);

        for (int64_t stile = split; stile < n_seg_tiles; stile += p.splits) {
            const int64_t t0 = stile * kTS;
            const int64_t seg_end = min(n_seg, t0 + kTS);
            __syncthreads();
            if (tid < kTS) {
                const int64_t j = t0 + tid;
                if (j < seg_end) {
                    const float *R = p.rec;
                    const int64_t st = p.stride;
                    float oxh = R[F_OX * st + j], oyh = R[F_OY * st + j], ozh = R[F_OZ * st + j];
                    float oxl = R[F_OXL * st + j], oyl = R[F_OYL * st + j], ozl = R[F_OZL * st + j];
                    float tx = R[F_TX * st + j], ty = R[F_TY * st + j], tz = R[F_TZ * st + j];
                    float ox = (oxh - cx) + oxl, oy = (oyh - cy) + oyl, oz = (ozh - cz) + ozl;
                    float ot = fmaf(ox, tx, fmaf(oy, ty, oz * tz));
                    sm.A[tid] = make_float4(tx, ty, tz, -ot);
                    sm.B[tid] = make_float4(-2.f * ox, -2.f * oy, -2.f * oz,
                                            fmaf(ox, ox, fmaf(oy, oy, oz * oz)));
                    float s0h = R[F_S0 * st + j], Lh = R[F_L * st + j];
                    sm.Cw[tid] = make_float2(s0h + kWinMargin, Lh + kWinMargin);
                    sm.cold.f[C_OXH][tid] = oxh; sm.cold.f[C_OYH][tid] = oyh;
                    sm.cold.f[C_OZH][tid] = ozh;
                    sm.cold.f[C_OXL][tid] = oxl; sm.cold.f[C_OYL][tid] = oyl;
                    sm.cold.f[C_OZL][tid] = ozl;
                    sm.cold.f[C_TXL][tid] = R[F_TXL * st + j];
                    sm.cold.f[C_TYL][tid] = R[F_TYL * st + j];
                    sm.cold.f[C_TZL][tid] = R[F_TZL * st + j];
                    sm.cold.f[C_S0H][tid] = s0h;
                    sm.cold.f[C_S0L][tid] = R[F_S0L * st + j];
                    sm.cold.f[C_LH][tid] = Lh;
                    sm.cold.f[C_LL][tid] = R[F_LL * st + j];
                    sm.cold.f[C_AMP][tid] = R[F_AMP * st + j];
                } else {
                    // a record no receiver can keep: far behind its own start
                    sm.A[tid] = make_float4(0.f, 0.f, 0.f, -1e15f);
                    sm.B[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
                    sm.Cw[tid] = make_float2(0.f, 0.f);
                }
            }
            __syncthreads();
            const int nt = (int)(seg_end - t0);
            for (int b0 = 0; b0 < nt; b0 += 32) {
                uint32_t m[kR];
#pragma unroll
                for (int k = 0; k < kR; ++k) m[k] = 0u;
#pragma unroll 8
                for (int jj = 0; jj < 32; ++jj) {
                    const float4 A = sm.A[b0 + jj];
                    const float4 B = sm.B[b0 + jj];
                    const float2 Cw = sm.Cw[b0 + jj];
#pragma unroll
                    for (int k = 0; k < kR; ++k) {
                        const float sl = fmaf(xp[k], A.x, fmaf(yp[k], A.y, fmaf(zp[k], A.z, A.w)));
                        const float sm_ = sl + Cw.x;                       // s + margin
                        const float d2 = fmaf(xp[k], B.x, fmaf(yp[k], B.y, fmaf(zp[k], B.z, xx[k] + B.w)));
                        const float n2 = fmaf(-sl, sl, d2);
                        const float q = fmaf(sm_, sm_, beta);
                        const float e = fmaf(alpha, n2, -q);
                        uint32_t kb;
                        if (WINDOW == GBT_WINDOW_LINE) {
                            kb = __float_as_uint(e) & ~__float_as_uint(sm_);
                        } else {
                            const float a = sl + kWinMargin;
                            const float bb = sl - Cw.y;
                            kb = __float_as_uint(e) & ~__float_as_uint(a) & __float_as_uint(bb);
                        }
                        m[k] = __funnelshift_l(kb, m[k], 1);
                    }
                }
#pragma unroll
                for (int k = 0; k < kR; ++k) {
                    uint32_t mm = (valid >> k) & 1u ? m[k] : 0u;
                    if (p.stats) n_pre += __popc(mm);
                    while (mm) {
                        const int jj = __clz(mm);
                        mm ^= 0x80000000u >> jj;
                        const int j = b0 + jj;
                        if (j >= nt) break;           // bits past the tile's end
                        survivor<NF, WINDOW>(p, xa[k], ya[k], za[k], sm.cold, sm.A[j], j, tmp[k],
                                             n_kept);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kR; ++k)
#pragma unroll
                for (int f = 0; f < NF; ++f) fold<NF>(sm.acc[f][k][tid], tmp[k][f]);
        }
        if (!p.stats) {
#pragma unroll
            for (int k = 0; k < kR; ++k) {
                if (ridx[k] < 0) continue;
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    if (f >= p.nf) break;
                    p.partial[((int64_t)split * p.nf + f) * p.n_recv + ridx[k]] = sm.acc[f][k][tid];
                }
            }
        }
        __syncthreads();
    }
    if (p.stats) {
        atomicAdd(&p.stats[1], (unsigned long long)n_pre);
        atomicAdd(&p.stats[2], (unsigned long long)n_kept);
    }
}

// ------------------------------------------------------------- prepass --

struct PrepParams {
    const int32_t *n_seg_ptr;
    const double *o, *t, *L, *s0;
    const int32_t *ray, *depth, *bmat;
    const float *gamma;
    const float *weight;       // per global ray, or nullptr -> 4 pi / N
    double w_default;
    int n_materials;
    float *rec;
    int64_t stride;
    // F64 path records (nullptr when not needed)
    double *amp64;
    unsigned int *status;
};

__device__ __forceinline__ void split_ff(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
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
    const double w = p.weight ? (double)p.weight[p.ray[j]] : p.w_default;
    const double amp = w * g;
    float *R = p.rec;
    const int64_t st = p.stride;
    float h, l;
    split_ff(p.o[3 * j + 0], h, l); R[F_OX * st + j] = h; R[F_OXL * st + j] = l;
    split_ff(p.o[3 * j + 1], h, l); R[F_OY * st + j] = h; R[F_OYL * st + j] = l;
    split_ff(p.o[3 * j + 2], h, l); R[F_OZ * st + j] = h; R[F_OZL * st + j] = l;
    split_ff(p.t[3 * j + 0], h, l); R[F_TX * st + j] = h; R[F_TXL * st + j] = l;
    split_ff(p.t[3 * j + 1], h, l); R[F_TY * st + j] = h; R[F_TYL * st + j] = l;
    split_ff(p.t[3 * j + 2], h, l); R[F_TZ * st + j] = h; R[F_TZL * st + j] = l;
    split_ff(p.s0[j], h, l); R[F_S0 * st + j] = h; R[F_S0L * st + j] = l;
    split_ff(p.L[j], h, l); R[F_L * st + j] = h; R[F_LL * st + j] = l;
    R[F_AMP * st + j] = (float)amp;
    if (p.amp64) p.amp64[j] = amp;
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
};

template <int WINDOW>
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
    double sr[GBT_MAX_FREQ], cr[GBT_MAX_FREQ], si[GBT_MAX_FREQ], ci[GBT_MAX_FREQ];
    for (int f = 0; f < GBT_MAX_FREQ; ++f) sr[f] = cr[f] = si[f] = ci[f] = 0.0;
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
            for (int f = 0; f < p.nf; ++f) {
                const double k = p.k[f], b = p.b[f];
                const double D = s * s + b * b;
                if (k * n2 * b / (2.0 * D) > p.cutoff) continue;
                // c = amp * (k b / 8 pi^2) / E * exp(i k s + i k n^2 / (2E)), E = s - i b
                const double re_exp = -k * n2 * b / (2.0 * D);
                const double ph = k * s + k * n2 * s / (2.0 * D);
                const double a = sa[q] * (k * b / (8.0 * kPi * kPi)) * exp(re_exp) / D;
                double sn, cs;
                sincos(ph, &sn, &cs);
                const double vr = a * (s * cs - b * sn), vi = a * (s * sn + b * cs);
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
    for (int f = 0; f < p.nf; ++f)
        p.partial[((int64_t)split * p.nf + f) * p.n_recv + ri] =
            make_double2(sr[f] + cr[f], si[f] + ci[f]);
}

// ------------------------------------------------------------- reduce --

struct ReduceParams {
    int64_t n;                 // nf * n_recv
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
    double re = 0.0, im = 0.0;
    for (int s = 0; s < p.splits; ++s) {
        if (p.p32) {
            const float4 v = p.p32[(int64_t)s * p.n + i];
            re += (double)v.x + (double)v.z;
            im += (double)v.y + (double)v.w;
        } else {
            const double2 v = p.p64[(int64_t)s * p.n + i];
            re += v.x;
            im += v.y;
        }
    }
    if (p.accumulate) {
        const float2 o = p.out[i];
        re += (double)o.x;
        im += (double)o.y;
    }
    p.out[i] = make_float2((float)re, (float)im);
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

__global__ void extract_order(const unsigned long long *keys, int64_t n, int32_t *order)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) order[i] = (int32_t)(keys[i] & 0xffffffffull);
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <int NF, int WINDOW>
void launch_fwd(const FwdParams &p, cudaStream_t s)
{
    const size_t smem = sizeof(FwdSmem<NF>);
    GBT_CUDA(cudaFuncSetAttribute(gbs_fwd_kernel<NF, WINDOW>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GBT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gbs_fwd_kernel<NF, WINDOW>,
                                                           kThreads, smem));
    const int grid = std::max(1, std::min(p.n_items, std::max(per_sm, 1) * num_sms()));
    GBT_CUDA(cudaMemsetAsync(p.work_counter, 0, sizeof(int), s));
    if (!p.stats) timing_begin(s);
    gbs_fwd_kernel<NF, WINDOW><<<grid, kThreads, smem, s>>>(p);
    GBT_CUDA(cudaGetLastError());
    if (!p.stats) timing_end(s);
}

template <int WINDOW>
void launch_fwd_nf(const FwdParams &p, cudaStream_t s)
{
    if (p.nf <= 1) launch_fwd<1, WINDOW>(p, s);
    else if (p.nf <= 2) launch_fwd<2, WINDOW>(p, s);
    else if (p.nf <= 4) launch_fwd<4, WINDOW>(p, s);
    else launch_fwd<8, WINDOW>(p, s);
}

}  // namespace

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
    const int64_t tiles = (a.n_recv + kTileRecv - 1) / kTileRecv;
    const int64_t slots = 2 * (int64_t)num_sms();        // resident CTAs
    int64_t s = (8 * slots + tiles - 1) / (tiles > 0 ? tiles : 1);
    s = std::max<int64_t>(1, std::min<int64_t>(s, (nseg_est + kTS - 1) / kTS));
    // partial sums stay under ~1 GiB
    const int64_t per_split = (int64_t)a.n_freq * std::max<int64_t>(a.n_recv, 1) * 16;
    s = std::min<int64_t>(s, std::max<int64_t>(1, (1LL << 30) / per_split));
    return (int)std::min<int64_t>(s, 4096);
}

static size_t records_bytes(const TraceDev &td)
{
    return align_up((size_t)F_COUNT * align_up((size_t)td.capacity, 64) * sizeof(float), 256);
}

size_t sum_workspace_bytes(const TraceDev &td, const gbt_sum_args &a, int splits)
{
    size_t b = records_bytes(td);
    b += align_up((size_t)td.capacity * sizeof(double), 256);               // amp64
    b += 256;                                                               // work counter
    const size_t part = (size_t)splits * a.n_freq * (size_t)a.n_recv;
    b += align_up(part * (a.precision == GBT_PRECISION_F64 ? sizeof(double2) : sizeof(float4)),
                  256);
    return b;
}

void sum_launch(const TraceDev &td, const SceneDev &sd, const gbt_sum_args &a, int splits,
                void *work, cudaStream_t s, unsigned long long *stats)
{
    char *w = static_cast<char *>(work);
    float *rec = reinterpret_cast<float *>(w);
    const int64_t stride = (int64_t)align_up((size_t)td.capacity, 64);
    w += records_bytes(td);
    double *amp64 = reinterpret_cast<double *>(w);
    w += align_up((size_t)td.capacity * sizeof(double), 256);
    int *counter = reinterpret_cast<int *>(w);
    w += 256;
    void *partial = w;
    const int32_t *n_seg_ptr = td.ray_off + td.n_rays;

    if (td.capacity > 0) {
        PrepParams pp{};
        pp.n_seg_ptr = n_seg_ptr;
        pp.o = td.o; pp.t = td.t; pp.L = td.L; pp.s0 = td.s0;
        pp.ray = td.ray; pp.depth = td.depth; pp.bmat = td.bmat;
        pp.gamma = a.gamma;
        pp.weight = a.ray_weight;
        pp.w_default = 4.0 * kPi / (double)td.n_fan;
        pp.n_materials = sd.n_materials;
        pp.rec = rec;
        pp.stride = stride;
        pp.amp64 = amp64;
        pp.status = status_word();
        prepass_kernel<<<(unsigned)((td.capacity + 255) / 256), 256, 0, s>>>(pp);
        GBT_CUDA(cudaGetLastError());
    }

    const int64_t nout = (int64_t)a.n_freq * a.n_recv;
    if (a.n_recv > 0) {
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
            dim3 grid((unsigned)((a.n_recv + kThreads64 - 1) / kThreads64), (unsigned)splits);
            if (a.window == GBT_WINDOW_LINE)
                gbs_fwd_f64_kernel<GBT_WINDOW_LINE><<<grid, kThreads64, 0, s>>>(q);
            else
                gbs_fwd_f64_kernel<GBT_WINDOW_SEGMENT><<<grid, kThreads64, 0, s>>>(q);
            GBT_CUDA(cudaGetLastError());
        } else {
            FwdParams q{};
            q.recv = a.recv; q.order = a.recv_order; q.n_recv = a.n_recv;
            q.n_seg_ptr = n_seg_ptr;
            q.rec = rec;
            q.stride = stride;
            q.nf = a.n_freq;
            q.cutoff = (float)a.cutoff;
            double amin = 1e300, bmax = 0.0;
            for (int f = 0; f < a.n_freq; ++f) {
                const double K = a.freq_hz[f] / sd.c;       // turns per metre
                const double k = 2.0 * kPi * K;
                const double b = a.beam_b[f];
                FreqConst &c = q.fc[f];
                c.K_hi = (float)K;
                c.K_lo = (float)(K - (double)c.K_hi);
                c.halfK = (float)(0.5 * K);
                c.kb2 = (float)(0.5 * k * b);
                c.kb2l2e = (float)(0.5 * k * b * 1.4426950408889634);
                c.b = (float)b;
                c.b2 = (float)(b * b);
                c.scale = (float)(k * b / (8.0 * kPi * kPi));
                amin = std::min(amin, 0.5 * k * b);
                bmax = std::max(bmax, b * b);
            }
            q.pre_alpha = (float)(amin / (a.cutoff + 1.0));
            q.pre_beta = (float)bmax;
            q.splits = splits;
            q.partial = reinterpret_cast<float4 *>(partial);
            q.stats = stats;
            const int64_t tiles = (a.n_recv + kTileRecv - 1) / kTileRecv;
            q.n_items = (int)(tiles * splits);
            q.work_counter = counter;
            if (a.window == GBT_WINDOW_LINE) launch_fwd_nf<GBT_WINDOW_LINE>(q, s);
            else launch_fwd_nf<GBT_WINDOW_SEGMENT>(q, s);
            if (stats) return;
        }
        ReduceParams rp{};
        rp.n = nout;
        rp.splits = splits;
        rp.p32 = a.precision == GBT_PRECISION_F64 ? nullptr : reinterpret_cast<float4 *>(partial);
        rp.p64 = a.precision == GBT_PRECISION_F64 ? reinterpret_cast<double2 *>(partial) : nullptr;
        rp.out = reinterpret_cast<float2 *>(a.out);
        rp.accumulate = a.accumulate;
        reduce_kernel<<<(unsigned)((nout + 255) / 256), 256, 0, s>>>(rp);
        GBT_CUDA(cudaGetLastError());
    }
}

size_t recv_order_scratch_bytes(int64_t n)
{
    int64_t npad = 1;
    while (npad < n) npad <<= 1;
    return align_up((size_t)npad * sizeof(unsigned long long), 256) + 256;
}

void recv_order_launch(const float *recv, int64_t n, int32_t *order, void *scratch, cudaStream_t s)
{
    if (n <= 0) return;
    int64_t npad = 1;
    while (npad < n) npad <<= 1;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(scratch);
    unsigned int *bb = reinterpret_cast<unsigned int *>(
        static_cast<char *>(scratch) + align_up((size_t)npad * sizeof(unsigned long long), 256));
    GBT_CUDA(cudaMemsetAsync(bb, 0xff, 3 * sizeof(unsigned int), s));
    GBT_CUDA(cudaMemsetAsync(bb + 3, 0x00, 3 * sizeof(unsigned int), s));
    bbox_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(recv, n, bb);
    const unsigned g = (unsigned)((npad + 255) / 256);
    morton_kernel<<<g, 256, 0, s>>>(recv, n, npad, bb, keys);
    for (int64_t k = 2; k <= npad; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) bitonic_step<<<g, 256, 0, s>>>(keys, npad, j, k);
    extract_order<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, order);
    GBT_CUDA(cudaGetLastError());
}

}  // namespace gbt
