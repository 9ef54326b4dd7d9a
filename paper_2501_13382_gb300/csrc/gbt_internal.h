// gbt_internal.h -- private declarations shared by libgbt's translation units.
#pragma once

#include <cuda_runtime.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include <stdexcept>
#include <string>

#include "gbt.h"

namespace gbt {

// Error carried through the host code; converted to gbt_status at the ABI.
struct Error : public std::runtime_error {
    gbt_status code;
    Error(gbt_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};

void check_cuda(cudaError_t e, const char *what);
[[noreturn]] void fail(gbt_status code, const std::string &msg);
#define GBT_CUDA(call) ::gbt::check_cuda((call), #call)
#define GBT_REQUIRE(cond, msg) \
    do { if (!(cond)) ::gbt::fail(GBT_ERR_INVALID_ARG, (msg)); } while (0)

// Device memory through the installed allocator (default: stream-ordered pool).
void *dalloc(size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);

// Per-device status word (bit flags set by kernels, read by gbt_sync).
unsigned int *status_word();
enum : unsigned int { STATUS_BOUNDS = 1u, STATUS_TIMEOUT = 2u, STATUS_BAD_INPUT = 4u };

int num_sms();

// Upper bound on a tile-list workspace, in list entries (0: the default of an eighth of all
// (tile, segment) pairs, at least 16M); tiles whose lists do not fit stream every segment.
void set_list_capacity(int64_t entries);

// Per-device non-blocking stream of the library's own bookkeeping (small readbacks,
// frees of destroyed handles), so that none of them waits for unrelated streams.
cudaStream_t service_stream();
// Records `ev` (created on first use) on s: the latest launch that read a handle.
void mark_used(cudaEvent_t &ev, cudaStream_t s);
// Reads one int32 from device memory once `after` (if any) has completed.
int32_t read_device_i32(const int32_t *p, cudaEvent_t after);
// Stream on which a destroyed handle's memory may be freed: ordered after `used` (the
// host waits for it only when a caller-installed allocator frees immediately).
cudaStream_t after_last_use(cudaEvent_t used);

// Count of kernels the library has put on a stream (gbt_launches_read).
void note_launches(int64_t n);

// Optional CUDA-event timing of the main pair kernels (gbt_timing_*).
void timing_begin(cudaStream_t s);
void timing_end(cudaStream_t s);

// Growable device buffer owned by a handle.
struct DeviceBuffer {
    void *ptr = nullptr;
    size_t bytes = 0;
    void *ensure(size_t n, cudaStream_t s);
    void release(cudaStream_t s);
};

constexpr double kPi = 3.14159265358979323846;
constexpr double kTMin = 1e-9;   // smallest accepted hit distance, m

// BVH node: the padded FP32 boxes of its two children (lo xyz, hi xyz each) and their
// references: >= 0 an inner node, kBvhNone no child, otherwise a leaf of 1..8
// consecutive entries of the triangle permutation, encoded -(first * 8 + count - 1) - 1.
struct alignas(16) BvhNode {
    float box[2][6];
    int32_t ref[2];
    int32_t pad[2];
};
static_assert(sizeof(BvhNode) == 64, "BVH node is four 16-byte words");
constexpr int32_t kBvhNone = INT32_MIN;
constexpr int kBvhLeaf = 4;          // most triangles per leaf
constexpr int kBvhStack = 64;        // traversal stack entries (build depth is at most 58)

// Scene on the device.  Per triangle 12 doubles: v0, e1 = v1 - v0, e2 = v2 - v0,
// unit normal (e1 x e2 normalised).
struct SceneDev {
    double c = 0;
    int ground = 0;
    int ground_material = 0;
    double ground_z = 0;
    int64_t n_tri = 0;
    int n_materials = 0;
    double *tri = nullptr;       // n_tri * 12
    float *trif = nullptr;       // n_tri * 9: v0, e1, e2 rounded to FP32 (BVH screen)
    int32_t *face = nullptr;     // n_tri
    int32_t *mat = nullptr;      // n_tri
    // bounding boxes of consecutive triangle clusters (kTriCluster each), in FP32,
    // expanded far beyond FP32 rounding so a box test never rejects a hit:
    // per cluster xmin, ymin, zmin, xmax, ymax, zmax
    float *cbox = nullptr;         // padded FP32 box per cluster of kTriCluster triangles
    float *tbox = nullptr;         // padded FP32 box per triangle
    int64_t n_clusters = 0;
    int accel = GBT_ACCEL_AUTO;
    BvhNode *bvh = nullptr;        // nodes (root 0), or nullptr when not built
    int32_t *bvh_perm = nullptr;   // triangle index of each leaf entry
    int64_t n_bvh_nodes = 0;
    int bvh_depth = 0;
    mutable cudaEvent_t used = nullptr;   // after the latest launch that read the scene
};
constexpr int kTriCluster = 8;

// Segment kernel record: the FP64 canonical segment split into float-float
// (hi, lo) pairs, 20 floats (80 bytes, 16-byte aligned) per segment, array of
// structures so one warp stages 32 consecutive records with 16-byte copies.
enum RecField {
    R_OXH = 0, R_OYH, R_OZH, R_S0H,      // origin hi, start arclength hi
    R_TXH, R_TYH, R_TZH, R_LH,           // unit direction hi, length hi
    R_OXL, R_OYL, R_OZL, R_S0L,          // lo parts
    R_TXL, R_TYL, R_TZL, R_LL,
    R_AMP,                               // W_ray * Gamma_path
    kRecFloats = 20
};

// Fan of take-off directions of a trace (angles in radians).
struct FanDev {
    int kind = GBT_FAN_FIBONACCI;
    int64_t n_phi = 0;                   // GBT_FAN_LATLONG: rays per polar row
    double th0 = 0, dth = 0, ph0 = 0, dph = 0;
};

// Default weight of global ray g of a fan of n_fan rays: 4 pi / N, or for the
// lat-long grid its cell's solid angle dphi (cos th_lo - cos th_hi), written
// 2 dphi sin(th_mid) sin(dth / 2).
__host__ __device__ inline double fan_weight(const FanDev &f, int64_t n_fan, int64_t g)
{
    if (f.kind != GBT_FAN_LATLONG) return 4.0 * 3.14159265358979323846 / (double)n_fan;
    const int64_t it = g / f.n_phi;
    const double th = f.th0 + ((double)it + 0.5) * f.dth;
    return 2.0 * f.dph * sin(th) * sin(0.5 * f.dth);
}

struct TraceDev {
    const gbt_scene_t *scene = nullptr;
    int64_t n_fan = 0, ray_begin = 0, n_rays = 0, capacity = 0;
    FanDev fan;
    int max_refl = 0;
    double max_path = 0;
    int32_t *ray_off = nullptr;  // n_rays + 1 (device); ray_off[n_rays] = segment count
    double *o = nullptr, *t = nullptr, *L = nullptr, *s0 = nullptr;
    int32_t *ray = nullptr, *depth = nullptr, *bmat = nullptr, *hit = nullptr;
    void *block = nullptr;       // single allocation holding everything above
    DeviceBuffer work;           // scratch for sums (records, partials)
    int64_t n_seg_host = -1;     // cached once read back
    cudaEvent_t used = nullptr;  // after the latest launch that read or wrote the trace
};

// ---- kernels' host-side launchers (trace.cu) ----
void scene_prepare(SceneDev &sd, const double *tri_raw_dev, cudaStream_t s);
void trace_launch(const SceneDev &sd, TraceDev &td, const gbt_source_desc &src,
                  void *scratch, size_t scratch_bytes, cudaStream_t s);
size_t trace_scratch_bytes(int64_t n_rays, int max_refl);
// Fills each segment's ray index and depth from the trace's offsets (imported traces).
void csr_ray_depth_launch(TraceDev &td, cudaStream_t s);

// ---- GBS launchers (gbs.cu) ----
// Whether a sum carries propagation losses (air absorption or porous surfaces).
bool has_losses(const gbt_sum_args &a);
size_t sum_workspace_bytes(const TraceDev &td, const gbt_sum_args &a, int splits);
int choose_splits(const TraceDev &td, const gbt_sum_args &a);
void sum_launch(const TraceDev &td, const SceneDev &sd, const gbt_sum_args &a, int splits,
                void *work, cudaStream_t s, unsigned long long *stats = nullptr);
void recv_order_launch(const float *recv, int64_t n, int32_t *order, void *scratch,
                       cudaStream_t s);
size_t recv_order_scratch_bytes(int64_t n);
void selftest_timeout_launch(long long spins, cudaStream_t s);
void recv_order_noalloc_launch(const float *recv, int64_t n, int32_t *order, cudaStream_t s);

// ---- batched persistent launch (gbs.cu) ----
struct BatchImpl;
BatchImpl *batch_create(const gbt_batch_desc &d, cudaStream_t s);
// Records the trace's and its scene's last use on s (after a launch that reads them).
void mark_trace_used(const gbt_trace_t *tr, cudaStream_t s);
void batch_submit(BatchImpl *b, cudaStream_t s);
void batch_destroy(BatchImpl *b);

// ---- time synthesis (gbs.cu): phasors A_f exp(-i 2 pi f t_n) formed on the device ----
void synth_launch(const float *p, int nf, int64_t n_recv, const double *freq_hz,
                  const double *amp, double t0, double dt, int64_t n_t, float *out,
                  int accumulate, cudaStream_t s);

// ---- backward (gbs.cu) ----
size_t bwd_workspace_bytes(const TraceDev &td, const gbt_sum_args &a);
void bwd_launch(const TraceDev &td, const SceneDev &sd, const gbt_sum_args &a,
                const float *grad_out, float *grad_gamma, float *grad_w, double *grad_b,
                void *work, cudaStream_t s);

}  // namespace gbt

struct gbt_scene_s {
    gbt::SceneDev d;
};

struct gbt_trace_s {
    gbt::TraceDev d;
};

struct gbt_batch_s {
    gbt::BatchImpl *impl;
};
