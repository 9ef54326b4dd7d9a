// api.cu -- host implementation of the libgbt C ABI (include/gbt.h).
// Argument validation, handle ownership, device memory, error reporting.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bvh_build.h"
#include "gbt_internal.h"

namespace gbt {

namespace {
thread_local std::string t_last_error;
std::mutex g_mu;
gbt_allocator g_alloc{};
bool g_has_alloc = false;
unsigned int *g_status[64] = {};
int g_sms[64] = {};

int current_device()
{
    int d = 0;
    GBT_CUDA(cudaGetDevice(&d));
    if (d < 0 || d >= 64) fail(GBT_ERR_UNSUPPORTED, "device index >= 64");
    return d;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <class F>
gbt_status guarded(F &&f)
{
    try {
        f();
        t_last_error.clear();
        return GBT_OK;
    } catch (const Error &e) {
        t_last_error = e.what();
        return e.code;
    } catch (const std::bad_alloc &) {
        t_last_error = "host allocation failed";
        return GBT_ERR_OOM;
    } catch (const std::exception &e) {
        t_last_error = e.what();
        return GBT_ERR_CUDA;
    } catch (...) {
        t_last_error = "unknown error";
        return GBT_ERR_CUDA;
    }
}
}  // namespace

[[noreturn]] void fail(gbt_status code, const std::string &msg) { throw Error(code, msg); }

void check_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return;
    const gbt_status code = (e == cudaErrorMemoryAllocation) ? GBT_ERR_OOM : GBT_ERR_CUDA;
    cudaGetLastError();   // clear a non-sticky error
    throw Error(code, std::string(what) + ": " + cudaGetErrorString(e));
}

void *dalloc(size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 256;
    gbt_allocator a;
    bool has;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        a = g_alloc;
        has = g_has_alloc;
    }
    void *p = nullptr;
    if (has) {
        p = a.alloc(bytes, s, a.ctx);
        if (!p) fail(GBT_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
    } else {
        static bool pool_set[64] = {};
        const int dev = current_device();
        if (!pool_set[dev]) {
            // keep freed blocks in the stream-ordered pool instead of returning them to
            // the driver at every synchronisation (process-local setting)
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t thr = ~0ull;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
            }
            cudaGetLastError();
            pool_set[dev] = true;
        }
        cudaError_t e = cudaMallocAsync(&p, bytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(GBT_ERR_OOM, "cudaMallocAsync(" + std::to_string(bytes) + "): " +
                                  cudaGetErrorString(e));
        }
    }
    return p;
}

void dfree(void *p, cudaStream_t s)
{
    if (!p) return;
    gbt_allocator a;
    bool has;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        a = g_alloc;
        has = g_has_alloc;
    }
    if (has) a.free(p, s, a.ctx);
    else cudaFreeAsync(p, s);
}

cudaStream_t service_stream()
{
    static cudaStream_t streams[64] = {};
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!streams[d]) GBT_CUDA(cudaStreamCreateWithFlags(&streams[d], cudaStreamNonBlocking));
    return streams[d];
}

void mark_used(cudaEvent_t &ev, cudaStream_t s)
{
    if (!ev) GBT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    GBT_CUDA(cudaEventRecord(ev, s));
}

void mark_trace_used(const gbt_trace_t *tr, cudaStream_t s)
{
    gbt_trace_t *t = const_cast<gbt_trace_t *>(tr);
    mark_used(t->d.used, s);
    if (t->d.scene) mark_used(t->d.scene->d.used, s);
}

int32_t read_device_i32(const int32_t *p, cudaEvent_t after)
{
    cudaStream_t q = service_stream();
    if (after) GBT_CUDA(cudaStreamWaitEvent(q, after, 0));
    int32_t v = 0;
    GBT_CUDA(cudaMemcpyAsync(&v, p, sizeof(v), cudaMemcpyDeviceToHost, q));
    GBT_CUDA(cudaStreamSynchronize(q));
    return v;
}

// Stream on which a destroyed handle's memory is freed once its last recorded use
// (`used`) has finished.  With the library's stream-ordered pool the frees are queued
// behind that use and the host does not wait; an installed allocator frees at once,
// so the host first waits for the use to end.  Neither waits for unrelated streams.
cudaStream_t after_last_use(cudaEvent_t used)
{
    cudaStream_t q = service_stream();
    if (!used) return q;
    bool custom;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        custom = g_has_alloc;
    }
    if (custom) GBT_CUDA(cudaEventSynchronize(used));
    else GBT_CUDA(cudaStreamWaitEvent(q, used, 0));
    return q;
}

unsigned int *status_word()
{
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status[d]) {
        void *p = nullptr;
        GBT_CUDA(cudaMalloc(&p, 256));
        GBT_CUDA(cudaMemset(p, 0, 256));
        g_status[d] = static_cast<unsigned int *>(p);
    }
    return g_status[d];
}

namespace {
struct TimingState {
    bool enabled = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    std::vector<cudaEvent_t> pool;
};
TimingState g_timing;
std::mutex g_timing_mu;

cudaEvent_t timing_event()
{
    if (!g_timing.pool.empty()) {
        cudaEvent_t e = g_timing.pool.back();
        g_timing.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    GBT_CUDA(cudaEventCreate(&e));
    return e;
}
}  // namespace

namespace {
std::atomic<int64_t> g_launches{0};
}

void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void timing_begin(cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_timing_mu);
    if (!g_timing.enabled) return;
    cudaEvent_t a = timing_event(), b = timing_event();
    GBT_CUDA(cudaEventRecord(a, s));
    g_timing.events.emplace_back(a, b);
}

void timing_end(cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_timing_mu);
    if (!g_timing.enabled || g_timing.events.empty()) return;
    GBT_CUDA(cudaEventRecord(g_timing.events.back().second, s));
}

int num_sms()
{
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_sms[d]) GBT_CUDA(cudaDeviceGetAttribute(&g_sms[d], cudaDevAttrMultiProcessorCount, d));
    return g_sms[d];
}

void *DeviceBuffer::ensure(size_t n, cudaStream_t s)
{
    if (n <= bytes && ptr) return ptr;
    release(s);
    ptr = dalloc(n, s);
    bytes = n;
    return ptr;
}

void DeviceBuffer::release(cudaStream_t s)
{
    if (ptr) dfree(ptr, s);
    ptr = nullptr;
    bytes = 0;
}

// ------------------------------------------------------------------ trace --

static void validate_source(const gbt_source_desc &src)
{
    GBT_REQUIRE(src.n_rays >= 1, "n_rays must be >= 1");
    GBT_REQUIRE(src.ray_begin >= 0 && src.ray_begin < src.n_rays, "ray_begin out of range");
    const int64_t cnt = src.ray_count == 0 ? src.n_rays - src.ray_begin : src.ray_count;
    GBT_REQUIRE(cnt >= 1 && src.ray_begin + cnt <= src.n_rays, "ray_count out of range");
    GBT_REQUIRE(src.max_reflections >= 0 && src.max_reflections <= 64,
                "max_reflections must be in [0, 64]");
    GBT_REQUIRE(src.max_path > 0 && isfinite(src.max_path), "max_path must be finite and > 0");
    GBT_REQUIRE(isfinite(src.pos[0]) && isfinite(src.pos[1]) && isfinite(src.pos[2]),
                "source position must be finite");
    GBT_REQUIRE(src.fan == GBT_FAN_FIBONACCI || src.fan == GBT_FAN_EXPLICIT ||
                    src.fan == GBT_FAN_LATLONG, "unknown fan");
    GBT_REQUIRE(src.fan != GBT_FAN_EXPLICIT || src.dirs, "explicit fan needs dirs");
    if (src.fan == GBT_FAN_LATLONG) {
        GBT_REQUIRE(src.n_theta >= 1 && src.n_rays % src.n_theta == 0,
                    "lat-long fan: n_theta must be >= 1 and divide n_rays");
        const double *th = src.theta_deg, *ph = src.phi_deg;
        GBT_REQUIRE(isfinite(th[0]) && isfinite(th[1]) && th[0] >= 0.0 && th[0] < th[1] &&
                        th[1] <= 180.0, "lat-long fan: need 0 <= theta_deg[0] < theta_deg[1] <= 180");
        GBT_REQUIRE(isfinite(ph[0]) && isfinite(ph[1]) && ph[0] < ph[1] && ph[1] - ph[0] <= 360.0,
                    "lat-long fan: need phi_deg[0] < phi_deg[1] <= phi_deg[0] + 360");
    }
    GBT_REQUIRE((double)cnt * (src.max_reflections + 1) < 2147483647.0,
                "segment capacity exceeds 2^31 - 1: trace fewer rays at a time");
}

// Device buffers of a trace of up to cnt rays (one allocation); td's ray range is set
// by the caller before each trace_launch into it.
static void alloc_trace_block(TraceDev &td, const gbt_scene_t *scene, const gbt_source_desc &src,
                              int64_t cnt, cudaStream_t s)
{
    td.scene = scene;
    td.n_fan = src.n_rays;
    td.fan = FanDev{};
    td.fan.kind = src.fan;
    if (src.fan == GBT_FAN_LATLONG) {
        const double deg = kPi / 180.0;
        td.fan.n_phi = src.n_rays / src.n_theta;
        td.fan.th0 = src.theta_deg[0] * deg;
        td.fan.dth = (src.theta_deg[1] - src.theta_deg[0]) * deg / (double)src.n_theta;
        td.fan.ph0 = src.phi_deg[0] * deg;
        td.fan.dph = (src.phi_deg[1] - src.phi_deg[0]) * deg / (double)td.fan.n_phi;
    }
    td.max_refl = src.max_reflections;
    td.max_path = src.max_path;
    td.capacity = cnt * (int64_t)(src.max_reflections + 1);
    const size_t cap = (size_t)td.capacity;
    size_t bytes = align_up((size_t)(cnt + 1) * 4, 256) + 2 * align_up(cap * 24, 256) +
                   2 * align_up(cap * 8, 256) + 4 * align_up(cap * 4, 256);
    td.block = dalloc(bytes, s);
    char *w = static_cast<char *>(td.block);
    auto take = [&](size_t b) { char *p = w; w += align_up(b, 256); return p; };
    td.ray_off = reinterpret_cast<int32_t *>(take((size_t)(cnt + 1) * 4));
    td.o = reinterpret_cast<double *>(take(cap * 24));
    td.t = reinterpret_cast<double *>(take(cap * 24));
    td.L = reinterpret_cast<double *>(take(cap * 8));
    td.s0 = reinterpret_cast<double *>(take(cap * 8));
    td.ray = reinterpret_cast<int32_t *>(take(cap * 4));
    td.depth = reinterpret_cast<int32_t *>(take(cap * 4));
    td.bmat = reinterpret_cast<int32_t *>(take(cap * 4));
    td.hit = reinterpret_cast<int32_t *>(take(cap * 4));
}

static gbt_trace_t *make_trace(const gbt_scene_t *scene, const gbt_source_desc &src, cudaStream_t s)
{
    validate_source(src);
    const int64_t cnt = src.ray_count == 0 ? src.n_rays - src.ray_begin : src.ray_count;
    gbt_trace_t *tr = new gbt_trace_s();
    TraceDev &td = tr->d;
    void *scratch = nullptr;
    try {
        alloc_trace_block(td, scene, src, cnt, s);
        td.ray_begin = src.ray_begin;
        td.n_rays = cnt;
        const size_t sb = trace_scratch_bytes(cnt, src.max_reflections);
        scratch = dalloc(sb, s);
        trace_launch(scene->d, td, src, scratch, sb, s);
        dfree(scratch, s);
        mark_trace_used(tr, s);
    } catch (...) {
        if (scratch) dfree(scratch, s);
        if (td.block) dfree(td.block, s);
        if (td.used) cudaEventDestroy(td.used);
        delete tr;
        throw;
    }
    return tr;
}

static void validate_sum(const gbt_trace_t *trace, const gbt_sum_args *a, bool need_out = true)
{
    GBT_REQUIRE(trace, "trace is NULL");
    GBT_REQUIRE(a, "args is NULL");
    GBT_REQUIRE(a->n_recv >= 0, "n_recv must be >= 0");
    GBT_REQUIRE(a->n_freq >= 1 && a->n_freq <= GBT_MAX_FREQ, "n_freq must be in [1, 16]");
    GBT_REQUIRE(a->window == GBT_WINDOW_SEGMENT || a->window == GBT_WINDOW_LINE, "unknown window");
    GBT_REQUIRE(a->precision == GBT_PRECISION_F32 || a->precision == GBT_PRECISION_F64,
                "unknown precision");
    GBT_REQUIRE(a->cutoff > 0 && isfinite(a->cutoff), "cutoff must be finite and > 0");
    GBT_REQUIRE(a->seg_split >= 0 && a->seg_split <= 4096, "seg_split must be in [0, 4096]");
    for (int f = 0; f < a->n_freq; ++f) {
        GBT_REQUIRE(a->freq_hz[f] > 0 && isfinite(a->freq_hz[f]), "frequencies must be > 0");
        GBT_REQUIRE(a->beam_b[f] > 0 && isfinite(a->beam_b[f]), "beam_b must be > 0");
        GBT_REQUIRE(a->absorption[f] >= 0 && isfinite(a->absorption[f]),
                    "absorption must be finite and >= 0 (Np/m)");
    }
    GBT_REQUIRE(a->gamma, "gamma is NULL");
    if (a->n_recv > 0) {
        GBT_REQUIRE(a->recv, "recv must be non-NULL");
        if (need_out) {
            GBT_REQUIRE(a->out, "out must be non-NULL");
            GBT_REQUIRE(((uintptr_t)a->out & 7u) == 0, "out must be 8-byte aligned");
        }
        GBT_REQUIRE(a->n_recv < 2147483647LL, "n_recv must be < 2^31");
    }
}

}  // namespace gbt

using namespace gbt;

// Named NVTX range around each public entry point (trace, sum, adjoint, solve, batch,
// receiver order), so profilers can attribute device work to the call that launched it;
// free when no profiling tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

extern "C" {

int32_t gbt_version(void) { return GBT_VERSION; }

const char *gbt_last_error(void) { return t_last_error.c_str(); }

gbt_status gbt_set_allocator(const gbt_allocator *allocator)
{
    return guarded([&] {
        if (allocator) GBT_REQUIRE(allocator->alloc && allocator->free, "allocator needs alloc and free");
        std::lock_guard<std::mutex> lk(g_mu);
        if (allocator) {
            g_alloc = *allocator;
            g_has_alloc = true;
        } else {
            g_alloc = gbt_allocator{};
            g_has_alloc = false;
        }
    });
}

// ------------------------------------------------------------------- BVH --
// BvhBuilder (bvh_build.h) builds the tracer's hierarchy when a scene is created.


gbt_status gbt_scene_create(const gbt_scene_desc *desc, void *stream, gbt_scene_t **out)
{
    return guarded([&] {
        GBT_REQUIRE(desc && out, "desc and out must be non-NULL");
        *out = nullptr;
        const gbt_scene_desc &d = *desc;
        GBT_REQUIRE(d.c > 0 && isfinite(d.c), "speed of sound must be > 0");
        GBT_REQUIRE(d.n_tri >= 0 && d.n_tri < (1LL << 26), "n_tri out of range");
        GBT_REQUIRE(d.n_materials >= 1, "n_materials must be >= 1");
        GBT_REQUIRE(!d.ground_enabled || (d.ground_material >= 0 && d.ground_material < d.n_materials),
                    "ground_material out of range");
        GBT_REQUIRE(isfinite(d.ground_z), "ground_z must be finite");
        GBT_REQUIRE(d.accel == GBT_ACCEL_AUTO || d.accel == GBT_ACCEL_BVH || d.accel == GBT_ACCEL_LINEAR,
                    "accel must be GBT_ACCEL_AUTO, GBT_ACCEL_BVH or GBT_ACCEL_LINEAR");
        if (d.n_tri > 0) {
            GBT_REQUIRE(d.tri_xyz && d.tri_material, "triangles need tri_xyz and tri_material");
            for (int64_t k = 0; k < d.n_tri; ++k) {
                GBT_REQUIRE(d.tri_material[k] >= 0 && d.tri_material[k] < d.n_materials,
                            "tri_material out of range");
                if (d.tri_face) GBT_REQUIRE(d.tri_face[k] >= 0, "tri_face must be >= 0");
                for (int q = 0; q < 9; ++q)
                    GBT_REQUIRE(isfinite(d.tri_xyz[9 * k + q]), "triangle vertices must be finite");
            }
        }
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        gbt_scene_t *sc = new gbt_scene_s();
        SceneDev &sd = sc->d;
        sd.c = d.c;
        sd.ground = d.ground_enabled ? 1 : 0;
        sd.ground_material = d.ground_material;
        sd.ground_z = d.ground_z;
        sd.n_tri = d.n_tri;
        sd.n_materials = d.n_materials;
        sd.accel = d.accel;
        void *raw = nullptr;
        try {
            const size_t nt = (size_t)std::max<int64_t>(d.n_tri, 1);
            sd.tri = static_cast<double *>(dalloc(nt * 12 * sizeof(double), s));
            sd.trif = static_cast<float *>(dalloc(nt * 9 * sizeof(float), s));
            sd.face = static_cast<int32_t *>(dalloc(nt * sizeof(int32_t), s));
            sd.mat = static_cast<int32_t *>(dalloc(nt * sizeof(int32_t), s));
            sd.n_clusters = (d.n_tri + kTriCluster - 1) / kTriCluster;
            sd.cbox = static_cast<float *>(
                dalloc((size_t)std::max<int64_t>(sd.n_clusters, 1) * 6 * sizeof(float), s));
            sd.tbox = static_cast<float *>(dalloc(nt * 6 * sizeof(float), s));
            if (d.n_tri > 0) {
                std::vector<int32_t> face(d.n_tri);
                for (int64_t k = 0; k < d.n_tri; ++k) face[k] = d.tri_face ? d.tri_face[k] : (int32_t)k;
                raw = dalloc((size_t)d.n_tri * 9 * sizeof(double), s);
                GBT_CUDA(cudaMemcpyAsync(raw, d.tri_xyz, (size_t)d.n_tri * 9 * sizeof(double),
                                         cudaMemcpyHostToDevice, s));
                GBT_CUDA(cudaMemcpyAsync(sd.face, face.data(), (size_t)d.n_tri * 4,
                                         cudaMemcpyHostToDevice, s));
                GBT_CUDA(cudaMemcpyAsync(sd.mat, d.tri_material, (size_t)d.n_tri * 4,
                                         cudaMemcpyHostToDevice, s));
                // FP32 boxes of each cluster of kTriCluster triangles and of each triangle,
                // on the host: exact min/max, then an expansion (1 mm plus 2e-6 relative)
                // far above the rounding of the FP32 slab test, rounded outward
                auto padded_box = [&](int64_t k0, int64_t k1, float *box) {
                    double lo[3] = {INFINITY, INFINITY, INFINITY};
                    double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
                    for (int64_t k = k0; k < k1; ++k)
                        for (int v = 0; v < 3; ++v)
                            for (int a = 0; a < 3; ++a) {
                                const double x = d.tri_xyz[9 * k + 3 * v + a];
                                lo[a] = std::min(lo[a], x);
                                hi[a] = std::max(hi[a], x);
                            }
                    for (int a = 0; a < 3; ++a) {
                        const double pad = 1e-3 + 2e-6 * std::max(fabs(lo[a]), fabs(hi[a]));
                        box[a] = nextafterf((float)(lo[a] - pad), -INFINITY);
                        box[3 + a] = nextafterf((float)(hi[a] + pad), INFINITY);
                    }
                };
                std::vector<float> box((size_t)sd.n_clusters * 6), tbox((size_t)d.n_tri * 6);
                for (int64_t c = 0; c < sd.n_clusters; ++c)
                    padded_box(c * kTriCluster, std::min<int64_t>(d.n_tri, (c + 1) * kTriCluster),
                               &box[6 * c]);
                for (int64_t k = 0; k < d.n_tri; ++k) padded_box(k, k + 1, &tbox[6 * k]);
                GBT_CUDA(cudaMemcpyAsync(sd.cbox, box.data(), box.size() * sizeof(float),
                                         cudaMemcpyHostToDevice, s));
                GBT_CUDA(cudaMemcpyAsync(sd.tbox, tbox.data(), tbox.size() * sizeof(float),
                                         cudaMemcpyHostToDevice, s));
                if (d.accel != GBT_ACCEL_LINEAR) {
                    BvhBuilder bb(d.tri_xyz, tbox, d.n_tri);
                    bb.run();
                    sd.n_bvh_nodes = (int64_t)bb.nodes.size();
                    sd.bvh_depth = bb.depth_max;
                    GBT_REQUIRE(sd.bvh_depth + 2 <= kBvhStack, "BVH deeper than the traversal stack");
                    sd.bvh = static_cast<BvhNode *>(dalloc(bb.nodes.size() * sizeof(BvhNode), s));
                    sd.bvh_perm = static_cast<int32_t *>(dalloc(bb.perm.size() * sizeof(int32_t), s));
                    GBT_CUDA(cudaMemcpyAsync(sd.bvh, bb.nodes.data(), bb.nodes.size() * sizeof(BvhNode),
                                             cudaMemcpyHostToDevice, s));
                    GBT_CUDA(cudaMemcpyAsync(sd.bvh_perm, bb.perm.data(), bb.perm.size() * sizeof(int32_t),
                                             cudaMemcpyHostToDevice, s));
                }
                scene_prepare(sd, static_cast<const double *>(raw), s);
                dfree(raw, s);
                raw = nullptr;
                GBT_CUDA(cudaStreamSynchronize(s));
            }
        } catch (...) {
            if (raw) dfree(raw, s);
            dfree(sd.tri, s); dfree(sd.trif, s); dfree(sd.face, s); dfree(sd.mat, s); dfree(sd.cbox, s);
            dfree(sd.tbox, s);
            if (sd.bvh) dfree(sd.bvh, s);
            if (sd.bvh_perm) dfree(sd.bvh_perm, s);
            delete sc;
            throw;
        }
        *out = sc;
    });
}

gbt_status gbt_scene_destroy(gbt_scene_t *scene)
{
    return guarded([&] {
        if (!scene) return;
        cudaStream_t q = after_last_use(scene->d.used);
        dfree(scene->d.tri, q);
        dfree(scene->d.trif, q);
        dfree(scene->d.face, q);
        dfree(scene->d.mat, q);
        dfree(scene->d.cbox, q);
        dfree(scene->d.tbox, q);
        if (scene->d.bvh) dfree(scene->d.bvh, q);
        if (scene->d.bvh_perm) dfree(scene->d.bvh_perm, q);
        if (scene->d.used) cudaEventDestroy(scene->d.used);
        delete scene;
    });
}

gbt_status gbt_trace(const gbt_scene_t *scene, const gbt_source_desc *src, void *stream,
                     gbt_trace_t **out)
{
    NvtxRange nvtx_range("gbt_trace");
    return guarded([&] {
        GBT_REQUIRE(scene && src && out, "scene, src and out must be non-NULL");
        *out = nullptr;
        *out = make_trace(scene, *src, static_cast<cudaStream_t>(stream));
    });
}

gbt_status gbt_trace_import(const gbt_scene_t *scene, const gbt_source_desc *src,
                            const gbt_segments *segs, void *stream, gbt_trace_t **out)
{
    NvtxRange nvtx_range("gbt_trace_import");
    return guarded([&] {
        GBT_REQUIRE(scene && src && segs && out, "scene, src, segs and out must be non-NULL");
        *out = nullptr;
        validate_source(*src);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int64_t cnt = src->ray_count == 0 ? src->n_rays - src->ray_begin : src->ray_count;
        const int64_t per_ray = (int64_t)src->max_reflections + 1;
        const int64_t n = segs->n_segments;
        GBT_REQUIRE(n >= 0 && n <= cnt * per_ray, "n_segments out of range for the ray range");
        GBT_REQUIRE(segs->ray_off, "ray_off must be non-NULL");
        GBT_REQUIRE(n == 0 || (segs->seg_o && segs->seg_t && segs->seg_L && segs->seg_s0 &&
                               segs->seg_bmat),
                    "segment arrays must be non-NULL");
        std::vector<int32_t> off((size_t)cnt + 1);
        GBT_CUDA(cudaMemcpyAsync(off.data(), segs->ray_off, off.size() * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
        GBT_CUDA(cudaStreamSynchronize(s));
        GBT_REQUIRE(off[0] == 0 && off[(size_t)cnt] == n, "ray_off must run from 0 to n_segments");
        for (int64_t i = 0; i < cnt; ++i) {
            const int64_t c = (int64_t)off[i + 1] - off[i];
            GBT_REQUIRE(c >= 0 && c <= per_ray,
                        "ray_off: each ray needs 0 .. max_reflections + 1 segments");
        }
        gbt_trace_t *tr = new gbt_trace_s();
        TraceDev &td = tr->d;
        try {
            alloc_trace_block(td, scene, *src, cnt, s);
            td.ray_begin = src->ray_begin;
            td.n_rays = cnt;
            auto copy = [&](void *dst, const void *from, size_t bytes) {
                if (bytes) GBT_CUDA(cudaMemcpyAsync(dst, from, bytes, cudaMemcpyDeviceToDevice, s));
            };
            copy(td.ray_off, segs->ray_off, ((size_t)cnt + 1) * sizeof(int32_t));
            copy(td.o, segs->seg_o, (size_t)n * 3 * sizeof(double));
            copy(td.t, segs->seg_t, (size_t)n * 3 * sizeof(double));
            copy(td.L, segs->seg_L, (size_t)n * sizeof(double));
            copy(td.s0, segs->seg_s0, (size_t)n * sizeof(double));
            copy(td.bmat, segs->seg_bmat, (size_t)n * sizeof(int32_t));
            if (segs->seg_hit) copy(td.hit, segs->seg_hit, (size_t)n * sizeof(int32_t));
            else if (n) GBT_CUDA(cudaMemsetAsync(td.hit, 0xff, (size_t)n * sizeof(int32_t), s));
            csr_ray_depth_launch(td, s);
            td.n_seg_host = n;
            mark_trace_used(tr, s);
        } catch (...) {
            if (td.block) dfree(td.block, s);
            if (td.used) cudaEventDestroy(td.used);
            delete tr;
            throw;
        }
        *out = tr;
    });
}

gbt_status gbt_trace_info_get(const gbt_trace_t *trace, gbt_trace_info *info)
{
    return guarded([&] {
        GBT_REQUIRE(trace && info, "trace and info must be non-NULL");
        gbt_trace_t *tr = const_cast<gbt_trace_t *>(trace);
        TraceDev &td = tr->d;
        if (td.n_seg_host < 0) td.n_seg_host = read_device_i32(td.ray_off + td.n_rays, td.used);
        memset(info, 0, sizeof(*info));
        info->n_fan = td.n_fan;
        info->ray_begin = td.ray_begin;
        info->n_rays = td.n_rays;
        info->seg_capacity = td.capacity;
        info->n_segments = td.n_seg_host;
        info->ray_off = td.ray_off;
        info->seg_o = td.o; info->seg_t = td.t; info->seg_L = td.L; info->seg_s0 = td.s0;
        info->seg_ray = td.ray; info->seg_depth = td.depth; info->seg_bmat = td.bmat;
        info->seg_hit = td.hit;
    });
}

gbt_status gbt_trace_destroy(gbt_trace_t *trace)
{
    return guarded([&] {
        if (!trace) return;
        cudaStream_t q = after_last_use(trace->d.used);
        trace->d.work.release(q);
        dfree(trace->d.block, q);
        if (trace->d.used) cudaEventDestroy(trace->d.used);
        delete trace;
    });
}

gbt_status gbt_sum(const gbt_trace_t *trace, const gbt_sum_args *args, void *stream)
{
    NvtxRange nvtx_range("gbt_sum");
    return guarded([&] {
        validate_sum(trace, args);
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        gbt_trace_t *tr = const_cast<gbt_trace_t *>(trace);
        const SceneDev &sd = tr->d.scene->d;
        const int splits = choose_splits(tr->d, *args);
        void *w = tr->d.work.ensure(sum_workspace_bytes(tr->d, *args, splits), s);
        sum_launch(tr->d, sd, *args, splits, w, s);
        mark_trace_used(tr, s);
    });
}

gbt_status gbt_synthesize(const float *p, int32_t n_freq, int64_t n_recv, const double *freq_hz,
                          const double *amp, double t0, double dt, int64_t n_t, float *out,
                          int32_t accumulate, void *stream)
{
    NvtxRange nvtx_range("gbt_synthesize");
    return guarded([&] {
        GBT_REQUIRE(n_freq >= 1 && n_freq <= GBT_MAX_FREQ, "n_freq must be in [1, 16]");
        GBT_REQUIRE(n_recv >= 0, "n_recv must be >= 0");
        GBT_REQUIRE(n_t >= 1 && n_t <= (int64_t(1) << 20), "n_t must be in [1, 2^20]");
        GBT_REQUIRE(freq_hz && amp, "freq_hz and amp must be non-NULL");
        GBT_REQUIRE(isfinite(t0) && isfinite(dt), "t0 and dt must be finite");
        for (int f = 0; f < n_freq; ++f)
            GBT_REQUIRE(isfinite(freq_hz[f]) && isfinite(amp[2 * f]) && isfinite(amp[2 * f + 1]),
                        "freq_hz and amp must be finite");
        GBT_REQUIRE(accumulate == 0 || accumulate == 1, "accumulate must be 0 or 1");
        if (n_recv == 0) return;
        GBT_REQUIRE(p && out, "p and out must be non-NULL");
        synth_launch(p, n_freq, n_recv, freq_hz, amp, t0, dt, n_t, out, accumulate,
                     static_cast<cudaStream_t>(stream));
    });
}

// ISO 9613-1: attenuation coefficient of air for pure tones, written from the
// standard's equations: the saturation vapour pressure over the triple-point
// isotherm gives the molar concentration h of water vapour; h and the pressure set
// the relaxation frequencies of oxygen and nitrogen; alpha (dB/m) is 8.686 f^2 times
// the classical-plus-rotational term plus the two vibrational relaxation terms.
// Returned as the amplitude decay rate, alpha / (20 log10 e) Np/m.
gbt_status gbt_air_absorption(int32_t n, const double *freq_hz, double temperature_c,
                              double humidity_pct, double pressure_kpa, double *np_per_m)
{
    return guarded([&] {
        GBT_REQUIRE(n >= 0, "n must be >= 0");
        if (n == 0) return;
        GBT_REQUIRE(freq_hz && np_per_m, "freq_hz and np_per_m must be non-NULL");
        GBT_REQUIRE(isfinite(temperature_c) && temperature_c >= -50.0 && temperature_c <= 60.0,
                    "temperature must be in [-50, 60] C");
        GBT_REQUIRE(isfinite(humidity_pct) && humidity_pct >= 0.0 && humidity_pct <= 100.0,
                    "relative humidity must be in [0, 100] %");
        GBT_REQUIRE(isfinite(pressure_kpa) && pressure_kpa > 0.0, "pressure must be > 0 kPa");
        for (int32_t i = 0; i < n; ++i)
            GBT_REQUIRE(isfinite(freq_hz[i]) && freq_hz[i] > 0.0, "frequencies must be > 0");
        const double t_kelvin = temperature_c + 273.15;
        const double tau = t_kelvin / 293.15;             // over the reference temperature
        const double pa = pressure_kpa / 101.325;         // over the reference pressure
        const double vapour_exp = 4.6151 - 6.8346 * pow(273.16 / t_kelvin, 1.261);
        const double h = humidity_pct * pow(10.0, vapour_exp) / pa;    // percent
        const double f_o = pa * (24.0 + 40400.0 * h * (0.02 + h) / (0.391 + h));
        const double f_n = pa / sqrt(tau) *
                           (9.0 + 280.0 * h * exp(-4.170 * (1.0 / cbrt(tau) - 1.0)));
        const double relax_o = 0.01275 * exp(-2239.1 / t_kelvin);
        const double relax_n = 0.1068 * exp(-3352.0 / t_kelvin);
        const double db_per_np = 20.0 / log(10.0);
        for (int32_t i = 0; i < n; ++i) {
            const double f2 = freq_hz[i] * freq_hz[i];
            const double bracket = 1.84e-11 * sqrt(tau) / pa +
                                   pow(tau, -2.5) * (relax_o / (f_o + f2 / f_o) +
                                                     relax_n / (f_n + f2 / f_n));
            np_per_m[i] = 8.686 * f2 * bracket / db_per_np;
        }
    });
}

gbt_status gbt_recv_order(const float *recv, int64_t n_recv, int32_t *order_out, void *stream)
{
    NvtxRange nvtx_range("gbt_recv_order");
    return guarded([&] {
        GBT_REQUIRE(n_recv >= 0 && n_recv < 2147483647LL, "n_recv out of range");
        if (n_recv == 0) return;
        GBT_REQUIRE(recv && order_out, "recv and order_out must be non-NULL");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t b = recv_order_scratch_bytes(n_recv);
        void *scr = dalloc(b, s);
        try {
            recv_order_launch(recv, n_recv, order_out, scr, s);
        } catch (...) {
            dfree(scr, s);
            throw;
        }
        dfree(scr, s);
    });
}

gbt_status gbt_recv_order_noalloc(const float *recv, int64_t n_recv, int32_t *order_out,
                                  void *stream)
{
    return guarded([&] {
        GBT_REQUIRE(n_recv >= 0, "n_recv must be >= 0");
        if (n_recv == 0) return;
        GBT_REQUIRE(recv && order_out, "recv and order_out must be non-NULL");
        recv_order_noalloc_launch(recv, n_recv, order_out, static_cast<cudaStream_t>(stream));
    });
}

gbt_status gbt_sum_backward(const gbt_trace_t *trace, const gbt_sum_args *args,
                            const float *grad_out, float *grad_gamma, float *grad_ray_weight,
                            double *grad_b, void *stream)
{
    NvtxRange nvtx_range("gbt_sum_backward");
    return guarded([&] {
        validate_sum(trace, args, false);
        GBT_REQUIRE(args->precision == GBT_PRECISION_F32, "backward supports F32 precision only");
        GBT_REQUIRE(grad_gamma, "grad_gamma is NULL");
        GBT_REQUIRE(args->n_recv == 0 || grad_out, "grad_out is NULL");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        gbt_trace_t *tr = const_cast<gbt_trace_t *>(trace);
        const SceneDev &sd = tr->d.scene->d;
        void *w = tr->d.work.ensure(bwd_workspace_bytes(tr->d, *args), s);
        bwd_launch(tr->d, sd, *args, grad_out, grad_gamma, grad_ray_weight, grad_b, w, s);
        mark_trace_used(tr, s);
    });
}

gbt_status gbt_solve(const gbt_scene_t *scene, const gbt_source_desc *src, const gbt_sum_args *args,
                     void *stream)
{
    NvtxRange nvtx_range("gbt_solve");
    return guarded([&] {
        GBT_REQUIRE(scene && src && args, "scene, src and args must be non-NULL");
        GBT_REQUIRE(src->ray_begin == 0 && src->ray_count == 0,
                    "gbt_solve traces the whole fan: ray_begin and ray_count must be 0");
        GBT_REQUIRE(src->fan != GBT_FAN_EXPLICIT,
                    "gbt_solve generates its fan: Fibonacci or lat-long, not explicit");
        GBT_REQUIRE(args->max_device_bytes >= 0, "max_device_bytes must be >= 0");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int64_t N = src->n_rays;
        const int64_t loss = has_losses(*args) ? 16 * (int64_t)args->n_freq : 0;
        const int64_t per_ray = (int64_t)(src->max_reflections + 1) *
                                (80 /*compact*/ + 80 /*padded*/ + 4 * kRecFloats + 32 /*cull*/ + 8 + 8 +
                                 loss);
        int64_t chunk = N;
        if (args->max_device_bytes > 0) {
            chunk = std::max<int64_t>(1, args->max_device_bytes / std::max<int64_t>(per_ray, 1));
        }
        chunk = std::min<int64_t>(chunk, (int64_t)(2147483646LL / (src->max_reflections + 1)));
        gbt_sum_args a = *args;
        if (chunk >= N) {
            // one pass: trace and sum on the caller's stream
            gbt_trace_t *tr = make_trace(scene, *src, s);
            try {
                validate_sum(tr, &a);
                const int splits = choose_splits(tr->d, a);
                void *w = tr->d.work.ensure(sum_workspace_bytes(tr->d, a, splits), s);
                sum_launch(tr->d, scene->d, a, splits, w, s);
            } catch (...) {
                tr->d.work.release(s);
                dfree(tr->d.block, s);
                if (tr->d.used) cudaEventDestroy(tr->d.used);
                delete tr;
                throw;
            }
            tr->d.work.release(s);
            dfree(tr->d.block, s);
            if (tr->d.used) cudaEventDestroy(tr->d.used);
            delete tr;
            mark_used(scene->d.used, s);
            return;
        }
        // Chunks of rays, double-buffered: chunk i is traced on a private stream into slot
        // i % 2 while the caller's stream sums chunk i - 1 from the other slot; every sum
        // accumulates into out in chunk order on the caller's stream.
        validate_source(*src);
        const int nslot = 2;
        TraceDev slot[nslot];
        void *scratch[nslot] = {nullptr, nullptr};
        cudaStream_t ts = nullptr;
        cudaEvent_t ready = nullptr, traced[nslot] = {nullptr, nullptr}, summed[nslot] = {nullptr, nullptr};
        const size_t sb = trace_scratch_bytes(chunk, src->max_reflections);
        // Frees are ordered on s after the last sum, and every trace precedes a sum on s; a
        // failed call may leave a trace in flight, so that path waits for the trace stream.
        auto cleanup = [&](bool failed) {
            if (ts && failed) cudaStreamSynchronize(ts);
            for (int k = 0; k < nslot; ++k) {
                slot[k].work.release(s);
                if (slot[k].block) dfree(slot[k].block, s);
                if (scratch[k]) dfree(scratch[k], s);
                if (traced[k]) cudaEventDestroy(traced[k]);
                if (summed[k]) cudaEventDestroy(summed[k]);
            }
            if (ready) cudaEventDestroy(ready);
            if (ts) cudaStreamDestroy(ts);
        };
        try {
            GBT_CUDA(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
            for (int k = 0; k < nslot; ++k) {
                GBT_CUDA(cudaEventCreateWithFlags(&traced[k], cudaEventDisableTiming));
                GBT_CUDA(cudaEventCreateWithFlags(&summed[k], cudaEventDisableTiming));
                alloc_trace_block(slot[k], scene, *src, chunk, s);
                scratch[k] = dalloc(sb, s);
                // the sum workspace for a full chunk, sized once
                slot[k].ray_begin = 0;
                slot[k].n_rays = chunk;
                slot[k].work.ensure(sum_workspace_bytes(slot[k], a, choose_splits(slot[k], a)), s);
            }
            GBT_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
            GBT_CUDA(cudaEventRecord(ready, s));          // allocations above are ordered on s
            GBT_CUDA(cudaStreamWaitEvent(ts, ready, 0));
            const int64_t nchunks = (N + chunk - 1) / chunk;
            for (int64_t i = 0; i < nchunks; ++i) {
                const int k = (int)(i % nslot);
                TraceDev &td = slot[k];
                gbt_source_desc cs = *src;
                cs.ray_begin = i * chunk;
                cs.ray_count = std::min<int64_t>(chunk, N - cs.ray_begin);
                if (i >= nslot) GBT_CUDA(cudaStreamWaitEvent(ts, summed[k], 0));   // slot free
                td.ray_begin = cs.ray_begin;
                td.n_rays = cs.ray_count;
                td.n_seg_host = -1;
                trace_launch(scene->d, td, cs, scratch[k], sb, ts);
                GBT_CUDA(cudaEventRecord(traced[k], ts));
                GBT_CUDA(cudaStreamWaitEvent(s, traced[k], 0));
                a.accumulate = (i == 0) ? args->accumulate : 1;
                const int splits = choose_splits(td, a);
                sum_launch(td, scene->d, a, splits, td.work.ensure(sum_workspace_bytes(td, a, splits), s), s);
                GBT_CUDA(cudaEventRecord(summed[k], s));
            }
            // the caller's stream is last: every trace was waited for by a sum on it
            mark_used(scene->d.used, s);
        } catch (...) {
            cleanup(true);
            throw;
        }
        cleanup(false);
    });
}

gbt_status gbt_list_capacity_set(int64_t entries)
{
    return guarded([&] {
        GBT_REQUIRE(entries >= 0, "entries must be >= 0");
        set_list_capacity(entries);
    });
}

gbt_status gbt_timing_enable(int32_t enable)
{
    return guarded([&] {
        std::lock_guard<std::mutex> lk(g_timing_mu);
        g_timing.enabled = enable != 0;
    });
}

gbt_status gbt_timing_read(int64_t *launches, double *total_ms, int32_t reset)
{
    return guarded([&] {
        GBT_REQUIRE(launches && total_ms, "launches and total_ms must be non-NULL");
        std::lock_guard<std::mutex> lk(g_timing_mu);
        double ms = 0.0;
        for (auto &pr : g_timing.events) {
            GBT_CUDA(cudaEventSynchronize(pr.second));
            float t = 0.f;
            GBT_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second));
            ms += t;
        }
        *launches = (int64_t)g_timing.events.size();
        *total_ms = ms;
        if (reset) {
            for (auto &pr : g_timing.events) {
                g_timing.pool.push_back(pr.first);
                g_timing.pool.push_back(pr.second);
            }
            g_timing.events.clear();
        }
    });
}

gbt_status gbt_launches_read(int64_t *launches, int32_t reset)
{
    return guarded([&] {
        GBT_REQUIRE(launches, "launches must be non-NULL");
        *launches = reset ? g_launches.exchange(0) : g_launches.load();
    });
}

gbt_status gbt_sum_stats_get(const gbt_trace_t *trace, const gbt_sum_args *args,
                             gbt_sum_stats *stats, void *stream)
{
    return guarded([&] {
        validate_sum(trace, args, false);
        GBT_REQUIRE(stats, "stats is NULL");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        gbt_trace_t *tr = const_cast<gbt_trace_t *>(trace);
        gbt_sum_args a = *args;
        a.precision = GBT_PRECISION_F32;
        const int splits = choose_splits(tr->d, a);
        void *w = tr->d.work.ensure(sum_workspace_bytes(tr->d, a, splits), s);
        unsigned long long *cnt = static_cast<unsigned long long *>(dalloc(64, s));
        GBT_CUDA(cudaMemsetAsync(cnt, 0, 64, s));
        try {
            sum_launch(tr->d, tr->d.scene->d, a, splits, w, s, cnt);
        } catch (...) {
            dfree(cnt, s);
            throw;
        }
        unsigned long long h[4] = {0, 0, 0, 0};
        int32_t nseg = 0;
        GBT_CUDA(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
        GBT_CUDA(cudaMemcpyAsync(&nseg, tr->d.ray_off + tr->d.n_rays, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
        GBT_CUDA(cudaStreamSynchronize(s));
        dfree(cnt, s);
        mark_trace_used(tr, s);
        stats->n_segments = nseg;
        stats->pairs = (int64_t)nseg * a.n_recv;
        stats->pairs_prefiltered = (int64_t)h[1];
        stats->triples_kept = (int64_t)h[2];
        stats->pairs_tested = (int64_t)h[3];
    });
}

gbt_status gbt_batch_create(const gbt_batch_desc *desc, void *stream, gbt_batch_t **out)
{
    return guarded([&] {
        GBT_REQUIRE(desc && out, "desc and out must be non-NULL");
        *out = nullptr;
        GBT_REQUIRE(desc->n_instances >= 1, "n_instances must be >= 1");
        GBT_REQUIRE(desc->traces && desc->args, "traces and args must be non-NULL");
        GBT_REQUIRE(desc->form == GBT_BATCH_AUTO || desc->form == GBT_BATCH_FUSED ||
                        desc->form == GBT_BATCH_CONCURRENT,
                    "form must be GBT_BATCH_AUTO, GBT_BATCH_FUSED or GBT_BATCH_CONCURRENT");
        for (int i = 0; i < desc->n_instances; ++i) validate_sum(desc->traces[i], &desc->args[i]);
        gbt_batch_t *b = new gbt_batch_s();
        try {
            b->impl = batch_create(*desc, static_cast<cudaStream_t>(stream));
        } catch (...) {
            delete b;
            throw;
        }
        *out = b;
    });
}

gbt_status gbt_batch_submit(gbt_batch_t *batch, void *stream)
{
    NvtxRange nvtx_range("gbt_batch_submit");
    return guarded([&] {
        GBT_REQUIRE(batch && batch->impl, "batch is NULL");
        batch_submit(batch->impl, static_cast<cudaStream_t>(stream));
    });
}

gbt_status gbt_batch_destroy(gbt_batch_t *batch)
{
    return guarded([&] {
        if (!batch) return;
        batch_destroy(batch->impl);
        delete batch;
    });
}

gbt_status gbt_selftest_timeout(int64_t spins, void *stream)
{
    return guarded([&] {
        GBT_REQUIRE(spins >= 1 && spins <= (1LL << 24), "spins must be in [1, 2^24]");
        selftest_timeout_launch((long long)spins, static_cast<cudaStream_t>(stream));
    });
}

gbt_status gbt_sync(void *stream)
{
    return guarded([&] {
        GBT_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
        unsigned int *sw = status_word();
        unsigned int v = 0;
        cudaStream_t q = service_stream();
        GBT_CUDA(cudaMemcpyAsync(&v, sw, sizeof(v), cudaMemcpyDeviceToHost, q));
        GBT_CUDA(cudaStreamSynchronize(q));
        if (v) {
            GBT_CUDA(cudaMemsetAsync(sw, 0, sizeof(unsigned int), q));
            GBT_CUDA(cudaStreamSynchronize(q));
            if (v & STATUS_TIMEOUT) fail(GBT_ERR_TIMEOUT, "a bounded device wait ran out");
            fail(GBT_ERR_DEVICE_STATUS, "device status flags 0x" + std::to_string(v));
        }
    });
}

}  // extern "C"
