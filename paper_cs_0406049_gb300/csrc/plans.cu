// plans.cu -- launch plans: defaults, the tuned-plan cache (in memory and as
// a JSON file) and the autotuner that fills it.
//
// A plan is (threads per CTA, vectors in flight per thread, resident CTAs per
// SM, bytes per vector access -- or 0 for the bulk-copy path).  Plans are
// keyed by device ("<name>:<SMs>"), operation, output dtype and the bit
// length of the element count, so one tuning run per size class covers every
// later call in that class.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "trace.h"
#include "internal.h"

namespace sincos_gb300 {

namespace {

using PlanKey = std::tuple<std::string, int, int, int>;   // device, op, dtype, bucket

std::mutex g_plan_mu;
std::map<PlanKey, sincos_plan> g_plans;
// Bumped on every change of g_plans; a thread's last lookup (plan_for) stays
// valid while it is unchanged.
std::atomic<uint64_t> g_plans_version{0};
std::once_flag g_env_once;

int bucket_of(int64_t n)
{
    int b = 0;
    while (n > 0) {
        ++b;
        n >>= 1;
    }
    return b;
}

std::string device_key(const DeviceInfo &dev)
{
    return std::string(dev.name) + ":" + std::to_string(dev.sms);
}

// Single arrays below 2^24 angles (power-of-two buckets up to 24) run the
// 4096-angle stages with 256-thread CTAs, several per SM, for every output
// type.  The big stages of the large-array default leave a partial last round
// there (2^22 binary32 angles: 512 chunks on 152 SMs).  A GB300 sweep in
// quarter-octave steps from 2^18 to 2^26 angles, against the large-array
// defaults (geometric mean of the ratios; back-to-back calls / L2 flushed
// between calls): 2^21..2^24 binary32 1.09 / 1.09, 16-bit 1.07-1.08 / 1.02;
// 2^18..2^21 binary32 1.01 / 1.14, 16-bit 1.01 / 1.02; 2^24..2^26 binary32
// 0.96 / 0.99 and 16-bit 0.99 / 1.00-1.01, where the defaults stay.
constexpr int kSmallStageBuckets = 24;

sincos_plan default_plan(int op, int dtype, int bucket)
{
    if (op == SINCOS_OP_PAIRS && bucket <= kSmallStageBuckets) return sincos_plan{256, 2, 2, 0};
    // Fastest plans of a GB300 sweep (2^26..2^28 elements, 4096-array batch).
    // About 1024 resident threads per SM with 2..8 vectors in flight each
    // beat full occupancy: fewer concurrent streams keep DRAM pages open.
    // The single-array forward defaults to the bulk (TMA-staged) path: 8192-
    // angle stages for binary32, 4096-angle stages (three CTAs per SM) for
    // 16-bit outputs, which with programmatic dependent launch beat the
    // 32-byte register path (6480 against 6350 GB/s at 2^26).  The batched
    // ring kernel likewise runs 4096-angle stages for binary32 (two CTAs per
    // SM: 6410 against 6256 GB/s plain, 6391 against 6111 compensated on the
    // 4096-array workload); batched 16-bit outputs keep the register path
    // (5740-5860 GB/s; the small-stage ring gave 6000 plain but 5555
    // compensated).
    if (op == SINCOS_OP_BACKWARD) return sincos_plan{512, 2, 2, 16};
    if (op == SINCOS_OP_EXPI) return sincos_plan{512, 2, 1, 0};
    if (op == SINCOS_OP_HUYGENS) return sincos_plan{256, 1, 8, 32};
    if (op == SINCOS_OP_BATCHED)
        return dtype == SINCOS_F32 ? sincos_plan{512, 2, 2, 0} : sincos_plan{1024, 2, 1, 16};
    return dtype == SINCOS_F32 ? sincos_plan{512, 2, 1, 0} : sincos_plan{512, 2, 3, 0};
}

int load_file(const char *path);

void load_env_cache()
{
    const char *p = std::getenv("SINCOS_TUNE_CACHE");
    if (p && *p) load_file(p);
}

// Minimal reader for the file written by sincos_plan_cache_save: finds each
// {...} object after "plans" and reads its string and integer fields.
bool read_string(const char *&p, std::string &out)
{
    if (*p != '"') return false;
    ++p;
    out.clear();
    while (*p && *p != '"') {
        if (*p == '\\' && p[1]) ++p;
        out.push_back(*p++);
    }
    if (*p != '"') return false;
    ++p;
    return true;
}

void skip_ws(const char *&p)
{
    while (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t' || *p == ',') ++p;
}

int load_file(const char *path)
{
    FILE *f = std::fopen(path, "rb");
    if (!f) return SINCOS_EINVAL;
    std::string text;
    char buf[4096];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, k);
    std::fclose(f);
    const char *p = std::strstr(text.c_str(), "\"plans\"");
    if (!p) return SINCOS_EINVAL;
    p = std::strchr(p, '[');
    if (!p) return SINCOS_EINVAL;
    ++p;
    std::map<PlanKey, sincos_plan> loaded;
    for (;;) {
        skip_ws(p);
        if (*p != '{') break;
        ++p;
        std::string device;
        long op = -1, dtype = -1, bucket = -1, block = 0, unroll = 0, ctas = 0, vec = 0;
        for (;;) {
            skip_ws(p);
            if (*p == '}') {
                ++p;
                break;
            }
            std::string key;
            if (!read_string(p, key)) return SINCOS_EINVAL;
            skip_ws(p);
            if (*p != ':') return SINCOS_EINVAL;
            ++p;
            skip_ws(p);
            if (*p == '"') {
                std::string val;
                if (!read_string(p, val)) return SINCOS_EINVAL;
                if (key == "device") device = val;
            } else {
                char *end = nullptr;
                const long v = std::strtol(p, &end, 10);
                if (end == p) return SINCOS_EINVAL;
                p = end;
                if (key == "op") op = v;
                else if (key == "dtype") dtype = v;
                else if (key == "bucket") bucket = v;
                else if (key == "block") block = v;
                else if (key == "unroll") unroll = v;
                else if (key == "ctas_per_sm") ctas = v;
                else if (key == "vec_bytes") vec = v;
            }
        }
        sincos_plan plan{(int)block, (int)unroll, (int)ctas, (int)vec};
        if (device.empty() || op < 0 || dtype < 0 || bucket < 0 || !plan_valid(plan))
            return SINCOS_EINVAL;
        loaded[PlanKey(device, (int)op, (int)dtype, (int)bucket)] = plan;
    }
    std::lock_guard<std::mutex> lock(g_plan_mu);
    for (auto &kv : loaded) g_plans[kv.first] = kv.second;
    g_plans_version.fetch_add(1, std::memory_order_release);
    return SINCOS_OK;
}

void store_plan(const DeviceInfo &dev, int op, int dtype, int64_t n, const sincos_plan &p)
{
    std::lock_guard<std::mutex> lock(g_plan_mu);
    g_plans[PlanKey(device_key(dev), op, dtype, bucket_of(n))] = p;
    g_plans_version.fetch_add(1, std::memory_order_release);
}

std::vector<sincos_plan> candidates(const DeviceInfo &dev, int op)
{
    std::vector<sincos_plan> out;
    if (op == SINCOS_OP_HUYGENS) {  // CTA size and points per thread only
        for (int block : {128, 256, 512})
            for (int pts : {1, 2, 4})
                for (int vec : {16, 32}) out.push_back(sincos_plan{block, pts, 8, vec});
        return out;
    }
    if (op != SINCOS_OP_BACKWARD)   // bulk path: one CTA per SM, CTA size only
        for (int block : {128, 256, 512, 1024}) out.push_back(sincos_plan{block, 2, 1, 0});
    if (op == SINCOS_OP_PAIRS || op == SINCOS_OP_BATCHED)   // 4096-angle stages, several CTAs per SM
        for (int block : {128, 256, 512}) out.push_back(sincos_plan{block, 2, 2, 0});
    const int max_threads = dev.max_threads_per_sm > 0 ? dev.max_threads_per_sm : 2048;
    for (int vec : {16, 32})
        for (int block : {128, 256, 512, 1024})
            for (int unroll : {1, 2, 4, 8})
                for (int ctas : {1, 2, 4, 8, 16})
                    if (block * ctas <= max_threads)
                        out.push_back(sincos_plan{block, unroll, ctas, vec});
    return out;
}

// Event-timed launches on one stream.
struct LaunchTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    bool ok = false;
    LaunchTimer()
    {
        ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    }
    ~LaunchTimer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    // Duration of `runs` back-to-back runs of `launch` on `st` in
    // milliseconds per run, or -1.
    template <class F>
    float once(F &&launch, cudaStream_t st, int runs = 1)
    {
        if (!ok) return -1.f;
        cudaEventRecord(a, st);
        for (int r = 0; r < runs; ++r)
            if (launch() != SINCOS_OK) return -1.f;
        cudaEventRecord(b, st);
        float t = 0.f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess)
            return -1.f;
        return t / (float)runs;
    }
};

float median_of(std::vector<float> v)
{
    std::sort(v.begin(), v.end());
    return v[v.size() / 2];
}

bool stream_is_capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Two rounds.  The screen times every candidate (one warm-up run, median of
// three bursts of two back-to-back runs, so that a plan whose launches
// overlap is not screened out on isolated launches); with a hundred
// candidates the single fastest median is
// often a lucky one, so the few fastest are then timed again round-robin --
// one burst of back-to-back runs of each per pass, so that a change of clock
// or of L2 state shifts them all alike, and so that what is timed is the
// steady rate of repeated calls, launch gaps included (and the overlap that
// programmatic dependent launch gives the bulk kernels: 8 runs per burst, so
// that 7 of them can follow their predecessor directly) -- and the lowest
// median of those passes wins.
constexpr int kScreenReps = 3;
constexpr int kScreenBurst = 2;
constexpr int kFinalists = 6;
constexpr int kConfirmPasses = 9;
constexpr int kConfirmBurst = 8;

template <class F>
int tune(const DeviceInfo &dev, int op, int dtype, int64_t n, cudaStream_t st, F &&launch_with,
         sincos_plan *best)
{
    if (stream_is_capturing(st)) return SINCOS_ECAPTURE;
    LaunchTimer timer;
    if (!timer.ok) return SINCOS_ECUDA;
    std::vector<std::pair<float, sincos_plan>> screened;
    for (const sincos_plan &p : candidates(dev, op)) {
        auto run = [&] { return launch_with(p); };
        if (run() != SINCOS_OK) continue;
        std::vector<float> ms;
        for (int r = 0; r < kScreenReps; ++r) {
            const float t = timer.once(run, st, kScreenBurst);
            if (t < 0.f) break;
            ms.push_back(t);
        }
        if ((int)ms.size() == kScreenReps) screened.emplace_back(median_of(ms), p);
    }
    cudaStreamSynchronize(st);
    cudaGetLastError();
    if (screened.empty()) return SINCOS_ECUDA;
    std::stable_sort(screened.begin(), screened.end(),
                     [](const auto &l, const auto &r) { return l.first < r.first; });
    if ((int)screened.size() > kFinalists) screened.resize(kFinalists);

    std::vector<std::vector<float>> ms(screened.size());
    for (int pass = 0; pass < kConfirmPasses; ++pass)
        for (size_t i = 0; i < screened.size(); ++i) {
            const float t =
                timer.once([&] { return launch_with(screened[i].second); }, st, kConfirmBurst);
            if (t > 0.f) ms[i].push_back(t);
        }
    cudaStreamSynchronize(st);
    cudaGetLastError();
    float best_ms = -1.f;
    sincos_plan best_plan = screened[0].second;
    for (size_t i = 0; i < screened.size(); ++i) {
        if (ms[i].empty()) continue;
        const float t = median_of(ms[i]);
        if (best_ms < 0.f || t < best_ms) {
            best_ms = t;
            best_plan = screened[i].second;
        }
    }
    if (best_ms < 0.f) return SINCOS_ECUDA;
    store_plan(dev, op, dtype, n, best_plan);
    if (best) *best = best_plan;
    return SINCOS_OK;
}

}  // namespace

bool plan_valid(const sincos_plan &p)
{
    return p.block >= 64 && p.block <= 1024 && p.block % 32 == 0 &&
           (p.unroll == 1 || p.unroll == 2 || p.unroll == 4 || p.unroll == 8) &&
           p.ctas_per_sm >= 1 && p.ctas_per_sm <= 32 &&
           (p.vec_bytes == 0 || p.vec_bytes == 16 || p.vec_bytes == 32) &&
           (p.vec_bytes != 0 || p.block == 128 || p.block == 256 || p.block == 512 ||
            p.block == 1024);
}

sincos_plan plan_for(const DeviceInfo &dev, int op, int dtype, int64_t n)
{
    std::call_once(g_env_once, load_env_cache);
    // Repeated calls of one kind (the common case) reuse the calling
    // thread's last answer while no plan has changed since.
    struct Last {
        uint64_t version = ~0ull;
        int ordinal = -1, op = -1, dtype = -1, bucket = -1;
        sincos_plan plan{};
    };
    thread_local Last last;
    const int bucket = bucket_of(n);
    const uint64_t version = g_plans_version.load(std::memory_order_acquire);
    if (last.version == version && last.ordinal == dev.ordinal && last.op == op &&
        last.dtype == dtype && last.bucket == bucket)
        return last.plan;
    sincos_plan p;
    {
        std::lock_guard<std::mutex> lock(g_plan_mu);
        auto it = g_plans.find(PlanKey(device_key(dev), op, dtype, bucket));
        p = it != g_plans.end() ? it->second : default_plan(op, dtype, bucket);
    }
    last = Last{version, dev.ordinal, op, dtype, bucket, p};
    return p;
}

// Defined in batched_api.cu: per-(device, stream) prefix scratch.
int batched_scratch(cudaStream_t st, int count, int64_t **prefix);

}  // namespace sincos_gb300

using namespace sincos_gb300;

extern "C" {

int sincos_plan_get(int op, int out_dtype, int64_t n, sincos_plan *plan)
{
    if (!plan || op < 0 || op > 4 || !valid_dtype(out_dtype) || n < 0) return SINCOS_EINVAL;
    const DeviceInfo *dev = nullptr;
    const int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    *plan = plan_for(*dev, op, out_dtype, n);
    return SINCOS_OK;
}

int sincos_plan_set(int op, int out_dtype, int64_t n, const sincos_plan *plan)
{
    if (!plan || op < 0 || op > 4 || !valid_dtype(out_dtype) || n < 0 || !plan_valid(*plan))
        return SINCOS_EINVAL;
    const DeviceInfo *dev = nullptr;
    const int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    std::call_once(g_env_once, load_env_cache);
    store_plan(*dev, op, out_dtype, n, *plan);
    return SINCOS_OK;
}

int sincos_autotune_pairs(const float *x, void *s, void *c, int64_t n, int out_dtype,
                          int reduction, int coef, sincos_stream_t stream, sincos_plan *best)
{
    SINCOS_TRACE("sincos_autotune_pairs");
    if (n <= 0 || !x || !s || !c || !valid_dtype(out_dtype) || !valid_reduction(reduction) ||
        !valid_coef(coef))
        return SINCOS_EINVAL;
    if (!aligned_to(x, 4) || !aligned_to(s, dtype_size(out_dtype)) ||
        !aligned_to(c, dtype_size(out_dtype)))
        return SINCOS_EINVAL;
    const size_t xb = (size_t)n * 4, ob = (size_t)n * dtype_size(out_dtype);
    for (const void *o : {(const void *)s, (const void *)c})
        if (ranges_overlap(x, xb, o, ob)) return SINCOS_EOVERLAP;
    const DeviceInfo *dev = nullptr;
    const int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    std::call_once(g_env_once, load_env_cache);
    cudaStream_t st = (cudaStream_t)stream;
    return tune(*dev, SINCOS_OP_PAIRS, out_dtype, n, st,
                [&](const sincos_plan &p) {
                    return launch_forward(x, s, c, n, out_dtype, reduction, coef, false, p, *dev, st);
                },
                best);
}

int sincos_autotune_expi(const float *x, float *z, int64_t n, int reduction, int coef,
                         sincos_stream_t stream, sincos_plan *best)
{
    SINCOS_TRACE("sincos_autotune_expi");
    if (n <= 0 || !x || !z || !valid_reduction(reduction) || !valid_coef(coef))
        return SINCOS_EINVAL;
    if (!all_float_aligned({x, z})) return SINCOS_EINVAL;
    if (ranges_overlap(x, 4u * (size_t)n, z, 8u * (size_t)n)) return SINCOS_EOVERLAP;
    const DeviceInfo *dev = nullptr;
    const int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    std::call_once(g_env_once, load_env_cache);
    cudaStream_t st = (cudaStream_t)stream;
    return tune(*dev, SINCOS_OP_EXPI, SINCOS_F32, n, st,
                [&](const sincos_plan &p) {
                    return launch_expi(x, z, n, reduction, coef, p, *dev, st);
                },
                best);
}

int sincos_autotune_huygens(const float *px, const float *py, const float *pz, int64_t m,
                            const float *qx, const float *qy, const float *qz, const float *ar,
                            const float *ai, int64_t n, float k, int reduction, float *u,
                            sincos_stream_t stream, sincos_plan *best)
{
    SINCOS_TRACE("sincos_autotune_huygens");
    if (m <= 0 || n < 0 || !px || !py || !pz || !u || !valid_reduction(reduction))
        return SINCOS_EINVAL;
    if (n > 0 && (!qx || !qy || !qz || !ar || !ai)) return SINCOS_EINVAL;
    if (!all_float_aligned({px, py, pz, qx, qy, qz, ar, ai, u})) return SINCOS_EINVAL;
    const DeviceInfo *dev = nullptr;
    const int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    std::call_once(g_env_once, load_env_cache);
    cudaStream_t st = (cudaStream_t)stream;
    return tune(*dev, SINCOS_OP_HUYGENS, SINCOS_F32, m, st,
                [&](const sincos_plan &p) {
                    return launch_huygens(px, py, pz, m, qx, qy, qz, ar, ai, n, k, reduction, u,
                                          p, st);
                },
                best);
}

int sincos_autotune_backward(const float *gs, const float *gc, const float *s, const float *c,
                             float *gx, int64_t n, sincos_stream_t stream, sincos_plan *best)
{
    SINCOS_TRACE("sincos_autotune_backward");
    if (n <= 0 || !gx || !s || !c) return SINCOS_EINVAL;
    if (!all_float_aligned({gs, gc, s, c, gx})) return SINCOS_EINVAL;
    for (const float *in : {gs, gc, s, c})
        if (in && ranges_overlap(in, 4u * (size_t)n, gx, 4u * (size_t)n)) return SINCOS_EOVERLAP;
    const DeviceInfo *dev = nullptr;
    const int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    std::call_once(g_env_once, load_env_cache);
    cudaStream_t st = (cudaStream_t)stream;
    return tune(*dev, SINCOS_OP_BACKWARD, SINCOS_F32, n, st,
                [&](const sincos_plan &p) {
                    return launch_backward(gs, gc, s, c, gx, n, false, p, *dev, st);
                },
                best);
}

int sincos_autotune_batched(const sincos_seg *segs, const int64_t *lens, int count,
                            int out_dtype, int reduction, int coef, sincos_stream_t stream,
                            sincos_plan *best)
{
    SINCOS_TRACE("sincos_autotune_batched");
    if (count <= 0 || !segs || !lens || !valid_dtype(out_dtype) || !valid_reduction(reduction) ||
        !valid_coef(coef))
        return SINCOS_EINVAL;
    if (!aligned_to(segs, 8) || !aligned_to(lens, 8)) return SINCOS_EINVAL;
    const DeviceInfo *dev = nullptr;
    int rc = current_device(&dev);
    if (rc != SINCOS_OK) return rc;
    std::call_once(g_env_once, load_env_cache);
    cudaStream_t st = (cudaStream_t)stream;
    if (stream_is_capturing(st)) return SINCOS_ECAPTURE;
    int64_t *prefix = nullptr;
    rc = batched_scratch(st, count, &prefix);
    if (rc != SINCOS_OK) return rc;
    return tune(*dev, SINCOS_OP_BATCHED, out_dtype, count, st,
                [&](const sincos_plan &p) {
                    return launch_batched(segs, lens, count, out_dtype, reduction, coef, prefix, p,
                                          *dev, st);
                },
                best);
}

int sincos_plan_cache_save(const char *path)
{
    if (!path) return SINCOS_EINVAL;
    FILE *f = std::fopen(path, "wb");
    if (!f) return SINCOS_EINVAL;
    std::lock_guard<std::mutex> lock(g_plan_mu);
    std::fprintf(f, "{\"version\": 1, \"plans\": [");
    bool first = true;
    for (auto &kv : g_plans) {
        std::string dev;
        for (char ch : std::get<0>(kv.first)) {
            if (ch == '"' || ch == '\\') dev.push_back('\\');
            dev.push_back(ch);
        }
        std::fprintf(f,
                     "%s\n  {\"device\": \"%s\", \"op\": %d, \"dtype\": %d, \"bucket\": %d, "
                     "\"block\": %d, \"unroll\": %d, \"ctas_per_sm\": %d, \"vec_bytes\": %d}",
                     first ? "" : ",", dev.c_str(), std::get<1>(kv.first), std::get<2>(kv.first),
                     std::get<3>(kv.first), kv.second.block, kv.second.unroll,
                     kv.second.ctas_per_sm, plan_vec_bytes(kv.second));
        first = false;
    }
    std::fprintf(f, "\n]}\n");
    return std::fclose(f) == 0 ? SINCOS_OK : SINCOS_EINVAL;
}

int sincos_plan_cache_load(const char *path)
{
    if (!path) return SINCOS_EINVAL;
    std::call_once(g_env_once, load_env_cache);
    return load_file(path);
}

}  // extern "C"
