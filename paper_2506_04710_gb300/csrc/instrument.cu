// Launch counting and optional per-kernel-class CUDA-event timing.
// Every kernel launch site in the library opens a KScope; when timing is
// enabled for the scope's class, an event pair is recorded on the launch
// stream around the launch and the elapsed time is accumulated on read.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "instrument.cuh"

namespace ztoep {

static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_mask{0};
static thread_local uint64_t *t_capture_sink = nullptr;  // launches recorded into a graph

void capture_count_begin(uint64_t *sink) { t_capture_sink = sink; }
void capture_count_end() { t_capture_sink = nullptr; }
void add_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool timing_serial() { return (g_mask.load(std::memory_order_relaxed) & ZTOEP_TIMING_SERIAL) != 0; }

struct Pending {
    int cls;
    cudaEvent_t a, b;
};

static std::mutex g_mu;
static std::vector<Pending> g_pending;
static std::vector<cudaEvent_t> g_pool;
static uint64_t g_count[K_NCLASS];
static double g_ms[K_NCLASS];

static cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

KScope::KScope(KClass c, cudaStream_t s) : cls_(c), s_(s), a_(nullptr) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s_, &cs);
    capturing_ = cs != cudaStreamCaptureStatusNone;
    if (!capturing_ && (g_mask.load(std::memory_order_relaxed) & (1 << c))) {
        std::lock_guard<std::mutex> lk(g_mu);
        a_ = take_event();
        cudaEventRecord(a_, s_);
    }
}

KScope::~KScope() {
    if (capturing_) {  // counted when the graph runs
        if (t_capture_sink) *t_capture_sink += n_;
        return;
    }
    g_launches.fetch_add(n_, std::memory_order_relaxed);
    if (a_) {
        std::lock_guard<std::mutex> lk(g_mu);
        cudaEvent_t b = take_event();
        cudaEventRecord(b, s_);
        g_pending.push_back({cls_, a_, b});
    }
}

static void drain() {  // caller holds g_mu
    for (auto &p : g_pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            g_ms[p.cls] += ms;
            g_count[p.cls] += 1;
        }
        g_pool.push_back(p.a);
        g_pool.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace ztoep

using namespace ztoep;

extern "C" {

uint64_t ztoep_launch_count(void) { return g_launches.load(); }

void ztoep_timing_enable(int32_t mask) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_mask.store(mask);
}

void ztoep_timing_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain();
    for (int c = 0; c < K_NCLASS; ++c) { g_count[c] = 0; g_ms[c] = 0.0; }
}

ztoep_status_t ztoep_timing_read(int32_t cls, uint64_t *timed_launches, double *total_ms) {
    if (cls < 0 || cls >= K_NCLASS || !timed_launches || !total_ms) return ZTOEP_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    drain();
    *timed_launches = g_count[cls];
    *total_ms = g_ms[cls];
    return ZTOEP_OK;
}

}  // extern "C"
