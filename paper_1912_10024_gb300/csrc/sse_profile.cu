// Kernel timing for calls made with SSE_FLAG_PROFILE: a CUDA event is recorded
// on the launching stream before and after each kernel (no synchronisation);
// sse_profile_read waits for the events and reports the device time per kernel
// name. Events are created on first use per device and reused.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <thread>
#include <vector>

#include "sse.h"
#include "sse_internal.h"

namespace sse {
namespace {

struct Rec {
    const char* name;
    int dev;
    std::thread::id owner;  // the host thread that launched the kernel
    cudaEvent_t e0, e1;
    bool closed;
};
struct Ev {
    int dev;
    cudaEvent_t e;
};

std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<Ev> g_free;
constexpr size_t kMaxRecs = 1 << 16;
thread_local bool t_on = false;

bool take_event(int dev, cudaEvent_t* out) {
    for (size_t i = 0; i < g_free.size(); ++i)
        if (g_free[i].dev == dev) {
            *out = g_free[i].e;
            g_free[i] = g_free.back();
            g_free.pop_back();
            return true;
        }
    return cudaEventCreate(out) == cudaSuccess;
}

}  // namespace

ProfScope::ProfScope(bool on) : prev_(t_on) { t_on = on; }
ProfScope::~ProfScope() { t_on = prev_; }

void prof_begin(const char* name, cudaStream_t st) {
    if (!t_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_recs.size() >= kMaxRecs) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    Rec r{name, dev, std::this_thread::get_id(), nullptr, nullptr, false};
    if (!take_event(dev, &r.e0)) return;
    if (!take_event(dev, &r.e1)) {
        g_free.push_back({dev, r.e0});
        return;
    }
    if (cudaEventRecord(r.e0, st) != cudaSuccess) {
        g_free.push_back({dev, r.e0});
        g_free.push_back({dev, r.e1});
        return;
    }
    g_recs.push_back(r);
}

void prof_end(cudaStream_t st) {
    if (!t_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    // this thread's open record (other threads may be between their own begin and end)
    const std::thread::id me = std::this_thread::get_id();
    for (size_t i = g_recs.size(); i-- > 0;)
        if (!g_recs[i].closed && g_recs[i].owner == me) {
            g_recs[i].closed = cudaEventRecord(g_recs[i].e1, st) == cudaSuccess;
            if (!g_recs[i].closed) {  // drop the record
                g_free.push_back({g_recs[i].dev, g_recs[i].e0});
                g_free.push_back({g_recs[i].dev, g_recs[i].e1});
                g_recs.erase(g_recs.begin() + (long)i);
            }
            return;
        }
}

}  // namespace sse

extern "C" int sse_profile_read(sse_profile_entry* out, int max) {
    using namespace sse;
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<sse_profile_entry> agg;
    int rc = 0;
    for (const Rec& r : g_recs) {
        float ms = 0.0f;
        if (r.closed) {
            if (cudaEventSynchronize(r.e1) != cudaSuccess || cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess)
                rc = -1;
        }
        if (r.closed && rc == 0) {
            size_t k = 0;
            while (k < agg.size() && strcmp(agg[k].name, r.name) != 0) ++k;
            if (k == agg.size()) agg.push_back({r.name, 0.0, 0});
            agg[k].ms += ms;
            agg[k].launches += 1;
        }
        g_free.push_back({r.dev, r.e0});
        g_free.push_back({r.dev, r.e1});
    }
    g_recs.clear();
    if (rc != 0) return -1;
    for (size_t k = 0; k < agg.size() && out && (int)k < max; ++k) out[k] = agg[k];
    return (int)agg.size();
}
