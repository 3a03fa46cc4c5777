// hy_profile.cpp -- kernel-class timing with CUDA events (include/hyperion.h,
// hy_profile_*).  When a class is enabled, the library records an event pair
// on the launching stream around each of its launches of that class, with
// the launch's algorithmic bytes; hy_profile_read resolves the pairs.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "hyperion.h"
#include "hy_internal.h"

namespace hy {
void set_last_error(const std::string &msg);
}

namespace {

struct Pair {
    int cls;
    cudaEvent_t a, b;
    double bytes, flops;
};

struct Acc {
    int64_t launches = 0;
    double ms = 0.0, bytes = 0.0, flops = 0.0;
};

std::atomic<uint32_t> g_mask{0};
std::mutex g_mu;
std::vector<cudaEvent_t> g_free;
std::vector<Pair> g_pending;
Acc g_acc[HY_PROF_CLASSES];

cudaEvent_t take_event()
{
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// resolve the oldest pending pairs until at most `keep` remain (waits)
void resolve(size_t keep)
{
    size_t done = 0;
    while (g_pending.size() - done > keep) {
        Pair &p = g_pending[done++];
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Acc &c = g_acc[p.cls];
            ++c.launches;
            c.ms += ms;
            c.bytes += p.bytes;
            c.flops += p.flops;
        }
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    g_pending.erase(g_pending.begin(), g_pending.begin() + done);
}

}  // namespace

namespace hy {

ProfScope::ProfScope(int cls, void *stream, double bytes, double flops)
    : cls_(cls), stream_(stream), bytes_(bytes), flops_(flops), a_(nullptr)
{
    if (cls < 0 || cls >= HY_PROF_CLASSES || !(g_mask.load() & (1u << cls))) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t e = take_event();
    if (!e) return;
    if (cudaEventRecord(e, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        g_free.push_back(e);
        return;
    }
    a_ = e;
}

ProfScope::~ProfScope()
{
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t a = static_cast<cudaEvent_t>(a_);
    cudaEvent_t b = take_event();
    if (!b || cudaEventRecord(b, static_cast<cudaStream_t>(stream_)) != cudaSuccess) {
        g_free.push_back(a);
        if (b) g_free.push_back(b);
        return;
    }
    g_pending.push_back(Pair{cls_, a, b, bytes_, flops_});
    if (g_pending.size() > 8192) resolve(4096);
}

}  // namespace hy

extern "C" {

hy_status hy_profile_enable(uint32_t class_mask)
{
    std::lock_guard<std::mutex> lk(g_mu);
    resolve(0);
    for (Acc &c : g_acc) c = Acc{};
    g_mask.store(class_mask & ((1u << HY_PROF_CLASSES) - 1u));
    return HY_OK;
}

hy_status hy_profile_read(int cls, int64_t *launches, double *ms, double *bytes, double *flops)
{
    if (cls < 0 || cls >= HY_PROF_CLASSES) {
        hy::set_last_error("profile class out of range");
        return HY_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    resolve(0);
    const Acc &c = g_acc[cls];
    if (launches) *launches = c.launches;
    if (ms) *ms = c.ms;
    if (bytes) *bytes = c.bytes;
    if (flops) *flops = c.flops;
    return HY_OK;
}

}  // extern "C"
