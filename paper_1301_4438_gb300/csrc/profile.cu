// Optional per-kernel-class timing (CUDA events on the launching stream) and a
// running count of kernel launches, read by the benchmark.  Off by default;
// when off, recording costs one branch per launch.
#include <mutex>
#include <vector>

#include "common.cuh"

namespace pluq {
namespace prof {

std::atomic<long long> g_launches{0};
std::atomic<int> g_on{0};

namespace {
struct Rec {
    cudaEvent_t a, b;
    int cls;
    double work;
};
std::mutex mu;
std::vector<Rec> recs;   // event pairs, reused across sessions
size_t used = 0;
cudaEvent_t pending_start[NCLS];
bool has_pending[NCLS];
}  // namespace

void start(int cls, cudaStream_t st)
{
    if (!((g_on.load(std::memory_order_relaxed) >> cls) & 1)) return;
    std::lock_guard<std::mutex> lk(mu);
    if (used == recs.size()) {
        Rec r;
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
        recs.push_back(r);
    }
    Rec &r = recs[used];
    r.cls = cls;
    r.work = 0;
    cudaEventRecord(r.a, st);
    has_pending[cls] = true;
    pending_start[cls] = r.a;
}

void stop(int cls, cudaStream_t st, double work)
{
    if (!((g_on.load(std::memory_order_relaxed) >> cls) & 1)) return;
    std::lock_guard<std::mutex> lk(mu);
    if (used >= recs.size() || !has_pending[cls]) return;
    Rec &r = recs[used];
    r.work = work;
    cudaEventRecord(r.b, st);
    has_pending[cls] = false;
    ++used;
}

void begin_session()
{
    std::lock_guard<std::mutex> lk(mu);
    used = 0;
    for (int c = 0; c < NCLS; ++c) has_pending[c] = false;
}

int read(int cls, long long *launches, double *ms, double *work)
{
    std::lock_guard<std::mutex> lk(mu);
    long long n = 0;
    double t = 0, w = 0;
    for (size_t i = 0; i < used; ++i) {
        if (recs[i].cls != cls) continue;
        if (cudaEventSynchronize(recs[i].b) != cudaSuccess) return -1;
        float e = 0;
        if (cudaEventElapsedTime(&e, recs[i].a, recs[i].b) != cudaSuccess) return -1;
        ++n;
        t += e;
        w += recs[i].work;
    }
    *launches = n;
    *ms = t;
    *work = w;
    return 0;
}

}  // namespace prof
}  // namespace pluq

using namespace pluq;

extern "C" {

long long pluq_launch_count(void) { return prof::g_launches.load(); }

pluq_status pluq_profile_enable(int class_mask)
{
    if (class_mask & ~((1 << prof::NCLS) - 1)) return PLUQ_EINVAL;
    if (class_mask) prof::begin_session();
    prof::g_on.store(class_mask);
    return PLUQ_OK;
}

pluq_status pluq_profile_read(int kernel_class, long long *h_launches, double *h_ms, double *h_work)
{
    if (kernel_class < 0 || kernel_class >= prof::NCLS || !h_launches || !h_ms || !h_work)
        return PLUQ_EINVAL;
    return prof::read(kernel_class, h_launches, h_ms, h_work) == 0 ? PLUQ_OK : PLUQ_ECUDA;
}

}  // extern "C"
