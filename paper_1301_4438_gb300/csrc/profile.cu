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
    bool done;
};
std::mutex mu;
std::vector<Rec> recs;   // event pairs, reused across sessions
size_t used = 0;
// the open record of each class, per host thread (recursion branches and batch
// workers launch from several threads at once)
thread_local long open_rec[NCLS] = {-1, -1, -1, -1, -1, -1};
thread_local unsigned open_session[NCLS] = {0, 0, 0, 0, 0, 0};
unsigned session = 1;
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
    r.done = false;
    cudaEventRecord(r.a, st);
    open_rec[cls] = (long)used;
    open_session[cls] = session;
    ++used;
}

void stop(int cls, cudaStream_t st, double work)
{
    if (!((g_on.load(std::memory_order_relaxed) >> cls) & 1)) return;
    std::lock_guard<std::mutex> lk(mu);
    const long i = open_rec[cls];
    if (i < 0 || open_session[cls] != session || (size_t)i >= used) return;
    Rec &r = recs[i];
    r.work = work;
    cudaEventRecord(r.b, st);
    r.done = true;
    open_rec[cls] = -1;
}

void begin_session()
{
    std::lock_guard<std::mutex> lk(mu);
    used = 0;
    ++session;
}

int read(int cls, long long *launches, double *ms, double *work)
{
    std::lock_guard<std::mutex> lk(mu);
    long long n = 0;
    double t = 0, w = 0;
    for (size_t i = 0; i < used; ++i) {
        if (recs[i].cls != cls || !recs[i].done) continue;
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
