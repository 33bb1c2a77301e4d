// Measured peak of the warp-level tensor-core MMA forms (mma.sync), the
// denominator of the "% of dense INT8 tensor peak" figure of the modular
// product.  sm_103a has no integer tcgen05 MMA, so the integer tensor path
// available here is mma.sync.m16n8k32 s8 x s8 -> s32; its bf16 counterpart
// (m16n8k16, fp32 accumulate) is timed beside it.  Every warp keeps its
// fragments in registers and runs CHAINS independent accumulations, so the
// loop is bound by the tensor pipe, not by latency or memory.
#include <algorithm>

#include "common.cuh"

namespace pluq {
namespace {

constexpr int CHAINS = 8;
constexpr int PT = 256;   // threads per block

// fragment values (any bit patterns will do) and a word the results are
// folded into, so that no MMA can be dropped as dead code
__device__ uint32_t g_peak_seed[32] = {
    0x01020304u, 0x7f80fe01u, 0x11223344u, 0x55667788u, 0x99aabbccu, 0xddeeff00u, 0x0badf00du,
    0xdeadbeefu, 0x13579bdfu, 0x2468ace0u, 0x0f1e2d3cu, 0x4b5a6978u, 0x8796a5b4u, 0xc3d2e1f0u,
    0x31415926u, 0x27182818u, 0x16180339u, 0x14142135u, 0x17320508u, 0x22360679u, 0x26457513u,
    0x28284271u, 0x30000000u, 0x31622776u, 0x33166247u, 0x34641016u, 0x36055512u, 0x37416573u,
    0x38729833u, 0x40000000u, 0x41231056u, 0x42426406u};
__device__ int32_t g_peak_sink;

__global__ void __launch_bounds__(PT) mma_s8_loop(int iters)
{
    const uint32_t *seed = g_peak_seed;
    const int lane = threadIdx.x & 31;
    uint32_t a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = seed[(lane + i) & 31];
#pragma unroll
    for (int i = 0; i < 2; ++i) b[i] = seed[(lane + 4 + i) & 31];
    int32_t acc[CHAINS][4];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[c][i] = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                "{%8,%9}, {%0,%1,%2,%3};"
                : "+r"(acc[c][0]), "+r"(acc[c][1]), "+r"(acc[c][2]), "+r"(acc[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int32_t s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c][0] ^ acc[c][1] ^ acc[c][2] ^ acc[c][3];
    atomicXor(&g_peak_sink, s);
}

__global__ void __launch_bounds__(PT) mma_bf16_loop(int iters)
{
    const uint32_t *seed = g_peak_seed;
    const int lane = threadIdx.x & 31;
    uint32_t a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = seed[(lane + i) & 31];
#pragma unroll
    for (int i = 0; i < 2; ++i) b[i] = seed[(lane + 4 + i) & 31];
    float acc[CHAINS][4];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[c][i] = 0.0f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
                "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                : "+f"(acc[c][0]), "+f"(acc[c][1]), "+f"(acc[c][2]), "+f"(acc[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
    atomicXor(&g_peak_sink, __float_as_int(s));
}

}  // namespace
}  // namespace pluq

using namespace pluq;

extern "C" pluq_status pluq_measure_mma_sync_peak(int form, double target_ms, double *h_tops,
                                                  double *h_ms)
{
    if ((form != 0 && form != 1) || target_ms <= 0 || !h_tops || !h_ms) return PLUQ_EINVAL;
    int dev = 0, sms = 0;
    PLUQ_CUDA_TRY(cudaGetDevice(&dev));
    PLUQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 4;   // 32 warps per SM
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pluq_status st = PLUQ_ECUDA;
    // ops of one mma.sync: 2 M N K
    const double ops_per = form == 0 ? 2.0 * 16 * 8 * 32 : 2.0 * 16 * 8 * 16;
    auto run = [&](int iters, float &ms) -> bool {
        if (cudaEventRecord(e0, 0) != cudaSuccess) return false;
        if (form == 0) mma_s8_loop<<<blocks, PT>>>(iters);
        else mma_bf16_loop<<<blocks, PT>>>(iters);
        if (last_launch() != PLUQ_OK) return false;
        if (cudaEventRecord(e1, 0) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
            return false;
        return cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    };
    do {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) break;
        float ms = 0;
        if (!run(256, ms)) break;                      // warm-up
        if (!run(2048, ms)) break;                     // calibration
        const int iters =
            (int)std::min(1e9, std::max(2048.0, 2048.0 * target_ms / std::max(ms, 1e-3f)));
        if (!run(iters, ms)) break;
        const double ops = ops_per * CHAINS * (double)iters * (blocks * (PT / 32));
        *h_tops = ops / (ms / 1e3) / 1e12;
        *h_ms = ms;
        st = PLUQ_OK;
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}
