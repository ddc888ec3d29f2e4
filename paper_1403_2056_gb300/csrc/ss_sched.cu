// Device-driven recursion (ss_sort_batch_async): a second copy of the
// engine's kernels, compiled as relocatable device code, with the level
// scheduler that launches them from the device (see the device-driven section
// of ss_kernels.cuh).  Kept apart from ss_engine.cu, whose kernels the host
// launches: compiled this way they measured slower on GB300, so the host
// path keeps its whole-program build.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <type_traits>

#include "ss_internal.cuh"

namespace ss {
namespace dv {

#define SS_KERNELS_SCHEDULER 1
#include "ss_kernels.cuh"

template <typename K>
static cudaError_t smem_attr(K kernel, size_t bytes, bool max_carveout) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e || !max_carveout) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

template <typename K>
static uint32_t per_sm(K kernel, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return (uint32_t)n;
}

// attributes of the kernels the scheduler launches, and the resident grids of
// the base-case classes, once per device
static std::mutex g_mu;
static bool g_done[64];
static uint32_t g_grid[64][2][kClasses];

template <bool A>
static cudaError_t base_attrs(int dev, uint32_t sms) {
    cudaError_t e;
    constexpr int N1 = SS_C1_NT, I1 = 256 / SS_C1_NT, N2 = SS_C2_NT, I2 = 1024 / SS_C2_NT, N3 = SS_C3_NT,
                  I3 = (int)(kSmallMax / SS_C3_NT);
    if ((e = smem_attr(k_base_cta<N1, I1, A>, sizeof(BaseSmem<N1, I1>), true))) return e;
    if ((e = smem_attr(k_base_cta<N2, I2, A>, sizeof(BaseSmem<N2, I2>), true))) return e;
    if ((e = smem_attr(k_base_cta<N3, I3, A>, sizeof(BaseSmem<N3, I3>), true))) return e;
    g_grid[dev][A][1] = sms * per_sm(k_base_cta<N1, I1, A>, N1, sizeof(BaseSmem<N1, I1>));
    g_grid[dev][A][2] = sms * per_sm(k_base_cta<N2, I2, A>, N2, sizeof(BaseSmem<N2, I2>));
    g_grid[dev][A][3] = sms * per_sm(k_base_cta<N3, I3, A>, N3, sizeof(BaseSmem<N3, I3>));
    return cudaSuccess;
}

static cudaError_t attrs(int dev, uint32_t sms) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_done[dev]) return cudaSuccess;
    cudaError_t e;
    if ((e = smem_attr(k_build_trees, sizeof(TreeSmem), false))) return e;
    if ((e = smem_attr(k_classify<kLevelD>, sizeof(ClassifySmem<kLevelD>), false))) return e;
    if ((e = smem_attr(k_scatter<MODE_SORT, kLevelD>, sizeof(ScatterSmem<kLevelD>), true))) return e;
    if ((e = base_attrs<false>(dev, sms))) return e;
    if ((e = base_attrs<true>(dev, sms))) return e;
    g_done[dev] = true;
    return cudaSuccess;
}

}  // namespace dv

int sched_start(SortPlan P, bool any_alpha, cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = dv::attrs(dev, P.sms);
    if (e) return cuda_fail(e, "scheduler kernel attributes");
    for (int k = 0; k < kClasses; k++) P.base_grid[k] = dv::g_grid[dev][any_alpha][k];
    if (any_alpha) {
        SS_LAUNCH("sched", st, dv::k_sched<true><<<1, 32, 0, st>>>(P));
    } else {
        SS_LAUNCH("sched", st, dv::k_sched<false><<<1, 32, 0, st>>>(P));
    }
    e = cudaGetLastError();
    return e ? cuda_fail(e, "scheduler launch") : SS_OK;
}

uint64_t sched_device_launches() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, dv::g_device_launches, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}

void sched_reset_device_launches() {
    const unsigned long long z = 0;
    if (cudaMemcpyToSymbol(dv::g_device_launches, &z, sizeof(z)) != cudaSuccess) cudaGetLastError();
}

int32_t sched_take_device_error() {
    int32_t v = 0;
    const int32_t z = 0;
    if (cudaMemcpyFromSymbol(&v, dv::g_device_error, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return SS_ERR_CUDA;
    }
    if (v && cudaMemcpyToSymbol(dv::g_device_error, &z, sizeof(z)) != cudaSuccess) cudaGetLastError();
    return v;
}

cudaError_t sched_copy_wait(long long budget, uint32_t withhold) {
    cudaError_t e = cudaMemcpyToSymbol(dv::g_copy_wait_cycles, &budget, sizeof(budget));
    if (!e) e = cudaMemcpyToSymbol(dv::g_copy_withheld, &withhold, sizeof(withhold));
    return e;
}

}  // namespace ss
