// Microbenchmarks that measure the denominators of the roofline fractions on
// the device the library runs on (rom_measure_peak): the FP32 and FP64 FMA
// pipes of the SIMT cores, the tcgen05 tensor pipe for kind::tf32 and
// kind::f16 (BF16) products, and the L2 read bandwidth.  Each kernel is a
// plain throughput loop over every SM; none computes anything of the model.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rom_internal.h"
#include "tc_common.cuh"

namespace romk {
namespace {

constexpr int kFmaChains = 8;      // independent FMA chains per thread
constexpr int kFmaThreads = 512;
constexpr int kMmaN = 256;         // MMA N (M = 128): the full-rate shape
constexpr int kMmaThreads = 128;
constexpr size_t kMmaSmem = 120 * 1024;  // > half an SM's shared memory: one CTA per SM
constexpr int kL2Threads = 512;

// x <- x * b + a on kFmaChains independent chains; the sum is stored only if it
// equals a value it never takes, so the loop cannot be removed.
template <typename T>
__global__ void __launch_bounds__(kFmaThreads) fma_peak_kernel(T a, T b, int iters, T* out) {
    T x[kFmaChains];
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) x[i] = a * (T)(i + 1) + (T)threadIdx.x * (T)1e-6;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kFmaChains; ++i) x[i] = fma(x[i], b, a);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kFmaChains; ++i) s += x[i];
    if (s == (T)-1.25) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One CTA per SM: lane 0 of warp 0 issues `iters` back-to-back 128 x 256 MMAs
// (K = 16 for BF16, K = 8 for TF32) from resident tiles into one TMEM
// accumulator, then waits (bounded) for their completion.
template <bool TF32>
__global__ void __launch_bounds__(kMmaThreads, 1) mma_peak_kernel(int iters, long long limit, int* timed_out) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* A = smem;                              // 128 rows x 128 B
    unsigned char* B = smem + 128 * 128;                  // 256 rows x 128 B
    uint64_t* done = reinterpret_cast<uint64_t*>(B + kMmaN * 128);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // small nonzero operands (BF16 pairs of 2^-7; read as TF32 the same words
    // are 2^-7 too), so that the pipe switches as it does on real data
    const uint32_t w = 0x3C003C00u;
    for (int i = tid; i < (128 + kMmaN) * 128 / 16; i += kMmaThreads)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(w, w, w, w);
    if (tid == 0) {
        mbarrier_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) { tmem_alloc(tslot, (uint32_t)kMmaN); tmem_relinquish(); }
    fence_proxy_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    if (warp == 0 && lane == 0) {
        const uint32_t idesc = mma_idesc(TF32 ? kFmtTF32 : kFmtBF16, 128u, (uint32_t)kMmaN);
        const uint32_t sA = cvta_shared(A), sB = cvta_shared(B);
        for (int it = 0; it < iters; ++it) {
            const uint32_t ko = 32u * (uint32_t)(it & 3);  // the four K steps of a 128-byte row
            mma_issue<TF32>(tbase, sw128_desc(sA + ko), sw128_desc(sB + ko), idesc, it > 0 ? 1u : 0u);
        }
        mma_commit(done);
        const long long t0 = clock64();
        while (!mbarrier_try_wait(done, 0)) {
            if (clock64() - t0 > limit) { atomicExch(timed_out, 1); break; }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, (uint32_t)kMmaN);
}

// Each block reads its slice of an L2-resident buffer `passes` times with
// 16-byte loads that are cached in L2 only.
__global__ void __launch_bounds__(kL2Threads) l2_read_kernel(const float4* __restrict__ buf, size_t n4,
                                                             int passes, float* out) {
    const size_t per = (n4 + gridDim.x - 1) / gridDim.x;
    const size_t lo = blockIdx.x * per;
    const size_t hi = lo + per < n4 ? lo + per : n4;
    float s = 0.f;
    for (int p = 0; p < passes; ++p)
        for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const float4 v = __ldcg(buf + i);
            s += v.x + v.y + v.z + v.w;
        }
    if (s == -1.25f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

struct Timer {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t init() {
        cudaError_t e = cudaEventCreate(&e0);
        return e == cudaSuccess ? cudaEventCreate(&e1) : e;
    }
    ~Timer() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

}  // namespace
}  // namespace romk

using namespace romk;

extern "C" rom_status rom_measure_peak(int kind, double* value, double* ms_out, void* stream) {
    if (!value || kind < ROM_PEAK_FP32 || kind > ROM_PEAK_L2) return ROM_E_INVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "rom_measure_peak");
    Timer tm;
    e = tm.init();
    if (e != cudaSuccess) return cuda_fail(e, "rom_measure_peak events");
    void* scratch = nullptr;
    int* flag = nullptr;
    const size_t l2_bytes = (size_t)32 << 20;
    const size_t out_bytes = (size_t)nsm * 4 * kFmaThreads * sizeof(double);
    e = cudaMalloc(&scratch, kind == ROM_PEAK_L2 ? l2_bytes + out_bytes : out_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (kind == ROM_PEAK_L2 && e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, l2_bytes, st);
    double work = 0.0;  // flops or bytes of the timed launch
    auto launch = [&](bool timed) -> cudaError_t {
        cudaError_t r = cudaSuccess;
        if (timed) r = cudaEventRecord(tm.e0, st);
        if (r != cudaSuccess) return r;
        switch (kind) {
            case ROM_PEAK_FP32:
            case ROM_PEAK_FP64: {
                const int blocks = nsm * 4, iters = kind == ROM_PEAK_FP32 ? 65536 : 2048;
                if (kind == ROM_PEAK_FP32)
                    fma_peak_kernel<float><<<blocks, kFmaThreads, 0, st>>>(1e-3f, 0.999f, iters,
                                                                          static_cast<float*>(scratch));
                else
                    fma_peak_kernel<double><<<blocks, kFmaThreads, 0, st>>>(1e-3, 0.999, iters,
                                                                           static_cast<double*>(scratch));
                work = 2.0 * blocks * kFmaThreads * (double)kFmaChains * iters;
                break;
            }
            case ROM_PEAK_TF32:
            case ROM_PEAK_BF16: {
                const bool tf = kind == ROM_PEAK_TF32;
                const int iters = 100000;
                void* fn = tf ? (void*)&mma_peak_kernel<true> : (void*)&mma_peak_kernel<false>;
                r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMmaSmem);
                if (r != cudaSuccess) return r;
                if (tf)
                    mma_peak_kernel<true><<<nsm, kMmaThreads, kMmaSmem, st>>>(iters, 4000000000LL, flag);
                else
                    mma_peak_kernel<false><<<nsm, kMmaThreads, kMmaSmem, st>>>(iters, 4000000000LL, flag);
                work = 2.0 * 128.0 * kMmaN * (tf ? 8.0 : 16.0) * iters * nsm;
                break;
            }
            case ROM_PEAK_L2: {
                const int passes = 512;  // about 1 ms at L2 rates
                l2_read_kernel<<<nsm * 4, kL2Threads, 0, st>>>(
                    static_cast<const float4*>(scratch), l2_bytes / 16, passes,
                    reinterpret_cast<float*>(static_cast<unsigned char*>(scratch) + l2_bytes));
                work = (double)l2_bytes * passes;
                break;
            }
        }
        r = cudaGetLastError();
        if (r == cudaSuccess && timed) r = cudaEventRecord(tm.e1, st);
        return r;
    };
    // one untimed launch (clocks up, L2 warm), then the timed one
    if (e == cudaSuccess) e = launch(false);
    if (e == cudaSuccess) e = launch(true);
    if (e == cudaSuccess) e = cudaEventSynchronize(tm.e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, tm.e0, tm.e1);
    int hflag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(scratch);
    cudaFree(flag);
    if (e != cudaSuccess) return cuda_fail(e, "rom_measure_peak");
    if (hflag) return ROM_E_TIMEOUT;
    // TFLOP/s for the pipes, GB/s for L2
    *value = kind == ROM_PEAK_L2 ? work / (ms * 1e-3) / 1e9 : work / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return ROM_OK;
}
