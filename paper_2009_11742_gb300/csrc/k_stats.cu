// Ensemble statistics of receiver traces (mean and quantile bands over the
// realizations, Sec. 4.5.2): one CTA per (record, receiver) loads the M
// values into shared memory, reduces the mean in FP64 by a fixed pairwise
// tree, sorts them with a bitonic network and interpolates the quantiles
// between order statistics (Hyndman-Fan type 7).
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/rom.h"

namespace romk {

constexpr int kStatThreads = 256;
constexpr int kStatMaxM = 4096;
constexpr int kStatMaxP = 16;

struct StatArgs {
    const float* traces;
    double* mean_out;
    double* q_out;
    double probs[kStatMaxP];
    int nrec, R, M, Mp, nprobs;
};

__global__ void __launch_bounds__(kStatThreads) trace_stats_kernel(const StatArgs a) {
    extern __shared__ float sx[];                                   // Mp values
    double* sd = reinterpret_cast<double*>(sx + a.Mp);              // kStatThreads partial sums
    const int kj = blockIdx.x;
    const int k = kj / a.R, j = kj % a.R;
    const int tid = threadIdx.x;
    for (int i = tid; i < a.Mp; i += kStatThreads)
        sx[i] = i < a.M ? a.traces[((size_t)k * a.M + i) * a.R + j] : INFINITY;
    __syncthreads();
    if (a.mean_out) {
        // thread t sums m = t, t + 256, ... in order; then a pairwise tree over t
        double s = 0.0;
        for (int i = tid; i < a.M; i += kStatThreads) s = __dadd_rn(s, (double)sx[i]);
        sd[tid] = s;
        __syncthreads();
        for (int w = kStatThreads / 2; w > 0; w >>= 1) {
            if (tid < w) sd[tid] = __dadd_rn(sd[tid], sd[tid + w]);
            __syncthreads();
        }
        if (tid == 0) a.mean_out[(size_t)k * a.R + j] = sd[0] / (double)a.M;
    }
    if (!a.q_out) return;
    // bitonic sort, ascending (padding +inf sorts last)
    for (int size = 2; size <= a.Mp; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < a.Mp / 2; i += kStatThreads) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const float x = sx[lo], y = sx[hi];
                if ((x > y) == up) { sx[lo] = y; sx[hi] = x; }
            }
            __syncthreads();
        }
    }
    if (tid < a.nprobs) {
        // explicit round-to-nearest operations: no contraction into FMAs
        const double h = __dmul_rn((double)(a.M - 1), a.probs[tid]);
        int i = (int)floor(h);
        if (i > a.M - 1) i = a.M - 1;
        const double t = __dsub_rn(h, (double)i);
        const double lo = (double)sx[i];
        const double hi = (double)sx[i + 1 < a.M ? i + 1 : a.M - 1];
        const double d = __dsub_rn(hi, lo);
        const double q = t >= 0.5 ? __dsub_rn(hi, __dmul_rn(d, __dsub_rn(1.0, t)))
                                  : __dadd_rn(lo, __dmul_rn(d, t));
        a.q_out[((size_t)tid * a.nrec + k) * a.R + j] = q;
    }
}

static bool device_pointer(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace romk

extern "C" rom_status rom_trace_stats(const float* traces, int nrec, int R, int M, const double* probs,
                                      int nprobs, double* mean_out, double* q_out, void* stream) {
    using namespace romk;
    if (!traces || nrec < 1 || R < 1 || M < 1 || M > kStatMaxM || nprobs < 0 || nprobs > kStatMaxP)
        return ROM_E_INVAL;
    if (nprobs > 0 && (!probs || !q_out)) return ROM_E_INVAL;
    if (!device_pointer(traces) || (mean_out && !device_pointer(mean_out)) ||
        (q_out && !device_pointer(q_out)))
        return ROM_E_INVAL;
    StatArgs a{};
    for (int i = 0; i < nprobs; ++i) {
        if (!(probs[i] >= 0.0 && probs[i] <= 1.0)) return ROM_E_INVAL;
        a.probs[i] = probs[i];
    }
    if (!mean_out && nprobs == 0) return ROM_OK;
    a.traces = traces;
    a.mean_out = mean_out;
    a.q_out = nprobs > 0 ? q_out : nullptr;
    a.nrec = nrec;
    a.R = R;
    a.M = M;
    a.nprobs = nprobs;
    int Mp = 2;
    while (Mp < M) Mp <<= 1;
    a.Mp = Mp;
    const size_t smem = (size_t)Mp * sizeof(float) + kStatThreads * sizeof(double);
    const size_t nblk = (size_t)nrec * R;
    if (nblk > 0x7fffffff) return ROM_E_INVAL;
    trace_stats_kernel<<<(unsigned)nblk, kStatThreads, smem, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? ROM_OK : ROM_E_CUDA;
}
