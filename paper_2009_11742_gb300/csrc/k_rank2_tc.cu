// Host side of the tensor-core rank-2 path: operator splitting into
// pre-swizzled tiles, planning (cluster size, columns per block, pipeline
// depth) and launch.
#include <cuda_runtime.h>

#include "rank2_launch.cuh"
#include "rank2_tc.cuh"
#include "rank2_tcs.cuh"

namespace romk {

// ---- operator tiles: out[((rt * NKC + kc) * NA + t) * 16 KB] = term t of
// rows 128 rt .. + 127, k = KC kc .. + KC - 1, SW128 K-major.
template <int P>
__global__ void tc_split_operator_kernel(const float* __restrict__ A, int Ksrc, int Kp,
                                         unsigned char* __restrict__ out) {
    using Sch = TcScheme<P>;
    constexpr int NA = Sch::NA, KC = Sch::KC;
    constexpr int ES = Sch::kTF32 ? 4 : 2;
    const int NKC = Kp / KC;
    const size_t total = (size_t)Kp * Kp;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(idx / Kp), col = (int)(idx % Kp);
        const float x = (row < Ksrc && col < Ksrc) ? A[(size_t)row * Ksrc + col] : 0.f;
        const int rt = row / kTcRows, r = row % kTcRows, kc = col / KC, k = col % KC;
        const uint32_t within = sw128_offset((uint32_t)r, (uint32_t)((k * ES) >> 4)) + ((k * ES) & 15);
        unsigned char* tile0 = out + ((size_t)(rt * NKC + kc) * NA) * kATileBytes + within;
        if constexpr (Sch::kTF32) {
            float hi, lo;
            split_tf32_rn(x, hi, lo);
            *reinterpret_cast<float*>(tile0) = hi;
            *reinterpret_cast<float*>(tile0 + kATileBytes) = lo;
        } else {
            float rem = x;
#pragma unroll
            for (int t = 0; t < NA; ++t) {
                const __nv_bfloat16 b = __float2bfloat16_rn(rem);
                *reinterpret_cast<__nv_bfloat16*>(tile0 + t * kATileBytes) = b;
                rem = rem - __bfloat162float(b);
            }
        }
    }
}

// ---- ROM_BF16S operator: per-row exponent (one warp per row), then the three
// integer digits of A[r][k] * 2^(7 - e_r) into the same tile layout.
__global__ void tcs_row_scale_kernel(const float* __restrict__ A, int Ksrc, int Kp, float* __restrict__ scale) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (row >= Kp) return;
    float mx = 0.f;
    if (row < Ksrc)
        for (int k = lane; k < Ksrc; k += 32) mx = fmaxf(mx, fabsf(A[(size_t)row * Ksrc + k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) scale[row] = ldexpf(1.f, bound_exponent(mx) - 7);
}

__global__ void tcs_split_operator_kernel(const float* __restrict__ A, int Ksrc, int Kp,
                                          const float* __restrict__ scale, unsigned char* __restrict__ out) {
    const int NKC = Kp / kTcsKC;
    const size_t total = (size_t)Kp * Kp;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(idx / Kp), col = (int)(idx % Kp);
        const float x = (row < Ksrc && col < Ksrc) ? A[(size_t)row * Ksrc + col] : 0.f;
        const int rt = row / kTcRows, r = row % kTcRows, kc = col / kTcsKC, k = col % kTcsKC;
        const uint32_t within = sw128_offset((uint32_t)r, (uint32_t)((k * 2) >> 4)) + ((k * 2) & 15);
        unsigned char* tile0 = out + ((size_t)(rt * NKC + kc) * kTcsTerms) * kATileBytes + within;
        float d0, d1, d2;
        slice_digits(x * (1.f / scale[row]), d0, d1, d2);
        *reinterpret_cast<__nv_bfloat16*>(tile0) = __float2bfloat16_rn(d0);
        *reinterpret_cast<__nv_bfloat16*>(tile0 + kATileBytes) = __float2bfloat16_rn(d1);
        *reinterpret_cast<__nv_bfloat16*>(tile0 + 2 * kATileBytes) = __float2bfloat16_rn(d2);
    }
}

__global__ void pad_rows_kernel(const float* __restrict__ src, int rows, int src_cols, int dst_cols,
                                float* __restrict__ dst) {
    const size_t total = (size_t)rows * dst_cols;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / dst_cols), c = (int)(idx % dst_cols);
        dst[idx] = c < src_cols ? src[(size_t)r * src_cols + c] : 0.f;
    }
}

template <int P>
static size_t tc_operator_bytes(int Kp) {
    return (size_t)Kp * Kp * TcScheme<P>::NA * (TcScheme<P>::kTF32 ? 4 : 2);
}

size_t tc_scale_offset(int prec, int Kp) {
    return prec == ROM_BF16S ? (size_t)Kp * Kp * kTcsTerms * 2 : 0;
}

size_t tc_operator_bytes_for(int prec, int Kp) {
    switch (prec) {
        case ROM_BF16S: return tc_scale_offset(prec, Kp) + (size_t)Kp * sizeof(float);
        case ROM_TF32X3: return tc_operator_bytes<ROM_TF32X3>(Kp);
        case ROM_BF16X3: return tc_operator_bytes<ROM_BF16X3>(Kp);
        case ROM_BF16: return tc_operator_bytes<ROM_BF16>(Kp);
        default: return 0;
    }
}

cudaError_t tc_prepare_operator(int prec, const float* A_rm, int Ksrc, int Kp, void* out,
                                cudaStream_t st) {
    const size_t total = (size_t)Kp * Kp;
    unsigned blocks = (unsigned)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    unsigned char* o = static_cast<unsigned char*>(out);
    if (prec == ROM_BF16S) {
        float* scale = reinterpret_cast<float*>(o + tc_scale_offset(prec, Kp));
        tcs_row_scale_kernel<<<(Kp + 7) / 8, 256, 0, st>>>(A_rm, Ksrc, Kp, scale);
        tcs_split_operator_kernel<<<blocks, 256, 0, st>>>(A_rm, Ksrc, Kp, scale, o);
        return cudaGetLastError();
    }
    switch (prec) {
        case ROM_TF32X3: tc_split_operator_kernel<ROM_TF32X3><<<blocks, 256, 0, st>>>(A_rm, Ksrc, Kp, o); break;
        case ROM_BF16X3: tc_split_operator_kernel<ROM_BF16X3><<<blocks, 256, 0, st>>>(A_rm, Ksrc, Kp, o); break;
        case ROM_BF16: tc_split_operator_kernel<ROM_BF16><<<blocks, 256, 0, st>>>(A_rm, Ksrc, Kp, o); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t tc_pad_rows(const float* src, int rows, int src_cols, int dst_cols, float* dst,
                        cudaStream_t st) {
    const size_t total = (size_t)rows * dst_cols;
    if (total == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    pad_rows_kernel<<<blocks, 256, 0, st>>>(src, rows, src_cols, dst_cols, dst);
    return cudaGetLastError();
}

template <int P>
static void* tc_kernel(int W) {
    return W == 64 ? (void*)&rank2_tc_kernel<P, 64> : (W == 128 ? (void*)&rank2_tc_kernel<P, 128> : nullptr);
}

static void* tc_kernel_for(int prec, int W) {
    switch (prec) {
        case ROM_TF32X3: return tc_kernel<ROM_TF32X3>(W);
        case ROM_BF16X3: return tc_kernel<ROM_BF16X3>(W);
        case ROM_BF16: return tc_kernel<ROM_BF16>(W);
        default: return nullptr;
    }
}

static size_t tc_smem_for(int prec, int W, int stages, int rpc, int Kp) {
    switch (prec) {
        case ROM_TF32X3: return tc_smem_bytes<ROM_TF32X3>(W, stages, rpc, Kp);
        case ROM_BF16X3: return tc_smem_bytes<ROM_BF16X3>(W, stages, rpc, Kp);
        case ROM_BF16: return tc_smem_bytes<ROM_BF16>(W, stages, rpc, Kp);
        default: return 0;
    }
}

int tc_exchange_terms(int prec) {
    switch (prec) {
        case ROM_BF16S: return kTcsTerms;
        case ROM_TF32X3: return TcScheme<ROM_TF32X3>::NX;
        case ROM_BF16X3: return TcScheme<ROM_BF16X3>::NX;
        case ROM_BF16: return TcScheme<ROM_BF16>::NX;
        default: return 0;
    }
}
int tc_element_bytes(int prec) { return prec == ROM_TF32X3 ? 4 : 2; }

// xr: the instance that adds the reduced reference state.
static void* tcs_kernel(int W, bool xr = false) {
    switch (W) {
        case 32: return xr ? (void*)&rank2_tcs_kernel<32, true> : (void*)&rank2_tcs_kernel<32, false>;
        case 48: return xr ? (void*)&rank2_tcs_kernel<48, true> : (void*)&rank2_tcs_kernel<48, false>;
        case 64: return xr ? (void*)&rank2_tcs_kernel<64, true> : (void*)&rank2_tcs_kernel<64, false>;
        case 80: return xr ? (void*)&rank2_tcs_kernel<80, true> : (void*)&rank2_tcs_kernel<80, false>;
        default: return nullptr;
    }
}

// ROM_BF16S: the block width with the least estimated time, taken as the
// number of waves of clusters times (W + a fixed per-chunk cost of about 48
// columns' worth of MMA time).
static bool plan_rank2_tcs(int Kp, int M, int R, int Wforce, TcPlan* p) {
    if (Kp <= 0 || Kp % kTcRows != 0 || Kp > 1024 || M <= 0) return false;
    const int cs = Kp / kTcRows;
    const int smax = device_smem_optin();
    const int cands[4] = {32, 48, 64, 80};
    long best = -1;
    for (int ci = 0; ci < 4; ++ci) {
        const int W = cands[ci];
        if (Wforce > 0 && W != Wforce) continue;
        void* fn = tcs_kernel(W);
        int stages = 0;
        for (int s = 4; s >= 2; --s)
            if (tcs_smem_bytes(W, s) <= (size_t)smax) { stages = s; break; }
        if (!fn || stages == 0) continue;
        const size_t smem = tcs_smem_bytes(W, stages);
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        ClusterLaunch probe(cs, 1, kTcsThreads, smem);
        const int nact = probe.max_active(fn);
        if (nact <= 0) continue;
        const int ncl = (M + W - 1) / W;
        const long waves = (ncl + nact - 1) / nact;
        const long cost = waves * (W + 48);
        if (best < 0 || cost < best) {
            best = cost;
            p->prec = ROM_BF16S;
            p->cs = cs;
            p->rpc = (R + cs - 1) / cs;
            p->W = W;
            p->stages = stages;
            p->smem = smem;
            p->nclusters = ncl;
            p->max_active_clusters = nact;
        }
    }
    return best >= 0;
}

bool plan_rank2_tc(int prec, int Kp, int M, int R, int Wforce, TcPlan* p) {
    if (prec == ROM_BF16S) return plan_rank2_tcs(Kp, M, R, Wforce, p);
    if (Kp <= 0 || Kp % kTcRows != 0 || Kp > 1024 || M <= 0) return false;
    p->cs = Kp / kTcRows;
    p->rpc = (R + p->cs - 1) / p->cs;
    const int smax = device_smem_optin();
    // columns per block: 64 or 128 (MMA N; each reader warp drains W/2 columns)
    void* fn64 = tc_kernel_for(prec, 64);
    if (!fn64) return false;
    const size_t smem64 = tc_smem_for(prec, 64, 2, p->rpc, Kp);
    if (smem64 > (size_t)smax) return false;
    if (cudaFuncSetAttribute(fn64, cudaFuncAttributeMaxDynamicSharedMemorySize, smax) != cudaSuccess ||
        cudaFuncSetAttribute(fn64, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    ClusterLaunch probe(p->cs, 1, kTcThreads, smem64);
    const int nact = probe.max_active(fn64);
    if (nact <= 0) return false;
    p->max_active_clusters = nact;
    int W = Wforce;
    if (W <= 0) W = ((M + nact - 1) / nact) <= 64 ? 64 : 128;
    if (W != 64 && W != 128) return false;
    // deepest pipeline (2..6 stages) that fits
    int stages = 0;
    for (int s = 6; s >= 2; --s) {
        if (tc_smem_for(prec, W, s, p->rpc, Kp) <= (size_t)smax) { stages = s; break; }
    }
    if (stages == 0) return false;
    p->W = W;
    p->stages = stages;
    p->smem = tc_smem_for(prec, W, stages, p->rpc, Kp);
    p->nclusters = (M + W - 1) / W;
    p->prec = prec;
    return true;
}

cudaError_t launch_rank2_tc(const TcArgs& a_in, const TcPlan& p, cudaStream_t st) {
    const bool xr = a_in.Xv != nullptr || a_in.Xs != nullptr;
    void* fn = p.prec == ROM_BF16S ? tcs_kernel(p.W, xr) : tc_kernel_for(p.prec, p.W);
    if (!fn) return cudaErrorInvalidValue;
    TcArgs a = a_in;
    a.W = p.W;
    a.stages = p.stages;
    a.rpc = p.rpc;
    size_t smem = p.smem;
    if (p.prec == ROM_BF16S && xr) {
        // room for the reference-state staging: fewer stages if needed
        const size_t smax = (size_t)device_smem_optin();
        int s = p.stages;
        while (s > 2 && tcs_smem_bytes(p.W, s) + tcs_xref_bytes(p.W) > smax) --s;
        smem = tcs_smem_bytes(p.W, s) + tcs_xref_bytes(p.W);
        if (smem > smax) return cudaErrorInvalidValue;
        a.stages = s;
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    ClusterLaunch L(p.cs, p.nclusters, p.prec == ROM_BF16S ? kTcsThreads : kTcThreads, smem, st);
    void* args[] = {(void*)&a};
    return L.launch(fn, args);
}

}  // namespace romk
