// Host planning / launch of the reverse-time adjoint kernel.
#include <cuda_runtime.h>

#include "rank2_adjoint.cuh"
#include "rank2_launch.cuh"

namespace romk {

static void* adjoint_kernel(int KI) {
#define ROM_ADJ_CASE(k) \
    case k: return (void*)&rank2_adjoint_kernel<k, 8>;
    switch (KI) {
        ROM_ADJ_CASE(1) ROM_ADJ_CASE(2) ROM_ADJ_CASE(3) ROM_ADJ_CASE(4)
        ROM_ADJ_CASE(5) ROM_ADJ_CASE(6) ROM_ADJ_CASE(7) ROM_ADJ_CASE(8)
        ROM_ADJ_CASE(9) ROM_ADJ_CASE(10) ROM_ADJ_CASE(11) ROM_ADJ_CASE(12)
        ROM_ADJ_CASE(13) ROM_ADJ_CASE(14) ROM_ADJ_CASE(15) ROM_ADJ_CASE(16)
        default: return nullptr;
    }
#undef ROM_ADJ_CASE
}

// Kp <= 512: one 32-row tile per CTA (Kp / 32 CTAs, operators in registers);
// 512 < Kp <= 1024: two tiles per CTA (Kp / 64 CTAs, operators read from L2).
bool plan_adjoint(int Kp, int M, int R, AdjPlan* p) {
    if (Kp <= 0 || Kp % 64 != 0 || Kp > 1024 || M <= 0 || R <= 0) return false;
    p->KI = Kp / 64;
    const int nrt = Kp > 512 ? 2 : 1;
    p->cs = Kp / (32 * nrt);
    p->cb = 8;
    const int smax = device_smem_optin();
    int wcap = 0;
    for (int w = 8; w <= 2048; w += 8) {
        if (adj_smem_layout(w, Kp, R, nrt).total > (size_t)smax) break;
        wcap = w;
    }
    if (wcap == 0) return false;
    void* fn = adjoint_kernel(p->KI);
    if (!fn) return false;
    const size_t smem_probe = adj_smem_layout(wcap, Kp, R, nrt).total;
    if (prepare_kernel<float>(fn, smem_probe) != cudaSuccess) return false;
    ClusterLaunch probe(p->cs, 1, kThreads, smem_probe);
    const int nact = probe.max_active(fn);
    if (nact <= 0) return false;
    int wv = (M + nact - 1) / nact;
    wv = ((wv + 7) / 8) * 8;
    if (wv > wcap) wv = wcap;
    p->Wv = wv;
    p->Wa = wv;
    p->nclusters = (M + wv - 1) / wv;
    p->smem = adj_smem_layout(p->Wa, Kp, R, nrt).total;
    return true;
}

cudaError_t launch_adjoint(const AdjArgs& a_in, const AdjPlan& p, cudaStream_t st) {
    AdjArgs a = a_in;
    a.Wv = p.Wv;
    a.Wa = p.Wa;
    void* fn = adjoint_kernel(p.KI);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = prepare_kernel<float>(fn, p.smem);
    if (e != cudaSuccess) return e;
    ClusterLaunch L(p.cs, p.nclusters, kThreads, p.smem, st);
    void* args[] = {(void*)&a};
    return L.launch(fn, args);
}

// out[m] = sum over CTAs (in rank order) of part[rank][m].
__global__ void sum_partials_kernel(const float* __restrict__ part, int cs, int M, float* __restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    float s = 0.f;
    for (int k = 0; k < cs; ++k) s += part[(size_t)k * M + m];
    out[m] = s;
}

cudaError_t launch_sum_partials(const float* part, int cs, int M, float* out, cudaStream_t st) {
    sum_partials_kernel<<<(M + 255) / 256, 256, 0, st>>>(part, cs, M, out);
    return cudaGetLastError();
}

}  // namespace romk
