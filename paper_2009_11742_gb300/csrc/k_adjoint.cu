// Host planning / launch of the reverse-time adjoint kernel.
#include <cuda_runtime.h>

#include "rank2_adjoint.cuh"
#include "rank2_launch.cuh"

namespace romk {

static void* adjoint_kernel(int KI) {
    switch (KI) {
        case 1: return (void*)&rank2_adjoint_kernel<1, 8>;
        case 2: return (void*)&rank2_adjoint_kernel<2, 8>;
        case 3: return (void*)&rank2_adjoint_kernel<3, 8>;
        case 4: return (void*)&rank2_adjoint_kernel<4, 8>;
        case 5: return (void*)&rank2_adjoint_kernel<5, 8>;
        case 6: return (void*)&rank2_adjoint_kernel<6, 8>;
        case 7: return (void*)&rank2_adjoint_kernel<7, 8>;
        case 8: return (void*)&rank2_adjoint_kernel<8, 8>;
        default: return nullptr;
    }
}

bool plan_adjoint(int Kp, int M, int R, AdjPlan* p) {
    if (Kp <= 0 || Kp % 64 != 0 || Kp > 512 || M <= 0 || R <= 0) return false;
    p->KI = Kp / 64;
    p->cs = Kp / 32;
    p->cb = 8;
    const int smax = device_smem_optin();
    int wcap = 0;
    for (int w = 8; w <= 2048; w += 8) {
        if (adj_smem_layout(w, Kp, R).total > (size_t)smax) break;
        wcap = w;
    }
    if (wcap == 0) return false;
    void* fn = adjoint_kernel(p->KI);
    if (!fn) return false;
    const size_t smem_probe = adj_smem_layout(wcap, Kp, R).total;
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
    p->smem = adj_smem_layout(p->Wa, Kp, R).total;
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
