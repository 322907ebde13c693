// Host planning / launch of the two-block split-role FP32 rank-2 kernels:
// variant 2 (one cluster barrier per phase) and variant 3 (dataflow).
#include <cuda_runtime.h>

#include "rank2_dataflow.cuh"
#include "rank2_launch.cuh"
#include "rank2_split.cuh"

namespace romk {

// mode: the split kernel instance (0 plain, 1 with the reduced reference
// state, 2 rank-3 grouped); the dataflow kernel tests for the reference
// state at run time and has no grouped form.
template <bool DF>
static void* two_block_kernel(int KI, int mode = 0) {
#define ROM_TB_CASE(k)                                                              \
    case k:                                                                         \
        return DF ? (void*)&rank2_dataflow_kernel<k>                                \
                  : (mode == 2   ? (void*)&rank2_split_kernel<k, 2>                 \
                     : mode == 1 ? (void*)&rank2_split_kernel<k, 1>                 \
                                 : (void*)&rank2_split_kernel<k, 0>);
    switch (KI) {
        ROM_TB_CASE(1) ROM_TB_CASE(2) ROM_TB_CASE(3) ROM_TB_CASE(4)
        ROM_TB_CASE(5) ROM_TB_CASE(6) ROM_TB_CASE(7) ROM_TB_CASE(8)
        default: return nullptr;
    }
#undef ROM_TB_CASE
}

template <bool DF>
static size_t two_block_smem(int Wa, int Kp, int rpc) {
    return DF ? dataflow_smem_layout(Wa, Kp, rpc).total : split_smem_layout(Wa, Kp, rpc).total;
}

template <bool DF>
static bool plan_two_block(int Kp, int M, int R, Rank2Plan* p, int cluster_budget = 0) {
    if (Kp <= 0 || Kp % 64 != 0 || Kp > 512 || M <= 0) return false;
    p->KI = Kp / 64;
    p->cs = Kp / 32;  // H = Kp / 64 CTAs per role
    p->cb = kSplitCB;
    p->resident = true;
    p->variant = DF ? 3 : 2;
    const int H = p->cs / 2;
    const int rpc = (R + H - 1) / H;
    const int smax = device_smem_optin();
    int wcap = 0;
    for (int w = kSplitCB; w <= 2048; w += kSplitCB) {
        if (two_block_smem<DF>(w, Kp, rpc) > (size_t)smax) break;
        wcap = w;
    }
    if (wcap == 0) return false;
    void* fn = two_block_kernel<DF>(p->KI);
    if (!fn) return false;
    const size_t smem_probe = two_block_smem<DF>(wcap, Kp, rpc);
    if (prepare_kernel<float>(fn, smem_probe) != cudaSuccess) return false;
    ClusterLaunch probe(p->cs, 1, kThreads, smem_probe);
    const int nact = probe.max_active(fn);
    if (nact <= 0) return false;
    p->max_active_clusters = nact;
    const int budget = cluster_budget > 0 && cluster_budget < nact ? cluster_budget : nact;
    p->nrt = 1;
    int wv = (M + 2 * budget - 1) / (2 * budget);
    wv = ((wv + kSplitCB - 1) / kSplitCB) * kSplitCB;
    if (wv > wcap) wv = wcap;
    p->Wv = wv;
    p->Wa = wv;
    const int nblocks = (M + wv - 1) / wv;
    p->nclusters = (nblocks + 1) / 2;
    p->smem = two_block_smem<DF>(p->Wa, Kp, rpc);
    return true;
}

template <bool DF>
static cudaError_t launch_two_block(const Rank2Args& a_in, const Rank2Plan& p, cudaStream_t st) {
    Rank2Args a = a_in;
    a.Wv = p.Wv;
    a.Wa = p.Wa;
    const int H = p.cs / 2;
    a.rpc = (a.R + H - 1) / H;
    if (DF && a.group) return cudaErrorInvalidValue;
    const int mode = a.group ? 2 : (a.Xv != nullptr || a.Xs != nullptr ? 1 : 0);
    if (a.group && (a.Xv || a.Xs)) return cudaErrorInvalidValue;
    void* fn = two_block_kernel<DF>(p.KI, mode);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = prepare_kernel<float>(fn, p.smem);
    if (e != cudaSuccess) return e;
    ClusterLaunch L(p.cs, p.nclusters, kThreads, p.smem, st);
    void* args[] = {(void*)&a};
    return L.launch(fn, args);
}

bool plan_rank2_split_f32(int Kp, int M, int R, Rank2Plan* p, int budget) { return plan_two_block<false>(Kp, M, R, p, budget); }

bool plan_rank2_dataflow_f32(int Kp, int M, int R, Rank2Plan* p) { return plan_two_block<true>(Kp, M, R, p); }
cudaError_t launch_rank2_split_f32(const Rank2Args& a, const Rank2Plan& p, cudaStream_t st) {
    return p.variant == 3 ? launch_two_block<true>(a, p, st) : launch_two_block<false>(a, p, st);
}

}  // namespace romk
