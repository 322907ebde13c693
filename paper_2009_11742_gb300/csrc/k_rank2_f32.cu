// FP32 instantiations of the cluster-persistent rank-2 SIMT kernel.
#include "rank2_launch.cuh"

namespace romk {

bool plan_rank2_simt_f32(int Kp, int M, int R, bool rank1, Rank2Plan* p, int budget) {
    return plan_rank2<float>(Kp, M, R, rank1, p, budget);
}

cudaError_t launch_rank2_simt_f32(const Rank2Args& a, const Rank2Plan& p, cudaStream_t st) {
    return launch_rank2<float>(a, p, st);
}

// The work-list form of the one-block kernel (batched scheduler, FP32).
static void* worklist_kernel(int KI, int cb) {
    if (cb != 8) return nullptr;
#define ROM_WL_CASE(k, res) \
    case k: return (void*)&rank2_simt_worklist_kernel<k, 8, res>;
    switch (KI) {
        ROM_WL_CASE(1, true) ROM_WL_CASE(2, true) ROM_WL_CASE(3, true) ROM_WL_CASE(4, true)
        ROM_WL_CASE(5, true) ROM_WL_CASE(6, true) ROM_WL_CASE(7, true) ROM_WL_CASE(8, true)
        ROM_WL_CASE(9, false) ROM_WL_CASE(10, false) ROM_WL_CASE(11, false) ROM_WL_CASE(12, false)
        ROM_WL_CASE(13, false) ROM_WL_CASE(14, false) ROM_WL_CASE(15, false) ROM_WL_CASE(16, false)
        default: return nullptr;
    }
#undef ROM_WL_CASE
}

// Work-list plan of the one-block kernel for 512 < Kp <= 1024 (two 32-row
// tiles per CTA, operators read from L2): W columns per block (one block per
// item), ncl clusters; receiver rows staged for rpc_max per CTA, or read from
// global memory when that leaves no room; 1 KB left for static shared memory.
bool plan_worklist_simt(int Kp, int rpc_max, int W, int ncl, Rank2Plan* p) {
    if (Kp <= 512 || Kp > 1024 || Kp % 64 != 0 || W < 8 || W % 8 != 0 || ncl < 1) return false;
    const int smax = device_smem_optin() - 1024;
    p->c_global = false;
    size_t smem = rank2_smem_layout<float>(W, Kp, rpc_max, 2).total;
    if (smem > (size_t)smax) {
        p->c_global = true;
        smem = rank2_smem_layout<float>(W, Kp, 0, 2).total;
        if (smem > (size_t)smax) return false;
    }
    void* fn = worklist_kernel(Kp / 64, 8);
    if (!fn || prepare_kernel<float>(fn, smem) != cudaSuccess) return false;
    p->KI = Kp / 64;
    p->nrt = 2;
    p->cs = Kp / 64;
    p->cb = 8;
    p->Wv = p->Wa = W;
    p->nclusters = ncl;
    p->smem = smem;
    p->resident = false;
    p->variant = 1;
    ClusterLaunch probe(p->cs, 1, kThreads, smem);
    p->max_active_clusters = probe.max_active(fn);
    return p->max_active_clusters > 0;
}

// a.rpc: the largest receiver rows per CTA over the work list's jobs (the
// shared-memory layout is sized by it); a.items / nitems / item_counter set.
cudaError_t launch_rank2_simt_worklist_f32(const Rank2Args& a_in, const Rank2Plan& p, cudaStream_t st) {
    Rank2Args a = a_in;
    a.Wv = p.Wv;
    a.Wa = p.Wa;
    a.nrt = p.nrt;
    a.c_global = p.c_global ? 1 : 0;
    void* fn = worklist_kernel(p.KI, p.cb);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = prepare_kernel<float>(fn, p.smem);
    if (e != cudaSuccess) return e;
    ClusterLaunch L(p.cs, p.nclusters, kThreads, p.smem, st);
    void* args[] = {(void*)&a};
    return L.launch(fn, args);
}

}  // namespace romk
