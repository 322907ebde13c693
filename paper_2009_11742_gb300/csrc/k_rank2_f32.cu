// FP32 instantiations of the cluster-persistent rank-2 SIMT kernel.
#include "rank2_launch.cuh"

namespace romk {

bool plan_rank2_simt_f32(int Kp, int M, int R, bool rank1, Rank2Plan* p, int budget) {
    return plan_rank2<float>(Kp, M, R, rank1, p, budget);
}

cudaError_t launch_rank2_simt_f32(const Rank2Args& a, const Rank2Plan& p, cudaStream_t st) {
    return launch_rank2<float>(a, p, st);
}

// The work-list kernel: one instance for every Kp <= 1024 (16 k groups).
static void* worklist_fn() { return (void*)&rank2_wl_kernel<16, 8>; }

size_t worklist_smem(int W, int Kp, int rpc, int nrt) {
    return rank2_smem_layout<float>(W, Kp, rpc, nrt).total;
}

// 1 KB is left for the kernel's static shared memory.
int worklist_max_clusters(int cs, size_t smem) {
    if (cs < 1 || cs > 16 || smem + 1024 > (size_t)device_smem_optin()) return 0;
    void* fn = worklist_fn();
    if (prepare_kernel<float>(fn, smem) != cudaSuccess) return 0;
    ClusterLaunch probe(cs, 1, kThreads, smem);
    return probe.max_active(fn);
}

cudaError_t launch_rank2_worklist_f32(const Rank2Args& a, int cs, int ncl, size_t smem, cudaStream_t st) {
    if (!a.group || !a.items || !a.item_counter || cs < 1 || cs > 16 || ncl < 1) return cudaErrorInvalidValue;
    void* fn = worklist_fn();
    cudaError_t e = prepare_kernel<float>(fn, smem);
    if (e != cudaSuccess) return e;
    ClusterLaunch L(cs, ncl, kThreads, smem, st);
    void* args[] = {(void*)&a};
    return L.launch(fn, args);
}

}  // namespace romk
