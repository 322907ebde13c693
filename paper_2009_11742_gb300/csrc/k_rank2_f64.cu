// FP64 (check path) instantiations of the cluster-persistent rank-2 SIMT kernel.
#include "rank2_launch.cuh"

namespace romk {

bool plan_rank2_simt_f64(int Kp, int M, int R, bool rank1, Rank2Plan* p, int budget) {
    return plan_rank2<double>(Kp, M, R, rank1, p, budget);
}

cudaError_t launch_rank2_simt_f64(const Rank2Args& a, const Rank2Plan& p, cudaStream_t st) {
    return launch_rank2<double>(a, p, st);
}

}  // namespace romk
