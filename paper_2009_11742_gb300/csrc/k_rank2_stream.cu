// Host planning / launch of the streaming companion kernel (rank2_stream.cuh)
// that runs beside the two-block split kernel on the SMs its clusters leave
// idle.
#include <cuda_runtime.h>
#include <math.h>

#include "rank2_launch.cuh"
#include "rank2_split.cuh"
#include "rank2_stream.cuh"

namespace romk {

// Instances for clusters of 2 and 4 CTAs, Kp = 64 .. 512 (the owned rows
// Kp / csz are whole 16-row groups; the last 64-row pass may be partial).
static void* stream_kernel(int KI, int csz) {
#define ROM_STR_CASE(k)                                                          \
    case k: return csz == 2 ? (void*)&rank2_stream_kernel<k, 2> : (void*)&rank2_stream_kernel<k, 4>;
    if (csz != 2 && csz != 4) return nullptr;
    switch (KI) {
        ROM_STR_CASE(1) ROM_STR_CASE(2) ROM_STR_CASE(3) ROM_STR_CASE(4)
        ROM_STR_CASE(5) ROM_STR_CASE(6) ROM_STR_CASE(7) ROM_STR_CASE(8)
        default: return nullptr;
    }
#undef ROM_STR_CASE
}

bool stream_supported(int Kp, int csz) {
    return Kp > 0 && Kp % 64 == 0 && Kp <= 512 && (csz == 2 || csz == 4) &&
           (Kp / csz) % 16 == 0 && stream_smem_layout(Kp, csz).total <= (size_t)device_smem_optin();
}

int stream_max_columns_per_cluster() { return kStrCols; }

cudaError_t launch_rank2_stream_f32(const Rank2Args& a_in, int csz, int cols_per_cluster, int nclusters,
                                    cudaStream_t st) {
    if (!stream_supported(a_in.Kp, csz) || cols_per_cluster < 1 || cols_per_cluster > kStrCols ||
        nclusters < 1)
        return cudaErrorInvalidValue;
    Rank2Args a = a_in;
    a.Wv = cols_per_cluster;
    a.Wa = cols_per_cluster;
    void* fn = stream_kernel(a.Kp / 64, csz);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = stream_smem_layout(a.Kp, csz).total;
    cudaError_t e = prepare_kernel<float>(fn, smem);
    if (e != cudaSuccess) return e;
    ClusterLaunch L(csz, nclusters, kStrThreads, smem, st);
    void* args[] = {(void*)&a};
    return L.launch(fn, args);
}

// Step-time model, microseconds per leapfrog step, fitted on GB300 at
// Kp = 512: the split kernel takes 2.24 + 0.466 W (Kp / 512) for W columns
// per block; the companion streams 2 (Kp / csz) Kp 4 bytes per CTA per step
// from L2 at about 71 GB/s per SM and spends about 3 us per step on its two
// cluster barriers, the row exchange and the epilogues (measured: 10.0 us
// with clusters of 4, 17.1 us with clusters of 2).
static double model_main_us(int Kp, int W) { return model_split_us(Kp, W); }
static double model_comp_us(int Kp, int csz) {
    return 2.0 * (Kp / (double)csz) * Kp * 4.0 / 71e3 + 3.0;
}

// Companion placement: the columns [M - comp_cols, M) go to comp_n clusters
// of comp_cs CTAs (comp_W columns each).  The main kernel keeps its
// saturated cluster count with narrower blocks.  Returns true and fills the
// comp_* fields of `p` when the model predicts a gain of at least 5 %.
bool plan_rank2_companion(int Kp, int M, int R, Rank2Plan* p) {
    Rank2Plan base;
    if (!plan_rank2_split_f32(Kp, M, R, &base)) return false;
    if (base.nclusters < base.max_active_clusters) return false;  // not saturated
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int idle = nsm - base.cs * base.nclusters;
    const double t_base = model_main_us(Kp, base.Wa);
    double best = 0.95 * t_base;
    bool found = false;
    for (int csz : {2, 4}) {
        if (!stream_supported(Kp, csz)) continue;
        // leave a fifth of the idle SMs free: not every idle SM may take a cluster
        const int cmax = (idle * 4 / 5) / csz;
        for (int w = base.Wa - kSplitCB; w >= kSplitCB; w -= kSplitCB) {
            const int main_cols = 2 * base.nclusters * w;
            const int comp_cols = M - main_cols;
            if (comp_cols <= 0) continue;
            const int comp_n = (comp_cols + kStrCols - 1) / kStrCols;
            if (comp_n > cmax) break;
            const double t = fmax(model_main_us(Kp, w), model_comp_us(Kp, csz));
            if (t < best) {
                best = t;
                found = true;
                *p = base;
                p->Wv = p->Wa = w;
                p->comp_cs = csz;
                p->comp_n = comp_n;
                p->comp_W = (comp_cols + comp_n - 1) / comp_n;
                p->comp_cols = comp_cols;
            }
        }
    }
    return found;
}

// The main plan and companion split for a caller-pinned companion: `cols`
// columns (at most M) to clusters of `csz` CTAs, the rest to the split kernel.
bool plan_rank2_companion_pinned(int Kp, int M, int R, int csz, int cols, Rank2Plan* p) {
    if (!stream_supported(Kp, csz) || cols < 1 || cols > M) return false;
    Rank2Plan main_plan{};
    if (cols < M) {
        if (!plan_rank2_split_f32(Kp, M - cols, R, &main_plan)) return false;
    } else {
        main_plan.variant = 2;
        main_plan.cs = Kp / 32;
        main_plan.nclusters = 0;  // the companion alone
    }
    *p = main_plan;
    p->comp_cs = csz;
    p->comp_n = (cols + kStrCols - 1) / kStrCols;
    p->comp_W = (cols + p->comp_n - 1) / p->comp_n;
    p->comp_cols = cols;
    return true;
}

}  // namespace romk
