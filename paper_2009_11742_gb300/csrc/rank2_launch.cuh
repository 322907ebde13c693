// Host-side planning and launch of the cluster-persistent SIMT rank-2 kernel.
#pragma once

#include <cuda_runtime.h>

#include <mutex>

#include "rank2_simt.cuh"

namespace romk {

// Launch configuration of a grid of `nclusters` clusters of `cs` CTAs (one
// cluster for an occupancy query).  The attribute array lives in the object,
// so it is neither copied nor moved.
struct ClusterLaunch {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1] = {};
    ClusterLaunch(int cs, int nclusters, int threads, size_t smem, cudaStream_t st = nullptr) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cs * nclusters, 1, 1);
        cfg.blockDim = dim3(threads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    ClusterLaunch(const ClusterLaunch&) = delete;
    ClusterLaunch& operator=(const ClusterLaunch&) = delete;
    // Clusters of this shape that fit on the device at once (0: none, or the
    // query failed; the error is cleared).
    int max_active(const void* fn) {
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return n;
    }
    cudaError_t launch(const void* fn, void** args) { return cudaLaunchKernelExC(&cfg, fn, args); }
};

// FP32 with operators streamed from L2 (KI > 8) in 8-column groups runs the
// 4-row, 32-lane half-step (GEN).
template <typename T, int KI, int CB, bool RES>
struct Rank2Kernel {
    static constexpr bool GEN = sizeof(T) == 4 && CB == 8 && KI > 8 && !RES;
    static void* fn() { return (void*)&rank2_simt_kernel<T, KI, CB, RES, GEN>; }
};

// Kernel entry for (KI, CB) with the residency rule of the element type:
// FP32 keeps both operators in registers up to KI = 8 (K <= 512); FP64 up to
// KI = 4 (K <= 256) and re-reads its 32-row operator slab from L2 each
// half-step beyond that.
// FP32 beyond KI = 8 (K > 512) streams two 32-row operator tiles per CTA per
// half-step (one-block kernel with nrt = 2; in 8-column groups with the 4-row
// half-step); FP64 stops at K = 512.
template <typename T, int CB>
static void* rank2_kernel_for(int KI, bool* resident) {
    constexpr bool f64 = sizeof(T) == 8;
    *resident = !(f64 && KI > 4) && KI <= 8;
    switch (KI) {
        case 1: return Rank2Kernel<T, 1, CB, true>::fn();
        case 2: return Rank2Kernel<T, 2, CB, true>::fn();
        case 3: return Rank2Kernel<T, 3, CB, true>::fn();
        case 4: return Rank2Kernel<T, 4, CB, true>::fn();
        case 5: return Rank2Kernel<T, 5, CB, !f64>::fn();
        case 6: return Rank2Kernel<T, 6, CB, !f64>::fn();
        case 7: return Rank2Kernel<T, 7, CB, !f64>::fn();
        case 8: return Rank2Kernel<T, 8, CB, !f64>::fn();
        default: break;
    }
    if constexpr (!f64) {
        switch (KI) {
            case 9: return Rank2Kernel<T, 9, CB, false>::fn();
            case 10: return Rank2Kernel<T, 10, CB, false>::fn();
            case 11: return Rank2Kernel<T, 11, CB, false>::fn();
            case 12: return Rank2Kernel<T, 12, CB, false>::fn();
            case 13: return Rank2Kernel<T, 13, CB, false>::fn();
            case 14: return Rank2Kernel<T, 14, CB, false>::fn();
            case 15: return Rank2Kernel<T, 15, CB, false>::fn();
            case 16: return Rank2Kernel<T, 16, CB, false>::fn();
            default: break;
        }
    }
    return nullptr;
}

template <typename T>
static void* rank2_kernel(int KI, int cb, bool* resident) {
    if (cb == 1) return rank2_kernel_for<T, 1>(KI, resident);
    if constexpr (sizeof(T) == 4) {
        if (cb == 8) return rank2_kernel_for<T, 8>(KI, resident);  // wide column group (FP32)
    }
    return nullptr;
}

static int device_smem_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

template <typename T>
static cudaError_t prepare_kernel(void* fn, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

// The plan for clusters of cs CTAs owning at most nrt 32-row tiles each
// (cs = 0: the kernel's own, Kp / 32 CTAs of one tile up to Kp = 512 and
// Kp / 64 of two above).  cluster_budget > 0 caps the clusters the plan
// assumes it may keep busy (the batched scheduler hands each ROM its share
// of the GPU).
template <typename T>
static bool plan_rank2_cs(int Kp, int M, int R, bool rank1, Rank2Plan* p, int cluster_budget, int cs) {
    const int kmax = sizeof(T) == 4 ? 1024 : 512;
    if (Kp <= 0 || Kp % 64 != 0 || Kp > kmax || M <= 0) return false;
    constexpr int CBW = 8;  // wide column group (FP32)
    p->KI = Kp / 64;
    if (cs == 0) {
        p->nrt = Kp > 512 ? 2 : 1;
        p->cs = Kp / (32 * p->nrt);
    } else {
        p->cs = cs;
        p->nrt = (Kp / 32 + cs - 1) / cs;
    }
    // FP64 runs one-column groups: it is bound by the SMs' few FP64 units,
    // not by the shuffles and loads a wider group saves, and a narrow group
    // lets a small ensemble spread one column per cluster.
    p->cb = (rank1 || sizeof(T) == 8) ? 1 : CBW;
    const int rpc = (R + p->cs - 1) / p->cs;
    const int smax = device_smem_optin();
    // widest allocation that fits shared memory; when the CTA's receiver rows
    // leave no room, they are read from global memory instead
    int wcap = 0;
    p->c_global = false;
    for (int pass = 0; pass < 2 && wcap == 0; ++pass) {
        p->c_global = pass == 1;
        const int rpc_s = p->c_global ? 0 : rpc;
        for (int w = p->cb; w <= 4096; w += p->cb) {
            if (rank2_smem_layout<T>(w, Kp, rpc_s, p->nrt).total > (size_t)smax) break;
            wcap = w;
        }
        if (rpc == 0) break;
    }
    if (wcap == 0) return false;
    const int rpc_smem = p->c_global ? 0 : rpc;
    void* fn = rank2_kernel<T>(p->KI, p->cb, &p->resident);
    if (!fn) return false;
    const int wprobe = rank1 ? 1 : wcap;
    const size_t smem_probe = rank2_smem_layout<T>(wprobe, Kp, rpc_smem, p->nrt).total;
    if (prepare_kernel<T>(fn, smem_probe) != cudaSuccess) return false;
    ClusterLaunch probe(p->cs, 1, kThreads, smem_probe);
    const int nact = probe.max_active(fn);
    if (nact <= 0) return false;
    p->max_active_clusters = nact;
    const int budget = cluster_budget > 0 && cluster_budget < nact ? cluster_budget : nact;
    int wv = (M + budget - 1) / budget;
    wv = ((wv + p->cb - 1) / p->cb) * p->cb;
    if (wv > wcap) wv = wcap;
    p->Wv = wv;
    p->Wa = wv;
    p->nclusters = (M + wv - 1) / wv;
    p->smem = rank2_smem_layout<T>(p->Wa, Kp, rpc_smem, p->nrt).total;
    p->variant = 1;
    return true;
}

// Wave count x step time of a plan with streamed operators (µs per step).
inline double rank2_plan_model_us(const Rank2Plan& p, int Kp) {
    const int act = p.max_active_clusters > 0 ? p.max_active_clusters : 1;
    const int waves = (p.nclusters + act - 1) / act;
    return waves * model_streamed_us(Kp, p.nrt, p.Wa);
}

// FP32 above Kp = 512 in 8-column groups (the 4-row half-step, which deals
// a job's row tiles to any cluster size) also tries clusters of 4 and 2:
// at most 7 clusters of Kp / 64 > 8 CTAs are co-resident, against 36 of 4
// and 76 of 2, and the shared memory caps the columns per cluster whatever
// its size.  The plan with the fewest modelled µs per step wins.
template <typename T>
static bool plan_rank2(int Kp, int M, int R, bool rank1, Rank2Plan* p, int cluster_budget = 0) {
    if (!plan_rank2_cs<T>(Kp, M, R, rank1, p, cluster_budget, 0)) return false;
    if (sizeof(T) != 4 || rank1 || cluster_budget > 0 || Kp <= 512 || p->cb != 8) return true;
    double best = rank2_plan_model_us(*p, Kp);
    for (int cs : {4, 2}) {
        Rank2Plan q{};
        if (!plan_rank2_cs<T>(Kp, M, R, rank1, &q, 0, cs)) continue;
        const double t = rank2_plan_model_us(q, Kp);
        if (t < best) {
            best = t;
            *p = q;
        }
    }
    return true;
}

template <typename T>
static cudaError_t launch_rank2(const Rank2Args& a_in, const Rank2Plan& p, cudaStream_t st) {
    Rank2Args a = a_in;
    a.Wv = p.Wv;
    a.Wa = p.Wa;
    a.nrt = p.nrt;
    a.rpc = (a.R + p.cs - 1) / p.cs;
    a.c_global = p.c_global ? 1 : 0;
    bool res = false;
    void* fn = rank2_kernel<T>(p.KI, p.cb, &res);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = prepare_kernel<T>(fn, p.smem);
    if (e != cudaSuccess) return e;
    ClusterLaunch L(p.cs, p.nclusters, kThreads, p.smem, st);
    void* args[] = {(void*)&a};
    return L.launch(fn, args);
}

}  // namespace romk
