// Host planning / launch of the reverse-time adjoint kernel.
#include <cuda_runtime.h>

#include "rank2_adjoint.cuh"
#include "rank2_launch.cuh"

namespace romk {

static void* adjoint_kernel_f32(int KI) {
#define ROM_ADJ_CASE(k) \
    case k: return (void*)&rank2_adjoint_kernel<float, k, 8>;
    switch (KI) {
        ROM_ADJ_CASE(1) ROM_ADJ_CASE(2) ROM_ADJ_CASE(3) ROM_ADJ_CASE(4)
        ROM_ADJ_CASE(5) ROM_ADJ_CASE(6) ROM_ADJ_CASE(7) ROM_ADJ_CASE(8)
        ROM_ADJ_CASE(9) ROM_ADJ_CASE(10) ROM_ADJ_CASE(11) ROM_ADJ_CASE(12)
        ROM_ADJ_CASE(13) ROM_ADJ_CASE(14) ROM_ADJ_CASE(15) ROM_ADJ_CASE(16)
        default: return nullptr;
    }
#undef ROM_ADJ_CASE
}

// FP64: 4 columns a pass (the register budget of the double operator rows).
static void* adjoint_kernel_f64(int KI) {
#define ROM_ADJ_CASE(k) \
    case k: return (void*)&rank2_adjoint_kernel<double, k, 4>;
    switch (KI) {
        ROM_ADJ_CASE(1) ROM_ADJ_CASE(2) ROM_ADJ_CASE(3) ROM_ADJ_CASE(4)
        ROM_ADJ_CASE(5) ROM_ADJ_CASE(6) ROM_ADJ_CASE(7) ROM_ADJ_CASE(8)
        default: return nullptr;
    }
#undef ROM_ADJ_CASE
}

// The split-role reverse kernel (FP32, Kp <= 512).
static void* adjoint_split_kernel(int KI) {
#define ROM_ADJ_CASE(k) \
    case k: return (void*)&rank2_adjoint_split_kernel<k>;
    switch (KI) {
        ROM_ADJ_CASE(1) ROM_ADJ_CASE(2) ROM_ADJ_CASE(3) ROM_ADJ_CASE(4)
        ROM_ADJ_CASE(5) ROM_ADJ_CASE(6) ROM_ADJ_CASE(7) ROM_ADJ_CASE(8)
        default: return nullptr;
    }
#undef ROM_ADJ_CASE
}

static void* adjoint_kernel(const AdjPlan& p) {
    if (p.split) return adjoint_split_kernel(p.KI);
    return p.f64 ? adjoint_kernel_f64(p.KI) : adjoint_kernel_f32(p.KI);
}

static size_t adjoint_smem(bool f64, int W, int Kp, int R, int nrt) {
    return f64 ? adj_smem_layout<double>(W, Kp, R, nrt).total : adj_smem_layout<float>(W, Kp, R, nrt).total;
}

// The plan for clusters of cs CTAs (cs = 0: Kp / 32 CTAs of one tile up to
// Kp = 512, Kp / 64 of two above).  Widths are multiples of 8.
static bool plan_adjoint_cs(int Kp, int M, int R, AdjPlan* p, bool f64, int cs) {
    p->f64 = f64;
    p->split = false;
    p->KI = Kp / 64;
    if (cs == 0) {
        p->nrt = Kp > 512 ? 2 : 1;
        p->cs = Kp / (32 * p->nrt);
    } else {
        p->cs = cs;
        p->nrt = (Kp / 32 + cs - 1) / cs;
    }
    p->cb = f64 ? 4 : 8;
    const int smax = device_smem_optin();
    int wcap = 0;
    for (int w = 8; w <= 2048; w += 8) {
        if (adjoint_smem(f64, w, Kp, R, p->nrt) > (size_t)smax) break;
        wcap = w;
    }
    if (wcap == 0) return false;
    void* fn = adjoint_kernel(*p);
    if (!fn) return false;
    const size_t smem_probe = adjoint_smem(f64, wcap, Kp, R, p->nrt);
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
    p->smem = adjoint_smem(f64, p->Wa, Kp, R, p->nrt);
    // waves x step-time model, to compare cluster sizes
    const int waves = (p->nclusters + nact - 1) / nact;
    p->model_us = waves * model_streamed_us(Kp, p->nrt, p->Wa);
    return true;
}

// The split-role plan (FP32, Kp <= 512): Kp / 32 CTAs, Wv columns per block
// (a multiple of 4), two blocks per cluster, spread over the co-resident
// clusters.
static bool plan_adjoint_split(int Kp, int M, int R, AdjPlan* p) {
    p->f64 = false;
    p->split = true;
    p->KI = Kp / 64;
    p->cs = Kp / 32;
    p->nrt = 1;
    p->cb = kSplitCB;
    const int smax = device_smem_optin();
    int wcap = 0;
    for (int w = kSplitCB; w <= 2048; w += kSplitCB) {
        if (adj_split_smem_layout(w, Kp, R).total > (size_t)smax) break;
        wcap = w;
    }
    if (wcap == 0) return false;
    void* fn = adjoint_split_kernel(p->KI);
    if (!fn) return false;
    const size_t smem_probe = adj_split_smem_layout(wcap, Kp, R).total;
    if (prepare_kernel<float>(fn, smem_probe) != cudaSuccess) return false;
    ClusterLaunch probe(p->cs, 1, kThreads, smem_probe);
    const int nact = probe.max_active(fn);
    if (nact <= 0) return false;
    int wv = (M + 2 * nact - 1) / (2 * nact);
    wv = ((wv + kSplitCB - 1) / kSplitCB) * kSplitCB;
    if (wv > wcap) wv = wcap;
    p->Wv = wv;
    p->Wa = wv;
    p->nclusters = ((M + wv - 1) / wv + 1) / 2;
    p->smem = adj_split_smem_layout(wv, Kp, R).total;
    p->model_us = 0.0;
    return true;
}

// FP32, Kp <= 512: the split-role kernel (both roles busy in every phase),
// else one 32-row tile per CTA (Kp / 32 CTAs, operators in registers).
// FP32 above: the operators are read from L2 and the row tiles dealt out to
// any cluster size, so Kp / 64 CTAs (7 co-resident), 4 (36) and 2 (76) are
// priced with the step-time model and the fastest kept.  FP64: Kp <= 512,
// one tile per CTA.
bool plan_adjoint(int Kp, int M, int R, AdjPlan* p, bool f64) {
    if (Kp <= 0 || Kp % 64 != 0 || Kp > (f64 ? 512 : 1024) || M <= 0 || R <= 0) return false;
    if (!f64 && Kp <= 512 && plan_adjoint_split(Kp, M, R, p)) return true;
    if (!plan_adjoint_cs(Kp, M, R, p, f64, 0)) return false;
    if (f64 || Kp <= 512) return true;
    for (int cs : {4, 2}) {
        AdjPlan q{};
        if (plan_adjoint_cs(Kp, M, R, &q, f64, cs) && q.model_us < p->model_us) *p = q;
    }
    return true;
}

template <typename T>
static cudaError_t launch_adjoint_t(const AdjArgsT<T>& a_in, const AdjPlan& p, cudaStream_t st) {
    if (p.f64 != (sizeof(T) == 8)) return cudaErrorInvalidValue;
    AdjArgsT<T> a = a_in;
    a.Wv = p.Wv;
    a.Wa = p.Wa;
    a.nrt = p.nrt;
    void* fn = adjoint_kernel(p);
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = prepare_kernel<float>(fn, p.smem);
    if (e != cudaSuccess) return e;
    ClusterLaunch L(p.cs, p.nclusters, kThreads, p.smem, st);
    void* args[] = {(void*)&a};
    return L.launch(fn, args);
}

cudaError_t launch_adjoint(const AdjArgsT<float>& a, const AdjPlan& p, cudaStream_t st) {
    return launch_adjoint_t<float>(a, p, st);
}
cudaError_t launch_adjoint(const AdjArgsT<double>& a, const AdjPlan& p, cudaStream_t st) {
    return launch_adjoint_t<double>(a, p, st);
}

// The reverse step's source term for a range of steps (Sec. 3.1: the
// misfit's derivative enters the adjoint of V through C^T):
//   src[q][k] = sum_jr C[jr][k] (traces[n + 1 - rec_base][m][jr] - ystar[n][m][jr]),
// q = s M + m, n = n_lo + s.  It does not depend on the adjoint state, so the
// reverse kernels read it instead of forming it on their critical path.
// Four chains over jr = 4 u + e, summed as (c0 + c1) + (c2 + c3).  It is a
// (ns M) x Kp x R product, tiled as one: a block takes 64 rows q x 64
// columns k, stages J receivers at a time of the residual rows and of C
// (k-major) in shared memory, and thread (tq, tk) = (t / 16, t % 16)
// accumulates rows 4 tq + i and columns tk + 16 j (i, j < 4), so that one
// read of four receivers of each operand feeds 16 multiply-adds.  FP32: J =
// 64 and a row stride of 17 16-byte groups (odd), so that the C reads of a
// quarter warp fall in distinct banks; FP64: J = 32 (static shared memory).
constexpr int kSrcT = 64;  // rows q and columns k per block
template <typename T>
struct AdjSrcTile {
    static constexpr int J = sizeof(T) == 4 ? 64 : 32;  // receivers per chunk
    static constexpr int S = J + 4;                     // row stride (elements)
};

template <typename T>
__global__ void __launch_bounds__(256) adj_source_kernel(const T* __restrict__ C_rm, const T* __restrict__ traces,
                                                         const T* __restrict__ ystar, int n_lo, int ns,
                                                         int rec_base, int M, int R, int Kp, T* __restrict__ src) {
    constexpr int J = AdjSrcTile<T>::J, ST = AdjSrcTile<T>::S;
    __shared__ __align__(16) T Rs[kSrcT * ST];  // [q][jr] residual rows
    __shared__ __align__(16) T Cs[kSrcT * ST];  // [k][jr] C columns
    const int Q = ns * M;
    const int q0 = blockIdx.x * kSrcT, k0 = blockIdx.y * kSrcT;
    const int t = threadIdx.x, tq = t / 16, tk = t % 16;
    T acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = T(0);
    for (int j0 = 0; j0 < R; j0 += J) {
        __syncthreads();  // the previous chunk's reads are done
        for (int idx = t; idx < kSrcT * J; idx += blockDim.x) {
            const int r = idx / J, jj = idx % J, jr = j0 + jj, q = q0 + r;
            T v = T(0);
            if (q < Q && jr < R) {
                const int sq = q / M, m = q - sq * M, n = n_lo + sq;
                v = traces[((size_t)(n + 1 - rec_base) * M + m) * R + jr] - ystar[((size_t)n * M + m) * R + jr];
            }
            Rs[r * ST + jj] = v;
        }
        for (int idx = t; idx < J * kSrcT; idx += blockDim.x) {
            const int jj = idx / kSrcT, kk = idx % kSrcT, jr = j0 + jj;
            Cs[kk * ST + jj] = jr < R ? C_rm[(size_t)jr * Kp + k0 + kk] : T(0);
        }
        __syncthreads();
        const int nu = min(J, R - j0 + 3) / 4;  // receiver quads of the chunk below R
        for (int u = 0; u < nu; ++u) {
            T rv[4][4], cv[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) load4(Rs + (4 * tq + i) * ST + 4 * u, rv[i]);
#pragma unroll
            for (int j = 0; j < 4; ++j) load4(Cs + (tk + 16 * j) * ST + 4 * u, cv[j]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[i][j][e] = fmadd(cv[j][e], rv[i][e], acc[i][j][e]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int q = q0 + 4 * tq + i;
        if (q < Q) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                src[(size_t)q * Kp + k0 + tk + 16 * j] =
                    (acc[i][j][0] + acc[i][j][1]) + (acc[i][j][2] + acc[i][j][3]);
        }
    }
}

template <typename T>
static cudaError_t launch_adj_source_t(const T* C_rm, const T* traces, const T* ystar, int n_lo, int ns,
                                       int rec_base, int M, int R, int Kp, T* src, cudaStream_t st) {
    if (ns < 1 || M < 1 || R < 1 || Kp < kSrcT || Kp % kSrcT != 0) return cudaErrorInvalidValue;
    const long long Q = (long long)ns * M;
    const dim3 grid((unsigned)((Q + kSrcT - 1) / kSrcT), Kp / kSrcT);
    adj_source_kernel<T><<<grid, 256, 0, st>>>(C_rm, traces, ystar, n_lo, ns, rec_base, M, R, Kp, src);
    return cudaGetLastError();
}
cudaError_t launch_adj_source(const float* C_rm, const float* traces, const float* ystar, int n_lo, int ns,
                              int rec_base, int M, int R, int Kp, float* src, cudaStream_t st) {
    return launch_adj_source_t<float>(C_rm, traces, ystar, n_lo, ns, rec_base, M, R, Kp, src, st);
}
cudaError_t launch_adj_source(const double* C_rm, const double* traces, const double* ystar, int n_lo, int ns,
                              int rec_base, int M, int R, int Kp, double* src, cudaStream_t st) {
    return launch_adj_source_t<double>(C_rm, traces, ystar, n_lo, ns, rec_base, M, R, Kp, src, st);
}

// out[m] = sum over CTAs (in rank order) of part[rank][m].
template <typename T>
__global__ void sum_partials_kernel(const T* __restrict__ part, int cs, int M, T* __restrict__ out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    T s = T(0);
    for (int k = 0; k < cs; ++k) s += part[(size_t)k * M + m];
    out[m] = s;
}

cudaError_t launch_sum_partials(const float* part, int cs, int M, float* out, cudaStream_t st) {
    sum_partials_kernel<float><<<(M + 255) / 256, 256, 0, st>>>(part, cs, M, out);
    return cudaGetLastError();
}
cudaError_t launch_sum_partials(const double* part, int cs, int M, double* out, cudaStream_t st) {
    sum_partials_kernel<double><<<(M + 255) / 256, 256, 0, st>>>(part, cs, M, out);
    return cudaGetLastError();
}

}  // namespace romk
