// Streaming companion kernel of the two-block FP32 split kernel.
//
// The split kernel (rank2_split.cuh) keeps both K x K operators in the
// registers of a 2K/32-CTA cluster (16 CTAs at K = 512).  Clusters that large
// fit only where a GPU processing cluster has that many free SMs, so some SMs
// stay idle.  This kernel runs beside it on those SMs and advances a few of
// the M realizations (columns are independent, Sec. 2.4) with the same
// velocity-first leapfrog (Sec. 3.1):
//
//   V += dt (Avs S + g f_n^T),   S += dt Asv V   (the new V).
//
// A cluster of CSZ (2 or 4) CTAs owns up to 4 columns (one column group);
// CTA c owns rows [c Kp / CSZ, (c + 1) Kp / CSZ) of V and of S and keeps the
// full V and S of its columns in shared memory.  The operators do not fit on
// so few SMs, so every half-step streams the CTA's rows of Avs (or Asv) from
// L2 in stages of 64 rows x 64 k: each thread loads its 4 rows x 4 k of a
// stage straight into a ring of registers that holds a whole 64-row pass
// (Kp / 64 stages), refilling each slot with the next pass's stage as soon as
// it is used, so a pass worth of loads is always in flight, across
// half-steps too (the operator does not depend on the state).  The
// arithmetic is the split kernel's, in the same order: thread (row quad q,
// k lane j) accumulates 4 rows x 4 columns over k = 64 i + 4 j + t with k
// ascending, and the same 16-lane butterfly reduce-scatter and fused
// epilogue (forcing g f^T, Kahan-compensated FP32 update) follow; receiver
// traces y = C V (Sec. 4.5.2) use the split kernel's receiver slabs and warp
// tiles.  So every column comes out bit for bit as the split kernel
// computes it.  After a half-step each CTA copies its new rows into its
// peers' copies (distributed shared memory) and one cluster barrier
// publishes them.  The kernel waits on nothing but those barriers.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "rank2_simt.cuh"
#include "rank2_split.cuh"
#include "rom_internal.h"

namespace romk {

constexpr int kStrThreads = kThreads;             // 256: thread (row quad q, k lane j)
constexpr int kStrRows = kSplitRows;              // 64 rows per pass (16 row quads)
constexpr int kStrKC = 64;                        // k extent of one stage
constexpr int kStrCols = kSplitCB;                // 4 columns per cluster (one column group)

struct StreamSmem {
    size_t Vf, Sf, cV, cS, f, Tpre, g, flags, total;
};

// Shared-memory layout for Kp padded rows and a CSZ-CTA cluster.
__host__ __device__ inline StreamSmem stream_smem_layout(int Kp, int csz) {
    StreamSmem s{};
    const size_t nr = (size_t)Kp / csz;
    size_t o = 0;
    s.Vf = o;    o += align16((size_t)kStrCols * Kp * sizeof(float));
    s.Sf = o;    o += align16((size_t)kStrCols * Kp * sizeof(float));
    s.cV = o;    o += align16((size_t)kStrCols * nr * sizeof(float));
    s.cS = o;    o += align16((size_t)kStrCols * nr * sizeof(float));
    s.f = o;     o += align16((size_t)kStrCols * sizeof(float));
    s.Tpre = o;  o += align16((size_t)kStrCols * 2 * sizeof(double));
    s.g = o;     o += align16(nr * sizeof(float));
    s.flags = o; o += 16;
    s.total = o;
    return s;
}

// KI = Kp / 64 (Kp <= 512); CSZ CTAs per cluster; Kp / CSZ a multiple of 16
// (a last pass of fewer than 64 rows leaves the row quads beyond the CTA's
// rows idle: they load nothing and write nothing).
template <int KI, int CSZ>
__global__ void __launch_bounds__(kStrThreads, 1) rank2_stream_kernel(const Rank2Args a) {
    constexpr int Kp = 64 * KI;
    constexpr int NR = Kp / CSZ;               // rows owned per CTA
    constexpr int NP = (NR + kStrRows - 1) / kStrRows;  // 64-row passes per half-step
    constexpr int NKS = Kp / kStrKC;           // k stages per pass (= KI)
    static_assert(NR % 16 == 0, "owned rows must be whole 16-row groups");
    constexpr int CB = kStrCols;
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    const int clu = blockIdx.x / CSZ;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int j = lane & 15;
    const int q = warp * 2 + (lane >> 4);      // row quad within a pass
    const int r0 = crank * NR;
    const int col0 = a.col_base + clu * a.Wv;
    const int ncol = min(a.Wv, a.M - clu * a.Wv);
    const float dt = (float)a.dt;

    extern __shared__ __align__(16) unsigned char smem[];
    const StreamSmem L = stream_smem_layout(Kp, CSZ);
    float* Vf = reinterpret_cast<float*>(smem + L.Vf);       // [4][Kp] full V of the columns
    float* Sf = reinterpret_cast<float*>(smem + L.Sf);       // [4][Kp] full S
    float* cV = reinterpret_cast<float*>(smem + L.cV);       // [4][NR] Kahan carries, own rows
    float* cS = reinterpret_cast<float*>(smem + L.cS);
    float* fcol = reinterpret_cast<float*>(smem + L.f);      // [4] forcing of the current step
    double* Tpre = reinterpret_cast<double*>(smem + L.Tpre); // [4][-1.5 T, pi / T]
    float* gown = reinterpret_cast<float*>(smem + L.g);      // [NR] source rows

    const float* Vin = static_cast<const float*>(a.V);
    const float* Sin = static_cast<const float*>(a.S);
    const float* cVin = static_cast<const float*>(a.compV);
    const float* cSin = static_cast<const float*>(a.compS);
    for (int idx = tid; idx < kStrCols * Kp; idx += kStrThreads) {
        const int c = idx / Kp, k = idx % Kp;
        const bool okc = c < ncol;
        Vf[idx] = (okc && k < a.Kv) ? Vin[(size_t)(col0 + c) * a.Kv + k] : 0.f;
        Sf[idx] = (okc && k < a.Ks) ? Sin[(size_t)(col0 + c) * a.Ks + k] : 0.f;
    }
    for (int idx = tid; idx < kStrCols * NR; idx += kStrThreads) {
        const int c = idx / NR, rl = idx % NR, row = r0 + rl;
        const bool okc = c < ncol;
        cV[idx] = (okc && cVin && row < a.Kv) ? cVin[(size_t)(col0 + c) * a.Kv + row] : 0.f;
        cS[idx] = (okc && cSin && row < a.Ks) ? cSin[(size_t)(col0 + c) * a.Ks + row] : 0.f;
    }
    for (int rl = tid; rl < NR; rl += kStrThreads) gown[rl] = static_cast<const float*>(a.g_p)[r0 + rl];
    if (tid < kStrCols) {
        const float T = (a.Tper && tid < ncol) ? static_cast<const float*>(a.Tper)[col0 + tid] : 1.f;
        Tpre[2 * tid] = -1.5 * (double)T;
        Tpre[2 * tid + 1] = 3.14159265358979323846 / (double)T;
        float f = 0.f;
        if (tid < ncol) {
            if (a.ftab) f = static_cast<const float*>(a.ftab)[col0 + tid];
            else if (a.Tper) f = wavelet_eval_pre(a.wavelet, (long long)a.n0, a.dt, Tpre[2 * tid], Tpre[2 * tid + 1]);
        }
        fcol[tid] = f;
    }
    __syncthreads();
    // every CTA is initialised before any peer copies rows into it
    cluster.sync();

    const int N = a.nsteps;
    const float* Avs = static_cast<const float*>(a.Avs_rm);
    const float* Asv = static_cast<const float*>(a.Asv_rm);
    // Stage (half h, pass p, k stage ks): this thread's part is rows
    // r0 + 64 p + 4 q .. + 3 of the half's operator at k = 64 ks + 4 j .. + 3.
    // A ring of NKS stages lives in registers: slot ks holds the current
    // pass's stage ks and is refilled with the next pass's stage ks (the
    // next half's first pass after the last one) as soon as it is used, so a
    // pass worth of loads is always in flight, across half-steps too.
    const size_t lane_off = (size_t)(r0 + 4 * q) * Kp + 4 * j;
    // this thread's row quad exists in pass p (only a partial last pass,
    // NR not a multiple of 64, leaves quads out)
    constexpr bool WHOLE = NR % kStrRows == 0;
    auto quad_in = [&](int p) { return WHOLE || kStrRows * p + 4 * q < NR; };
    float4 ring[NKS][4];
    if (!WHOLE) {  // quads absent from the first pass never load theirs
#pragma unroll
        for (int ks = 0; ks < NKS; ++ks)
#pragma unroll
            for (int r = 0; r < 4; ++r) ring[ks][r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (N > 0 && quad_in(0)) {
        const float* src = Avs + lane_off;
#pragma unroll
        for (int ks = 0; ks < NKS; ++ks)
#pragma unroll
            for (int r = 0; r < 4; ++r)
                ring[ks][r] = __ldcg(reinterpret_cast<const float4*>(src + (size_t)r * Kp + ks * kStrKC));
    }

    float* traces = static_cast<float*>(a.traces);
    const float* Cp = static_cast<const float*>(a.C_p);
    const int H = Kp / 64;                            // the split kernel's receiver slabs
    const int rpc = (a.R + H - 1) / H;
    for (int n = 0; n < N; ++n) {
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const float* X = h ? Vf : Sf;             // operand of this half
            float* Y = h ? Sf : Vf;                   // state updated in its own rows
            float* cY = h ? cS : cV;
            const int Kown = h ? a.Ks : a.Kv;
#pragma unroll 1
            for (int p = 0; p < NP; ++p) {
                // the pass whose stages refill the ring
                const bool last = p + 1 == NP;
                const bool has_next = !(last && h == 1 && n + 1 == N) && quad_in(last ? 0 : p + 1);
                const float* nsrc = (last ? (h ? Avs : Asv) : (h ? Asv : Avs)) +
                                    (size_t)(last ? 0 : (p + 1) * kStrRows) * Kp + lane_off;
                float acc[4][CB];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < CB; ++cc) acc[r][cc] = 0.f;
#pragma unroll
                for (int ks = 0; ks < NKS; ++ks) {
                    float op[4][4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        op[r][0] = ring[ks][r].x;
                        op[r][1] = ring[ks][r].y;
                        op[r][2] = ring[ks][r].z;
                        op[r][3] = ring[ks][r].w;
                    }
                    if (has_next) {
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            ring[ks][r] = __ldcg(reinterpret_cast<const float4*>(nsrc + (size_t)r * Kp + ks * kStrKC));
                    }
                    float x[CB][4];
#pragma unroll
                    for (int cc = 0; cc < CB; ++cc) load4(X + (size_t)cc * Kp + 64 * ks + 4 * j, x[cc]);
                    // the split kernel's FMA order: k ascending within the lane's stripe
#pragma unroll
                    for (int t = 0; t < 4; ++t)
#pragma unroll
                        for (int cc = 0; cc < CB; ++cc)
#pragma unroll
                            for (int r = 0; r < 4; ++r)
                                acc[r][cc] = __fmaf_rn(op[r][t], x[cc][t], acc[r][cc]);
                }
                // reduce-scatter over the 16 k lanes and the fused epilogue
                float v[4 * CB];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < CB; ++cc) v[r * CB + cc] = acc[r][cc];
                int vi;
                bool active;
                const float tot = reduce_scatter16<float, 4 * CB>(v, j, vi, active);
                const int rl = p * kStrRows + 4 * q + vi / CB;
                const int c = vi % CB;
                if (active && quad_in(p) && c < ncol && r0 + rl < Kown) {
                    float inc = tot;
                    if (h == 0) inc = __fmaf_rn(gown[rl], fcol[c], inc);
                    inc = inc * dt;
                    float* yp = Y + c * Kp + r0 + rl;
                    *yp = kahan_add(*yp, inc, cY[c * NR + rl]);
                }
            }
            __syncthreads();
            // copy the new own rows into every peer's full copy
            for (int idx = tid; idx < kStrCols * (NR / 4); idx += kStrThreads) {
                const int c = idx / (NR / 4), q4 = idx % (NR / 4);
                float* src = Y + c * Kp + r0 + 4 * q4;
                const float4 val = *reinterpret_cast<const float4*>(src);
#pragma unroll
                for (int pp = 1; pp < CSZ; ++pp)
                    *reinterpret_cast<float4*>(cluster.map_shared_rank(src, (crank + pp) % CSZ)) = val;
            }
            // forcing of the next step (its first use is after the barrier below)
            if (h == 1 && tid < ncol && n + 1 < N) {
                float f = 0.f;
                if (a.ftab) f = static_cast<const float*>(a.ftab)[(size_t)(n + 1) * a.Mtot + col0 + tid];
                else if (a.Tper) f = wavelet_eval_pre(a.wavelet, (long long)a.n0 + n + 1, a.dt, Tpre[2 * tid], Tpre[2 * tid + 1]);
                fcol[tid] = f;
            }
            cluster.sync();
            // receiver traces of V^{n+1}: the split kernel's receiver slabs
            // crank, crank + CSZ, ..., each with the same warp tiles
            if (h == 0 && traces && ((n + 1) % a.r) == 0) {
                const int rec = (n + 1) / a.r - 1;
                for (int sl = crank; sl < H; sl += CSZ) {
                    const int nj = min(rpc, a.R - sl * rpc);
                    if (nj <= 0) break;
                    split_traces(Cp + (size_t)sl * rpc * Kp, Vf, Kp, nj, ncol, warp, lane,
                                 traces + ((size_t)rec * a.Mtot + col0) * a.R + sl * rpc, a.R);
                }
            }
        }
    }
    // ---- write back the own rows and carries
    int bad = 0;
    for (int idx = tid; idx < ncol * NR; idx += kStrThreads) {
        const int c = idx / NR, rl = idx % NR, row = r0 + rl;
        if (row < a.Kv) {
            const float x = Vf[c * Kp + row];
            static_cast<float*>(a.V)[(size_t)(col0 + c) * a.Kv + row] = x;
            if (a.compV) static_cast<float*>(a.compV)[(size_t)(col0 + c) * a.Kv + row] = cV[c * NR + rl];
            bad |= !is_finite(x);
        }
        if (row < a.Ks) {
            const float x = Sf[c * Kp + row];
            static_cast<float*>(a.S)[(size_t)(col0 + c) * a.Ks + row] = x;
            if (a.compS) static_cast<float*>(a.compS)[(size_t)(col0 + c) * a.Ks + row] = cS[c * NR + rl];
            bad |= !is_finite(x);
        }
    }
    bad = __syncthreads_or(bad);
    if (bad && tid == 0 && a.status) atomicCAS(a.status, 0, 6 /* ROM_E_NONFINITE */);
}

}  // namespace romk
