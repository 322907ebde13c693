// Cluster-persistent SIMT kernel for the rank-2 Galerkin leapfrog.
//
// One launch integrates all nsteps steps.  Work split (GB300 layout):
//  * A thread-block cluster of CS = Kp / 32 CTAs owns one block of Wv state
//    columns (realizations) for the whole run.  Columns are independent
//    (Sec. 2.4: the rank-2 system is M rank-1 systems sharing the operator),
//    so clusters never talk to each other.
//  * CTA `rank` of a cluster owns rows [32 rank, 32 rank + 32) of both V and S
//    and keeps the matching 32 rows of Avs and Asv in REGISTERS for the whole
//    run (thread (row pair p, chunk j) holds rows 2p, 2p+1 at k = 64 i + 4 j + q).
//  * Every CTA keeps a full copy of its column block of V and S in shared
//    memory.  A half-step reads the whole operand (S for the velocity update,
//    the new V for the stress update, Sec. 3.1 "velocity first"), updates its
//    own 32 rows, and pushes those rows into the peer CTAs' copies through
//    distributed shared memory; one cluster barrier per half-step publishes
//    them.
//  * The epilogue fuses the point-source forcing g f_n^T (Sec. 2.2, 3.2), the
//    Kahan-compensated FP32 state update, and every r steps the receiver traces
//    y = C V (Sec. 4.5.2, rows of C split across the cluster).
// Variants of the same body:
//  * FP64 beyond Kp = 256 and FP32 beyond Kp = 512 re-read each CTA's operator
//    rows from L2 every half-step instead of holding them (FP32: two 32-row
//    tiles per CTA, or more on smaller clusters).
//  * GEN (FP32 with streamed operators): the row tiles are dealt out to any
//    cluster size and the products run on a 4-row, 32-lane half-step, which
//    feeds 16 multiply-adds from each 16-byte state read instead of 8.
//  * rank2_wl_kernel: the batched work list, one persistent launch whose
//    clusters take (job, column block) items of jobs of any Kp <= 1024.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "rom_internal.h"

namespace romk {

namespace cg = cooperative_groups;

constexpr int kThreads = 256;     // 16 row pairs x 16 k-chunks
constexpr int kRowsPerCta = 32;

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared-memory carve-up of one CTA (byte offsets).
struct Rank2Smem {
    size_t Vf, Sf, C, f, T, g, cV, cS, total;
};

// nrt: 32-row tiles owned per CTA (1, or 2 with operators streamed from L2;
// the work-list launch: the most any CTA of the cluster owns).
template <typename T>
__host__ __device__ inline Rank2Smem rank2_smem_layout(int Wa, int Kp, int rpc, int nrt = 1) {
    Rank2Smem s{};
    size_t o = 0;
    s.Vf = o; o += align16((size_t)Wa * Kp * sizeof(T));
    s.Sf = o; o += align16((size_t)Wa * Kp * sizeof(T));
    s.C = o;  o += align16((size_t)rpc * Kp * sizeof(T));
    s.f = o;  o += align16((size_t)Wa * sizeof(T));
    s.T = o;  o += align16((size_t)Wa * sizeof(T));
    s.g = o;  o += align16((size_t)nrt * kRowsPerCta * sizeof(T));
    s.cV = o; o += align16((size_t)nrt * Wa * kRowsPerCta * sizeof(float));
    s.cS = o; o += align16((size_t)nrt * Wa * kRowsPerCta * sizeof(float));
    s.total = o;
    return s;
}

// The value index reduce_scatter16<T, NV> leaves with lane chunk j (the same
// stage rule, without the data), so that a lane can fetch what its epilogue
// needs before the products.
template <int NV>
__device__ __forceinline__ int rs16_slot(int j) {
    int base = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int n = NV >> s;
        if (n > 1 && (j & (8 >> s))) base += n / 2;
    }
    return base;
}

__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }

// Butterfly reduce-scatter of NV partial sums over the 16 lanes of a
// half-warp (lane bits 0..3).  Afterwards the lane holds the full sum of
// value index `vi`; when NV < 16 the lowest bits are all-reduced, and only
// lanes with those bits clear report `active`.
template <typename T, int NV>
__device__ __forceinline__ T reduce_scatter16(T (&v)[NV], int j, int& vi, bool& active) {
    static_assert(NV >= 1 && NV <= 16 && (NV & (NV - 1)) == 0, "NV must be a power of 2 <= 16");
    int base = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int o = 8 >> s;
        const int n = NV >> s;  // values still held before this stage
        if (n > 1) {
            const int half = n / 2;
            const bool up = (j & o) != 0;
#pragma unroll
            for (int k = 0; k < half; ++k) {
                const T send = up ? v[k] : v[k + half];
                const T keep = up ? v[k + half] : v[k];
                v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
            base += up ? half : 0;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
    vi = base;
    constexpr int allred_bits = (NV >= 16) ? 0 : (NV == 8 ? 1 : (NV == 4 ? 2 : (NV == 2 ? 3 : 4)));
    active = (j & ((1 << allred_bits) - 1)) == 0;
    return v[0];
}

// One half-step on the CTA's own 32 rows:  Y_own += dt (op . X [+ g f^T]).
template <typename T, int KI, int CB, bool FORCED>
__device__ __forceinline__ void half_step(const T (&op)[2][4 * KI], const T* __restrict__ X,
                                          T* __restrict__ Y, float* __restrict__ comp,
                                          const T* __restrict__ gown, const T* __restrict__ fcol,
                                          const T dt, const int Wa, const int Kp, const int row0,
                                          const int rp, const int j) {
    for (int c0 = 0; c0 < Wa; c0 += CB) {
        T acc[2][CB];
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) { acc[0][cc] = T(0); acc[1][cc] = T(0); }
#pragma unroll
        for (int i = 0; i < KI; ++i) {
            T x[CB][4];
#pragma unroll
            for (int cc = 0; cc < CB; ++cc) load4(X + (size_t)(c0 + cc) * Kp + 64 * i + 4 * j, x[cc]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
#pragma unroll
                for (int cc = 0; cc < CB; ++cc) {
                    acc[0][cc] = fmadd(op[0][4 * i + q], x[cc][q], acc[0][cc]);
                    acc[1][cc] = fmadd(op[1][4 * i + q], x[cc][q], acc[1][cc]);
                }
            }
        }
        T v[2 * CB];
#pragma unroll
        for (int cc = 0; cc < CB; ++cc) { v[cc] = acc[0][cc]; v[CB + cc] = acc[1][cc]; }
        int vi;
        bool active;
        const T tot = reduce_scatter16<T, 2 * CB>(v, j, vi, active);
        if (active) {
            const int rl = 2 * rp + vi / CB;
            const int c = c0 + vi % CB;
            T* yp = Y + (size_t)c * Kp + row0 + rl;
            T inc = tot;
            if (FORCED) inc = fmadd(gown[rl], fcol[c], inc);
            inc = inc * dt;
            if constexpr (sizeof(T) == 4) {
                *yp = kahan_add(*yp, inc, comp[c * kRowsPerCta + rl]);
            } else {
                *yp = *yp + inc;
            }
        }
    }
}

// Copy the CTA's own 32 rows of every column of buffer Y into the same place
// of every other CTA of the cluster (distributed shared memory stores).
template <typename T>
__device__ __forceinline__ void push_own_rows(cg::cluster_group& cluster, T* Y, int Wa, int Kp,
                                              int row0, int cs, int crank, int nrt) {
    const int VPC = nrt * kRowsPerCta * (int)sizeof(T) / 16;  // 16-byte vectors per column
    const int nvec = Wa * VPC;
    for (int idx = threadIdx.x; idx < nvec; idx += kThreads) {
        const int c = idx / VPC, part = idx % VPC;
        float4* src = reinterpret_cast<float4*>(Y + (size_t)c * Kp + row0) + part;
        const float4 val = *src;
        for (int k = 1; k < cs; ++k) {
            int d = crank + k;
            if (d >= cs) d -= cs;
            float4* dst = cluster.map_shared_rank(src, d);
            *dst = val;
        }
    }
}

template <typename T, int KI>
__device__ __forceinline__ void load_op_rows(T (&op)[2][4 * KI], const T* __restrict__ A, int Kp,
                                             int row, int j) {
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
#pragma unroll
        for (int i = 0; i < KI; ++i) {
            T x[4];
            load4_ro(A + (size_t)(row + rr) * Kp + 64 * i + 4 * j, x);
#pragma unroll
            for (int q = 0; q < 4; ++q) op[rr][4 * i + q] = x[q];
        }
    }
}

// ---- the work-list kernel's half-step (FP32, operators streamed from L2):
// warp w holds rows 4w .. 4w + 3 of a 32-row tile and lane l the k values
// 128 i + 4 l + q, so each 16-byte read of the state feeds 16 multiply-adds
// (4 rows x 4 k) and the partial sums meet in a 32-lane reduce-scatter.
// Only k < Kp exist (Kp a multiple of 64: the last group may be half full).

// Butterfly reduce-scatter of 32 partial sums over the 32 lanes of a warp:
// afterwards lane l holds the full sum of value index `vi`.
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane, int& vi) {
    int base = 0;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int o = 16 >> s;
        const int half = 16 >> s;  // values kept after this stage
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const float send = up ? v[k] : v[k + half];
            const float keep = up ? v[k + half] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
        base += up ? half : 0;
    }
    vi = base;
    return v[0];
}

template <int KQ>
__device__ __forceinline__ void wl_load_op(float (&op)[4][4 * KQ], const float* __restrict__ A, int Kp,
                                             int row, int lane) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int i = 0; i < KQ; ++i) {
            float x[4] = {0.f, 0.f, 0.f, 0.f};  // k >= Kp: never used
            if (128 * i + 4 * lane < Kp) load4_ro(A + (size_t)(row + r) * Kp + 128 * i + 4 * lane, x);
#pragma unroll
            for (int q = 0; q < 4; ++q) op[r][4 * i + q] = x[q];
        }
    }
}

// Y_own += dt (op . X [+ g f^T]) on the tile starting at row0 (8 columns a pass).
template <int KQ, bool FORCED>
__device__ __forceinline__ void wl_half_step(const float (&op)[4][4 * KQ], const float* __restrict__ X,
                                               float* __restrict__ Y, float* __restrict__ comp,
                                               const float* __restrict__ gown,
                                               const float* __restrict__ fcol, const float dt,
                                               const int Wa, const int Kp, const int row0,
                                               const int warp, const int lane) {
    constexpr int CB = 8;
    for (int c0 = 0; c0 < Wa; c0 += CB) {
        float acc[4][CB];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int cc = 0; cc < CB; ++cc) acc[r][cc] = 0.f;
#pragma unroll
        for (int i = 0; i < KQ; ++i) {
            if (128 * i + 4 * lane >= Kp) continue;
            float x[CB][4];
#pragma unroll
            for (int cc = 0; cc < CB; ++cc) load4(X + (size_t)(c0 + cc) * Kp + 128 * i + 4 * lane, x[cc]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int cc = 0; cc < CB; ++cc)
#pragma unroll
                    for (int r = 0; r < 4; ++r) acc[r][cc] = fmadd(op[r][4 * i + q], x[cc][q], acc[r][cc]);
        }
        float v[4 * CB];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int cc = 0; cc < CB; ++cc) v[r * CB + cc] = acc[r][cc];
        int vi;
        const float tot = reduce_scatter32(v, lane, vi);
        const int rl = 4 * warp + vi / CB;
        const int c = c0 + vi % CB;
        float inc = tot;
        if (FORCED) inc = fmadd(gown[rl], fcol[c], inc);
        inc = inc * dt;
        float* yp = Y + (size_t)c * Kp + row0 + rl;
        *yp = kahan_add(*yp, inc, comp[c * kRowsPerCta + rl]);
    }
}

// Forcing value f_n of local column c (global column gc0 + c).
template <typename T>
__device__ __forceinline__ T forcing_at(const Rank2Args& a, const T* Tcol, int c, int ncol,
                                        int gc0, int n) {
    if (c >= ncol) return T(0);
    if (a.ftab) return static_cast<const T*>(a.ftab)[(size_t)n * a.Mtot + gc0 + c];
    return (T)wavelet_eval(a.wavelet, (long long)a.n0 + n, a.dt, Tcol[c]);
}

// The reduced reference state's share of a half-step on the CTA's own rows:
// Y_own += dt Xref, with the same Kahan carries (FP32), as a pass after the
// products (Xref: the block's first column, Krows x columns).  Used only when
// the term is given, so the product loop above is the same with or without it.
template <typename T>
__device__ __forceinline__ void add_reference(T* __restrict__ Y, float* __restrict__ comp,
                                              const T* __restrict__ Xref, const int Krows,
                                              const int ncol, const T dt, const int Wa,
                                              const int Kp, const int row0, const int nrt) {
    for (int idx = threadIdx.x; idx < nrt * ncol * kRowsPerCta; idx += kThreads) {
        const int rt = idx / (ncol * kRowsPerCta);
        const int rem = idx - rt * ncol * kRowsPerCta;
        const int c = rem / kRowsPerCta, rl = rem % kRowsPerCta;
        const int row = row0 + rt * kRowsPerCta + rl;
        if (row >= Krows) continue;
        const T inc = Xref[(size_t)c * Krows + row] * dt;
        T* yp = Y + (size_t)c * Kp + row;
        if constexpr (sizeof(T) == 4) {
            *yp = kahan_add(*yp, inc, comp[(size_t)rt * Wa * kRowsPerCta + c * kRowsPerCta + rl]);
        } else {
            *yp = *yp + inc;
        }
    }
}

// The one-block kernel's work on one column block: columns [gc0, gc0 + ncol)
// of the caller's arrays, operator `gop` of the table (rank-3 launch) or the
// launch's own operator (gop null).
// GEN (work-list launch, operators streamed from L2, FP32): the Kp / 32 row
// tiles are dealt out to the cluster's CTAs as evenly as they go (the first
// Kp/32 mod cs CTAs take one more; a CTA may own none), a.nrt is the most
// any CTA owns, and the products run on the 4-row half-step above for any
// Kp <= 64 KI.  Otherwise every CTA owns a.nrt tiles and Kp = 64 KI.
template <typename T, int KI, int CB, bool RESIDENT, bool GEN = false>
__device__ __forceinline__ void simt_body(cg::cluster_group& cluster, const Rank2Args& a,
                                          const GroupOp* gop, const int gc0, const int ncol) {
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int Wa = a.Wa;
    const int Kp = a.Kp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = lane & 15;
    const int rp = warp * 2 + (lane >> 4);
    const int nrt = a.nrt;  // tiles the layout holds per CTA
    int nrt_own = nrt, row0 = crank * nrt * kRowsPerCta;
    if (GEN) {
        const int tiles = Kp / kRowsPerCta, base = tiles / cs, rem = tiles % cs;
        nrt_own = base + (crank < rem ? 1 : 0);
        row0 = (crank * base + (crank < rem ? crank : rem)) * kRowsPerCta;
    }
    const int own_rows = nrt_own * kRowsPerCta;
    const T dt = (T)a.dt;

    extern __shared__ __align__(16) unsigned char smem[];
    // receiver rows staged in shared memory, or (c_global: too many to stage
    // beside the state) read from the row-major C in global memory
    const Rank2Smem L = rank2_smem_layout<T>(Wa, Kp, a.c_global ? 0 : a.rpc, nrt);
    T* Vf = reinterpret_cast<T*>(smem + L.Vf);
    T* Sf = reinterpret_cast<T*>(smem + L.Sf);
    T* Cown = reinterpret_cast<T*>(smem + L.C);
    T* fcol = reinterpret_cast<T*>(smem + L.f);
    T* Tcol = reinterpret_cast<T*>(smem + L.T);
    T* gown = reinterpret_cast<T*>(smem + L.g);
    float* cV = reinterpret_cast<float*>(smem + L.cV);
    float* cS = reinterpret_cast<float*>(smem + L.cS);

    const T* __restrict__ Vin = static_cast<const T*>(a.V);
    const T* __restrict__ Sin = static_cast<const T*>(a.S);

    // ---- load the column block (all rows) and the per-CTA constants
    for (int idx = tid; idx < Wa * Kp; idx += kThreads) {
        const int c = idx / Kp, k = idx - (idx / Kp) * Kp;
        Vf[idx] = (c < ncol && k < a.Kv) ? Vin[(size_t)(gc0 + c) * a.Kv + k] : T(0);
        Sf[idx] = (c < ncol && k < a.Ks) ? Sin[(size_t)(gc0 + c) * a.Ks + k] : T(0);
    }
    // carries: [row tile][column][32 rows]
    for (int idx = tid; idx < nrt_own * Wa * kRowsPerCta; idx += kThreads) {
        const int rt = idx / (Wa * kRowsPerCta);
        const int rem = idx - rt * Wa * kRowsPerCta;
        const int c = rem / kRowsPerCta, rl = rem % kRowsPerCta, row = row0 + rt * kRowsPerCta + rl;
        const float* cvin = static_cast<const float*>(a.compV);
        const float* csin = static_cast<const float*>(a.compS);
        cV[idx] = (cvin && c < ncol && row < a.Kv) ? cvin[(size_t)(gc0 + c) * a.Kv + row] : 0.f;
        cS[idx] = (csin && c < ncol && row < a.Ks) ? csin[(size_t)(gc0 + c) * a.Ks + row] : 0.f;
    }
    const T* Cp = static_cast<const T*>(gop ? gop->C_p : a.C_p);
    for (int idx = tid; idx < (a.c_global ? 0 : a.rpc * Kp); idx += kThreads) {
        const int jj = idx / Kp, k = idx % Kp, jr = crank * a.rpc + jj;
        Cown[idx] = (Cp && jr < a.R) ? Cp[(size_t)jr * Kp + k] : T(0);
    }
    for (int i = tid; i < own_rows; i += kThreads) gown[i] = static_cast<const T*>(gop ? gop->g_p : a.g_p)[row0 + i];
    for (int c = tid; c < Wa; c += kThreads) {
        Tcol[c] = (a.Tper && c < ncol) ? static_cast<const T*>(a.Tper)[gc0 + c] : T(1);
    }
    __syncthreads();
    for (int c = tid; c < Wa; c += kThreads) {
        fcol[c] = (a.Tper || a.ftab) ? forcing_at<T>(a, Tcol, c, ncol, gc0, 0) : T(0);
    }

    T opA[2][4 * KI];
    T opB[2][4 * KI];
    constexpr int KQ = (KI + 1) / 2;  // GEN: k groups of 128 covering 64 KI
    float opQ[GEN ? 4 : 1][GEN ? 4 * KQ : 1];  // GEN: 4 rows of them
    const T* __restrict__ Avs = static_cast<const T*>(gop ? gop->Avs_rm : a.Avs_rm);
    const T* __restrict__ Asv = static_cast<const T*>(gop ? gop->Asv_rm : a.Asv_rm);
    if (RESIDENT && nrt_own > 0) {
        load_op_rows<T, KI>(opA, Avs, Kp, row0 + 2 * rp, j);
        load_op_rows<T, KI>(opB, Asv, Kp, row0 + 2 * rp, j);
    }
    // every CTA's copies must be initialised before any peer pushes into them
    cluster.sync();

    T* traces = static_cast<T*>(a.traces);
    for (int n = 0; n < a.nsteps; ++n) {
        // ---- velocity half-step: V_own += dt (Avs_own S + g f_n^T [+ Xv])
        for (int rt = 0; rt < nrt_own; ++rt) {
            const int rowt = row0 + rt * kRowsPerCta;
            if constexpr (GEN) {
                wl_load_op<KQ>(opQ, Avs, Kp, rowt + 4 * warp, lane);
                wl_half_step<KQ, true>(opQ, Sf, Vf, cV + rt * Wa * kRowsPerCta,
                                             gown + rt * kRowsPerCta, fcol, dt, Wa, Kp, rowt, warp, lane);
            } else {
                if (!RESIDENT) load_op_rows<T, KI>(opA, Avs, Kp, rowt + 2 * rp, j);
                half_step<T, KI, CB, true>(opA, Sf, Vf, cV + rt * Wa * kRowsPerCta,
                                           gown + rt * kRowsPerCta, fcol, dt, Wa, Kp, rowt, rp, j);
            }
        }
        if (a.Xv) {  // kernel parameters, read where used: no register held across the loop
            __syncthreads();
            add_reference<T>(Vf, cV, static_cast<const T*>(a.Xv) + (size_t)gc0 * a.Kv,
                             a.Kv, ncol, dt, Wa, Kp, row0, nrt_own);
        }
        __syncthreads();
        push_own_rows<T>(cluster, Vf, Wa, Kp, row0, cs, crank, nrt_own);
        cluster.sync();

        // ---- stress half-step with the new velocity: S_own += dt (Asv_own V [+ Xs])
        for (int rt = 0; rt < nrt_own; ++rt) {
            const int rowt = row0 + rt * kRowsPerCta;
            if constexpr (GEN) {
                wl_load_op<KQ>(opQ, Asv, Kp, rowt + 4 * warp, lane);
                wl_half_step<KQ, false>(opQ, Vf, Sf, cS + rt * Wa * kRowsPerCta, gown, fcol, dt, Wa,
                                              Kp, rowt, warp, lane);
            } else {
                if (!RESIDENT) load_op_rows<T, KI>(opB, Asv, Kp, rowt + 2 * rp, j);
                half_step<T, KI, CB, false>(opB, Vf, Sf, cS + rt * Wa * kRowsPerCta, gown, fcol, dt, Wa,
                                            Kp, rowt, rp, j);
            }
        }
        if (a.Xs) {
            __syncthreads();
            add_reference<T>(Sf, cS, static_cast<const T*>(a.Xs) + (size_t)gc0 * a.Ks,
                             a.Ks, ncol, dt, Wa, Kp, row0, nrt_own);
            __syncthreads();
        }

        // ---- receiver traces y = C V^{n+1} (this CTA's rows of C)
        if (traces && ((n + 1) % a.r) == 0) {
            const int rec = (n + 1) / a.r - 1;
            const int npair = a.rpc * ncol;
            for (int pr = warp; pr < npair; pr += kThreads / 32) {
                const int jj = pr / ncol, c = pr % ncol, jr = crank * a.rpc + jj;
                if (jr >= a.R) continue;
                const T* crow = a.c_global ? Cp + (size_t)jr * Kp : Cown + (size_t)jj * Kp;
                T acc = T(0);
                for (int k = 4 * lane; k < Kp; k += 128) {
                    T cx[4], vx[4];
                    load4(crow + k, cx);
                    load4(Vf + (size_t)c * Kp + k, vx);
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc = fmadd(cx[q], vx[q], acc);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) traces[((size_t)rec * a.Mtot + gc0 + c) * a.R + jr] = acc;
            }
        }
        // ---- forcing of the next step (read by the next velocity epilogue)
        if (n + 1 < a.nsteps) {
            for (int c = tid; c < Wa; c += kThreads) {
                fcol[c] = (a.Tper || a.ftab) ? forcing_at<T>(a, Tcol, c, ncol, gc0, n + 1) : T(0);
            }
        }
        __syncthreads();
        push_own_rows<T>(cluster, Sf, Wa, Kp, row0, cs, crank, nrt_own);
        cluster.sync();
    }

    // ---- write back this CTA's rows (and the Kahan carries)
    T* Vout = static_cast<T*>(a.V);
    T* Sout = static_cast<T*>(a.S);
    float* cvout = static_cast<float*>(a.compV);
    float* csout = static_cast<float*>(a.compS);
    int bad = 0;
    for (int idx = tid; idx < ncol * own_rows; idx += kThreads) {
        const int c = idx / own_rows, ro = idx % own_rows, row = row0 + ro;
        const int ci = (ro / kRowsPerCta) * Wa * kRowsPerCta + c * kRowsPerCta + ro % kRowsPerCta;
        if (row < a.Kv) {
            const T x = Vf[(size_t)c * Kp + row];
            Vout[(size_t)(gc0 + c) * a.Kv + row] = x;
            if (cvout) cvout[(size_t)(gc0 + c) * a.Kv + row] = cV[ci];
            bad |= !is_finite(x);
        }
        if (row < a.Ks) {
            const T x = Sf[(size_t)c * Kp + row];
            Sout[(size_t)(gc0 + c) * a.Ks + row] = x;
            if (csout) csout[(size_t)(gc0 + c) * a.Ks + row] = cS[ci];
            bad |= !is_finite(x);
        }
    }
    bad = __syncthreads_or(bad);
    if (bad && tid == 0 && a.status) atomicCAS(a.status, 0, (int)6 /* ROM_E_NONFINITE */);
}

// GEN: the 4-row half-step of the work-list kernel (FP32 with operators
// streamed from L2 and 8-column groups only).
template <typename T, int KI, int CB, bool RESIDENT, bool GEN = false>
__global__ void __launch_bounds__(kThreads, 1) rank2_simt_kernel(const Rank2Args a) {
    static_assert(!GEN || (sizeof(T) == 4 && CB == 8 && !RESIDENT), "GEN: FP32, 8-column groups, streamed");
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    // rank-3 grouped launch: operator `job` of the table, column block `blk` of it
    const int job = a.group ? (int)(blockIdx.x / cs) / a.group_cpj : 0;
    const int blk = a.group ? (int)(blockIdx.x / cs) % a.group_cpj : (int)(blockIdx.x / cs);
    const GroupOp* gop = a.group ? a.group + job : nullptr;
    const int col0 = blk * a.Wv;                 // first column of this block (within the job)
    const int ncol = min(a.Wv, a.M - col0);      // valid columns
    simt_body<T, KI, CB, RESIDENT, GEN>(cluster, a, gop, a.col_base + job * a.M + col0, ncol);
}

// Work-list launch of the batched scheduler (FP32): one persistent launch
// for jobs of any Kp <= 64 KI.  The clusters take (job, column block) items
// from a.items in the order a global counter hands them out, each job with
// its own operator, state, periods, traces, constants, width and Kp from the
// table a.group, until none are left.  The cluster size is the launch's:
// a job's rows are dealt out to its CTAs (simt_body, GEN) and its receiver
// rows split ceil(R / cs) per CTA, so one instance serves every job.
template <int KI, int CB>
__global__ void __launch_bounds__(kThreads, 1) rank2_wl_kernel(const Rank2Args a) {
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    __shared__ int s_item;
    for (;;) {
        if (crank == 0 && threadIdx.x == 0) {
            const int k = atomicAdd(a.item_counter, 1);
            for (int r = 0; r < cs; ++r) *cluster.map_shared_rank(&s_item, r) = k;
        }
        cluster.sync();
        const int k = s_item;
        if (k >= a.nitems) break;
        const WorkItem wi = a.items[k];
        const GroupOp* gop = a.group + wi.job;
        Rank2Args aj = a;
        aj.Avs_rm = gop->Avs_rm;
        aj.Asv_rm = gop->Asv_rm;
        aj.g_p = gop->g_p;
        aj.C_p = gop->C_p;
        aj.V = gop->V;
        aj.S = gop->S;
        aj.Tper = gop->Tper;
        aj.traces = gop->traces;
        aj.status = gop->status;
        aj.dt = gop->dt;
        aj.Kv = gop->Kv;
        aj.Ks = gop->Ks;
        aj.Kp = gop->Kp;
        aj.R = gop->R;
        aj.M = gop->M;
        aj.Mtot = gop->M;
        aj.wavelet = gop->wavelet;
        aj.Wv = aj.Wa = gop->Wa;
        aj.nrt = (gop->Kp / kRowsPerCta + cs - 1) / cs;
        aj.rpc = (gop->R + cs - 1) / cs;
        aj.c_global = gop->c_global;
        aj.col_base = 0;
        aj.group = nullptr;
        simt_body<float, KI, CB, false, true>(cluster, aj, nullptr, wi.col0, min(aj.Wv, wi.ncol));
        // every CTA has read the slot and finished the item before the next fetch
        cluster.sync();
    }
}

}  // namespace romk
