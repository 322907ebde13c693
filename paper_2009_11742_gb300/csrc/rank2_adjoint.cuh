// Reverse-time adjoint of the rank-2 leapfrog for the receiver-trace misfit
//     L = sum_{n=1..N} sum_m || C V_m^n - ystar_m^n ||^2 .
// The paper has no adjoint; this is the exact reverse of the forward step
// V^{n+1} = V^n + dt (Avs S^n + g f_n^T), S^{n+1} = S^n + dt Asv V^{n+1}
// (Sec. 3.1).  With lamV, lamS the adjoints of (V, S), reverse step n
// (n = N-1 .. 0) is
//     half A:  lamV <- lamV + 2 C^T r^{n+1} + dt Asv^T lamS      (= a_V^n)
//              dL/dT_m += dt g^T a_V^n[:, m] df/dT(t_n; T_m)
//     half B:  lamS <- lamS + dt Avs^T a_V^n
// with r^n = C V^n - ystar^n, starting from lamV = lamS = 0; after n = 0,
// lamV = dL/dV^0 and lamS = dL/dS^0.
//
// The kernel is the one-block cluster kernel of rank2_simt.cuh run backwards
// in time with the transposed operators (the column-major copies of Asv and
// Avs are the row-major Asv^T and Avs^T).  FP32: resident in registers up to
// Kp = 512 (one 32-row tile per CTA), and for 512 < Kp <= 1024 read from L2
// for each of the CTA's two 32-row tiles every half-step, as the forward
// kernel does there; the adjoint state is Kahan-compensated.  FP64 (the
// check path, Kp <= 512, one tile per CTA): resident up to Kp = 256 and
// read from L2 per half-step above, plain sums, as the FP64 forward kernel.
// Half A's epilogue adds the rank-R source 2 C^T r^{n+1}, read precomputed
// for the launch's range of steps (adj_source_kernel) and copied one step
// ahead.  A deterministic per-CTA column reduction accumulates the period
// gradient.  The split-role kernel below (FP32, Kp <= 512) is the faster
// form there.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "rank2_simt.cuh"
#include "rank2_split.cuh"
#include "rom_internal.h"

namespace romk {

// Steps of df/dT tabulated at a time (shared memory, kAdjTab x Wa values).
constexpr int kAdjTab = 64;

struct AdjSmem {
    size_t Vf, Sf, cV, cS, src, g, T, gT, dfT, total;
};

// nrt: 32-row tiles owned per CTA (1 for Kp <= 512, 2 above); T the element
// type (the carries are FP32 and only the FP32 path has them).  The source
// term arrives precomputed (src: two step buffers of Wa x own rows), so the
// layout does not depend on R.
template <typename T>
__host__ __device__ inline AdjSmem adj_smem_layout(int Wa, int Kp, int R, int nrt = 1) {
    (void)R;
    AdjSmem s{};
    const size_t own = (size_t)nrt * kRowsPerCta;
    const size_t ncarry = sizeof(T) == 4 ? (size_t)Wa * own : 0;
    size_t o = 0;
    s.Vf = o;   o += align16((size_t)Wa * Kp * sizeof(T));
    s.Sf = o;   o += align16((size_t)Wa * Kp * sizeof(T));
    s.cV = o;   o += align16(ncarry * sizeof(float));
    s.cS = o;   o += align16(ncarry * sizeof(float));
    s.src = o;  o += align16(2 * (size_t)Wa * own * sizeof(T));
    s.g = o;    o += align16(own * sizeof(T));
    s.T = o;    o += align16((size_t)Wa * sizeof(T));
    s.gT = o;   o += align16((size_t)Wa * sizeof(T));
    s.dfT = o;  o += align16((size_t)kAdjTab * Wa * sizeof(T));
    s.total = o;
    return s;
}

// Half A of a reverse step on one 32-row tile of the CTA (rows row0 ..):
//   Y_own += dt (op . X) + 2 C_own^T r   (Kahan-compensated in FP32),
// with C_own^T r read precomputed from asrc ([Wa][sstride], the tile's rows).
template <typename T, int KI, int CB>
__device__ __forceinline__ void adj_half_a(const T (&op)[2][4 * KI], const T* __restrict__ X,
                                           T* __restrict__ Y, float* __restrict__ comp,
                                           const T* __restrict__ asrc, const int sstride, const T dt,
                                           const int Wa, const int Kp, const int row0, const int rp,
                                           const int j) {
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
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int cc = 0; cc < CB; ++cc) {
                    acc[0][cc] = fmadd(op[0][4 * i + q], x[cc][q], acc[0][cc]);
                    acc[1][cc] = fmadd(op[1][4 * i + q], x[cc][q], acc[1][cc]);
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
            const T inc = fmadd(tot, dt, T(2) * asrc[c * sstride + rl]);
            T* yp = Y + (size_t)c * Kp + row0 + rl;
            if constexpr (sizeof(T) == 4) {
                *yp = kahan_add(*yp, inc, comp[c * kRowsPerCta + rl]);
            } else {
                *yp = *yp + inc;
            }
        }
    }
}

// Half A in the 4-row, 32-lane form of the work-list kernel (FP32 with the
// operators streamed from L2): warp w holds rows 4w .. 4w + 3 of the tile,
// lane l the k values 128 i + 4 l + q (k < Kp); the epilogue adds
// 2 C_own^T r, read precomputed from asrc ([Wa][sstride], the tile's rows).
template <int KQ>
__device__ __forceinline__ void wl_adj_half_a(const float (&op)[4][4 * KQ], const float* __restrict__ X,
                                              float* __restrict__ Y, float* __restrict__ comp,
                                              const float* __restrict__ asrc, const int sstride,
                                              const float dt, const int Wa, const int Kp, const int row0,
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
                    for (int r = 0; r < 4; ++r) acc[r][cc] = __fmaf_rn(op[r][4 * i + q], x[cc][q], acc[r][cc]);
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
        const float inc = __fmaf_rn(tot, dt, 2.f * asrc[c * sstride + rl]);
        float* yp = Y + (size_t)c * Kp + row0 + rl;
        *yp = kahan_add(*yp, inc, comp[c * kRowsPerCta + rl]);
    }
}

// KI = Kp / 64.  FP32 (GEN, KI <= 16): both halves run in the 4-row form;
// for KI <= 8 each CTA owns one 32-row tile and keeps its rows of both
// transposed operators in registers, above that the Kp / 32 row tiles are
// dealt out to the cluster's CTAs (the first Kp/32 mod cs take one more;
// a.nrt is the most any CTA owns) and the operators are streamed per tile.
// FP64 (KI <= 8): the 2-row form, one tile per CTA, resident for KI <= 4.
template <typename T, int KI, int CB>
__global__ void __launch_bounds__(kThreads, 1) rank2_adjoint_kernel(const AdjArgsT<T> a) {
    constexpr bool F32 = sizeof(T) == 4;
    static_assert(F32 ? KI <= 16 : KI <= 8, "unsupported size");
    constexpr bool GEN = F32;
    static_assert(!GEN || CB == 8, "the 4-row form runs 8-column groups");
    constexpr bool RES = F32 ? KI <= 8 : KI <= 4;
    constexpr int KQ = (KI + 1) / 2;  // GEN: k groups of 128
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int blk = blockIdx.x / cs;
    const int col0 = blk * a.Wv;
    const int ncol = min(a.Wv, a.M - col0);
    const int Wa = a.Wa, Kp = a.Kp, R = a.R;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = lane & 15;
    const int rp = warp * 2 + (lane >> 4);
    // row tiles: the layout holds NRT per CTA, this CTA owns nrt_own from row0
    const int NRT = GEN ? a.nrt : 1;
    const int OWN = NRT * kRowsPerCta;
    int nrt_own = NRT, row0 = crank * OWN;
    if (GEN) {
        const int tiles = Kp / kRowsPerCta, base = tiles / cs, rem = tiles % cs;
        nrt_own = base + (crank < rem ? 1 : 0);
        row0 = (crank * base + (crank < rem ? crank : rem)) * kRowsPerCta;
    }
    const int own_rows = nrt_own * kRowsPerCta;
    const T dt = (T)a.dt;

    extern __shared__ __align__(16) unsigned char smem[];
    const AdjSmem L = adj_smem_layout<T>(Wa, Kp, R, NRT);
    T* Vf = reinterpret_cast<T*>(smem + L.Vf);
    T* Sf = reinterpret_cast<T*>(smem + L.Sf);
    float* cV = reinterpret_cast<float*>(smem + L.cV);
    float* cS = reinterpret_cast<float*>(smem + L.cS);
    T* srcS = reinterpret_cast<T*>(smem + L.src);   // [2][Wa][OWN]: C^T r, by step parity
    T* gown = reinterpret_cast<T*>(smem + L.g);
    T* Tcol = reinterpret_cast<T*>(smem + L.T);
    T* gTacc = reinterpret_cast<T*>(smem + L.gT);
    T* dfT = reinterpret_cast<T*>(smem + L.dfT);    // [kAdjTab][Wa]: df/dT of the chunk

    for (int idx = tid; idx < Wa * Kp; idx += kThreads) {
        const int c = idx / Kp, k = idx % Kp;
        Vf[idx] = (c < ncol && k < a.Kv) ? a.lamV[(size_t)(col0 + c) * a.Kv + k] : T(0);
        Sf[idx] = (c < ncol && k < a.Ks) ? a.lamS[(size_t)(col0 + c) * a.Ks + k] : T(0);
    }
    // carries (FP32): [row tile][column][32 rows]
    for (int idx = tid; idx < (F32 ? nrt_own * Wa * kRowsPerCta : 0); idx += kThreads) {
        const int rt = idx / (Wa * kRowsPerCta);
        const int rem = idx - rt * Wa * kRowsPerCta;
        const int c = rem / kRowsPerCta, rl = rem % kRowsPerCta, row = row0 + rt * kRowsPerCta + rl;
        cV[idx] = (c < ncol && row < a.Kv) ? a.compV[(size_t)(col0 + c) * a.Kv + row] : 0.f;
        cS[idx] = (c < ncol && row < a.Ks) ? a.compS[(size_t)(col0 + c) * a.Ks + row] : 0.f;
    }
    for (int ro = tid; ro < OWN; ro += kThreads) gown[ro] = ro < own_rows ? a.g_p[row0 + ro] : T(0);
    for (int c = tid; c < Wa; c += kThreads) {
        Tcol[c] = (c < ncol) ? a.Tper[col0 + c] : T(1);
        gTacc[c] = (c < ncol) ? a.gTpart[(size_t)crank * a.M + col0 + c] : T(0);
    }
    T opA[GEN ? 1 : 2][GEN ? 1 : 4 * KI], opB[GEN ? 1 : 2][GEN ? 1 : 4 * KI];
    float opQA[GEN ? 4 : 1][GEN ? 4 * KQ : 1], opQB[GEN ? 4 : 1][GEN ? 4 * KQ : 1];
    if constexpr (GEN) {
        if (RES && nrt_own > 0) {
            wl_load_op<KQ>(opQA, a.opA_rm, Kp, row0 + 4 * warp, lane);
            wl_load_op<KQ>(opQB, a.opB_rm, Kp, row0 + 4 * warp, lane);
        }
    } else if (RES) {
        load_op_rows<T, KI>(opA, a.opA_rm, Kp, row0 + 2 * rp, j);
        load_op_rows<T, KI>(opB, a.opB_rm, Kp, row0 + 2 * rp, j);
    }
    // the own rows' C^T r of reverse step n (precomputed for the range) into
    // step buffer pb, 16 bytes (E rows) per copy, zero for absent columns and rows
    constexpr int E = 16 / (int)sizeof(T);
    auto prefetch_src = [&](int n, int pb) {
        T* dst = srcS + (size_t)pb * Wa * OWN;
        for (int idx = tid; idx < Wa * (OWN / E); idx += kThreads) {
            const int c = idx / (OWN / E), ro = E * (idx % (OWN / E));
            const bool ok = c < ncol && ro < own_rows;
            const T* gsrc = ok ? a.src + ((size_t)(n - a.n_lo) * a.M + col0 + c) * Kp + row0 + ro
                               : a.src;  // a valid address for the zero fill
            cp_async16(dst + (size_t)c * OWN + ro, gsrc, ok ? 16 : 0);
        }
    };
    if (a.n_hi > a.n_lo) prefetch_src(a.n_hi - 1, 0);
    cluster.sync();

    for (int n = a.n_hi - 1; n >= a.n_lo; --n) {
        // df/dT(t_n; T_c) for the next kAdjTab steps, all threads at once: the
        // evaluation (FP64 time arithmetic) stays off the per-step critical
        // path.  The previous chunk's last readers passed the cluster barrier
        // at the end of the previous step; the barrier after the residual
        // below publishes the new entries.
        const int done = a.n_hi - 1 - n;
        if (done % kAdjTab == 0) {
            for (int idx = tid; idx < kAdjTab * ncol; idx += kThreads) {
                const int i = idx / ncol, c = idx % ncol;
                if (n - i >= a.n_lo)
                    dfT[i * Wa + c] = wavelet_dT_eval<T>(a.wavelet, (long long)a.n0 + n - i, a.dt, Tcol[c]);
            }
        }
        const T* dfn = dfT + (done % kAdjTab) * Wa;
        // this step's C^T r, copied one step earlier into buffer done & 1; the
        // next step's copies go to the other buffer, whose last readers passed
        // the cluster barriers of the previous step
        cp_async_wait_all();
        __syncthreads();
        if (n > a.n_lo) prefetch_src(n - 1, (done + 1) & 1);
        // ---- half A: lamV <- lamV + 2 C^T r^{n+1} + dt Asv^T lamS
        for (int rt = 0; rt < nrt_own; ++rt) {
            const int rowt = row0 + rt * kRowsPerCta;
            if constexpr (GEN) {
                if (!RES) wl_load_op<KQ>(opQA, a.opA_rm, Kp, rowt + 4 * warp, lane);
                wl_adj_half_a<KQ>(opQA, Sf, Vf, cV + rt * Wa * kRowsPerCta,
                                  srcS + (size_t)(done & 1) * Wa * OWN + rt * kRowsPerCta, OWN, dt, Wa, Kp,
                                  rowt, warp, lane);
            } else {
                if (!RES) load_op_rows<T, KI>(opA, a.opA_rm, Kp, rowt + 2 * rp, j);
                adj_half_a<T, KI, CB>(opA, Sf, Vf, cV + rt * Wa * kRowsPerCta,
                                      srcS + (size_t)(done & 1) * Wa * OWN + rt * kRowsPerCta, OWN, dt, Wa, Kp,
                                      rowt, rp, j);
            }
        }
        __syncthreads();
        // period gradient: dt (g_own . a_V[:, c]) df/dT(t_n; T_c), fixed reduction order
        for (int c = warp; c < ncol; c += kThreads / 32) {
            T s = T(0);
            if (nrt_own > 0) s = gown[lane] * Vf[(size_t)c * Kp + row0 + lane];
            for (int rt = 1; rt < nrt_own; ++rt)
                s = fmadd(gown[rt * kRowsPerCta + lane], Vf[(size_t)c * Kp + row0 + rt * kRowsPerCta + lane], s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) gTacc[c] = fmadd(dt * s, dfn[c], gTacc[c]);
        }
        push_own_rows<T>(cluster, Vf, Wa, Kp, row0, cs, crank, nrt_own);
        cluster.sync();
        // ---- half B: lamS <- lamS + dt Avs^T a_V
        for (int rt = 0; rt < nrt_own; ++rt) {
            const int rowt = row0 + rt * kRowsPerCta;
            if constexpr (GEN) {
                if (!RES) wl_load_op<KQ>(opQB, a.opB_rm, Kp, rowt + 4 * warp, lane);
                wl_half_step<KQ, false>(opQB, Vf, Sf, cS + rt * Wa * kRowsPerCta, gown, gown, dt, Wa, Kp, rowt,
                                        warp, lane);
            } else {
                if (!RES) load_op_rows<T, KI>(opB, a.opB_rm, Kp, rowt + 2 * rp, j);
                half_step<T, KI, CB, false>(opB, Vf, Sf, cS + rt * Wa * kRowsPerCta, gown, gown, dt, Wa,
                                            Kp, rowt, rp, j);
            }
        }
        __syncthreads();
        push_own_rows<T>(cluster, Sf, Wa, Kp, row0, cs, crank, nrt_own);
        cluster.sync();
    }

    int bad = 0;
    for (int idx = tid; idx < ncol * own_rows; idx += kThreads) {
        const int c = idx / own_rows, ro = idx % own_rows, row = row0 + ro;
        const int ci = (ro / kRowsPerCta) * Wa * kRowsPerCta + c * kRowsPerCta + ro % kRowsPerCta;
        if (row < a.Kv) {
            const T x = Vf[(size_t)c * Kp + row];
            a.lamV[(size_t)(col0 + c) * a.Kv + row] = x;
            if (F32) a.compV[(size_t)(col0 + c) * a.Kv + row] = cV[ci];
            bad |= !is_finite(x);
        }
        if (row < a.Ks) {
            const T x = Sf[(size_t)c * Kp + row];
            a.lamS[(size_t)(col0 + c) * a.Ks + row] = x;
            if (F32) a.compS[(size_t)(col0 + c) * a.Ks + row] = cS[ci];
            bad |= !is_finite(x);
        }
    }
    for (int c = tid; c < ncol; c += kThreads) a.gTpart[(size_t)crank * a.M + col0 + c] = gTacc[c];
    bad = __syncthreads_or(bad);
    if (bad && tid == 0 && a.status) atomicCAS(a.status, 0, 6 /* ROM_E_NONFINITE */);
}

// ---- split-role reverse kernel (FP32, Kp <= 512).  The reverse step has
// the forward step's shape: half A updates lamV from lamS, half B updates
// lamS from the new lamV.  So the forward split kernel's schedule
// (rank2_split.cuh) carries over: two column blocks half a step apart,
// V-role CTAs holding their 64 rows of Asv^T in registers and owning those
// rows of lamV, S-role CTAs doing the same with Avs^T and lamS, each finished
// tile pushed into the other role's operand copy, one cluster barrier per
// phase.  Time runs backwards: block A takes reverse step n = n_hi - 1 - k in
// phase 2k, block B in phase 2k + 1.  The V role's epilogue adds 2 C^T r,
// which does not depend on the adjoint state: adj_source_kernel forms it for
// the launch's range of steps beforehand, and each V-role CTA copies its own
// rows of it one phase ahead.  The S role, whose operand copy holds the same
// new lamV, adds its slab's share of the period gradient to a per-CTA
// partial after each of its phases.
struct AdjSplitSmem {
    size_t X, own, comp, src, g, T, gT, dfT, total;
};

__host__ __device__ inline AdjSplitSmem adj_split_smem_layout(int Wa, int Kp, int R) {
    (void)R;  // the source term arrives precomputed, so the layout does not depend on R
    AdjSplitSmem s{};
    size_t o = 0;
    s.X = o;    o += align16((size_t)2 * Wa * Kp * sizeof(float));
    s.own = o;  o += align16((size_t)2 * Wa * kOwnStride * sizeof(float));
    s.comp = o; o += align16((size_t)2 * Wa * kOwnStride * sizeof(float));
    s.src = o;  o += align16((size_t)2 * Wa * kOwnStride * sizeof(float));
    s.g = o;    o += align16((size_t)kSplitRows * sizeof(float));
    s.T = o;    o += align16((size_t)2 * Wa * sizeof(float));
    s.gT = o;   o += align16((size_t)2 * Wa * sizeof(float));
    s.dfT = o;  o += align16((size_t)2 * kAdjTab * Wa * sizeof(float));
    s.total = o;
    return s;
}

template <int KI>
__global__ void __launch_bounds__(kThreads, 1) rank2_adjoint_split_kernel(const AdjArgsT<float> a) {
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int H = cs / 2;
    const int crank = (int)cluster.block_rank();
    const bool vrole = crank < H;
    const int sl = vrole ? crank : crank - H;  // row slab
    const int row0 = sl * kSplitRows;
    const int peer0 = vrole ? H : 0;           // first CTA of the other role
    const int clu = blockIdx.x / cs;
    const int Wa = a.Wa, Kp = a.Kp, R = a.R, M = a.M;
    const int gc0_0 = 2 * clu * a.Wv, gc0_1 = gc0_0 + a.Wv;
    const int nc0 = max(0, min(a.Wv, M - gc0_0)), nc1 = max(0, min(a.Wv, M - gc0_1));
    auto gc0 = [&](int b) { return b ? gc0_1 : gc0_0; };
    auto ncol = [&](int b) { return b ? nc1 : nc0; };
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = lane & 15;
    const int q = warp * 2 + (lane >> 4);      // row quad
    const float dt = (float)a.dt;

    extern __shared__ __align__(16) unsigned char smem[];
    const AdjSplitSmem L = adj_split_smem_layout(Wa, Kp, R);
    float* X = reinterpret_cast<float*>(smem + L.X);         // [2][Wa][Kp] operand copies
    float* own = reinterpret_cast<float*>(smem + L.own);     // [2][Wa][72] owned rows
    float* comp = reinterpret_cast<float*>(smem + L.comp);   // [2][Wa][72] Kahan carries
    float* srcS = reinterpret_cast<float*>(smem + L.src);    // [2][Wa][72] C^T r, by phase parity
    float* gown = reinterpret_cast<float*>(smem + L.g);      // [64]
    float* Tcol = reinterpret_cast<float*>(smem + L.T);      // [2][Wa]
    float* gTacc = reinterpret_cast<float*>(smem + L.gT);    // [2][Wa] period-gradient partials
    float* dfT = reinterpret_cast<float*>(smem + L.dfT);     // [2][kAdjTab][Wa] df/dT per block

    const int Kown = vrole ? a.Kv : a.Ks;
    const float* own_in = vrole ? a.lamV : a.lamS;
    const float* comp_in = vrole ? a.compV : a.compS;
    // operand copies: V role = the full lamS of each block; the S role's are
    // filled by the first V-role pushes
    for (int idx = tid; idx < 2 * Wa * Kp; idx += kThreads) {
        const int b = idx / (Wa * Kp);
        const int rem = idx - b * Wa * Kp;
        const int c = rem / Kp, k = rem - (rem / Kp) * Kp;
        X[idx] = (vrole && c < ncol(b) && k < a.Ks) ? a.lamS[(size_t)(gc0(b) + c) * a.Ks + k] : 0.f;
    }
    for (int idx = tid; idx < 2 * Wa * kOwnStride; idx += kThreads) {
        const int b = idx / (Wa * kOwnStride);
        const int rem = idx - b * Wa * kOwnStride;
        const int c = rem / kOwnStride, rl = rem % kOwnStride, row = row0 + rl;
        const bool ok = rl < kSplitRows && c < ncol(b) && row < Kown;
        own[idx] = ok ? own_in[(size_t)(gc0(b) + c) * Kown + row] : 0.f;
        comp[idx] = ok ? comp_in[(size_t)(gc0(b) + c) * Kown + row] : 0.f;
    }
    if (tid < kSplitRows) gown[tid] = a.g_p[row0 + tid];  // the S role's gradient slab
    for (int idx = tid; idx < 2 * Wa; idx += kThreads) {
        const int b = idx / Wa, c = idx % Wa;
        const bool ok = c < ncol(b);
        Tcol[idx] = ok ? a.Tper[gc0(b) + c] : 1.f;
        gTacc[idx] = ok ? a.gTpart[(size_t)crank * M + gc0(b) + c] : 0.f;
    }
    float op[4][4 * KI];
    load_op_quad<KI>(op, vrole ? a.opA_rm : a.opB_rm, Kp, row0 + 4 * q, j);

    // the own rows' C^T r of block b, reverse step n (precomputed for the
    // range), into parity buffer pb: 16 bytes per copy, zero for absent columns
    auto prefetch_src = [&](int b, int n, int pb) {
        float* dst = srcS + (size_t)pb * Wa * kOwnStride;
        for (int idx = tid; idx < Wa * (kSplitRows / 4); idx += kThreads) {
            const int c = idx / (kSplitRows / 4), piece = idx % (kSplitRows / 4);
            const bool ok = c < ncol(b);
            const float* gsrc = ok ? a.src + ((size_t)(n - a.n_lo) * M + gc0(b) + c) * Kp + row0 + 4 * piece
                                   : a.src;  // a valid address for the zero fill
            cp_async16(dst + (size_t)c * kOwnStride + 4 * piece, gsrc, ok ? 16 : 0);
        }
    };
    const int NR = a.n_hi - a.n_lo;  // reverse steps of this segment
    if (vrole && NR > 0 && ncol(0) > 0) prefetch_src(0, a.n_hi - 1, 0);
    // every CTA's copies must be initialised before any peer pushes into them
    cluster.sync();

    const int nphase = 2 * NR + 1;
    for (int p = 0; p < nphase; ++p) {
        int b, k;
        if (vrole) { b = p & 1; k = (p - b) >> 1; }
        else { b = (p & 1) ^ 1; k = (p - 1 - b) >> 1; }
        const bool work = k >= 0 && k < NR && ncol(b) > 0;
        const int n = a.n_hi - 1 - k;
        float* Xb = X + (size_t)b * Wa * Kp;
        float* ownb = own + (size_t)b * Wa * kOwnStride;
        float* compb = comp + (size_t)b * Wa * kOwnStride;
        if (vrole) {
            // this phase's source term (copied during the previous phase into
            // parity buffer p & 1), then the next phase's copies into the other
            // buffer (read last in phase p - 1, which a cluster barrier has closed)
            cp_async_wait_all();
            __syncthreads();
            const int b2 = (p + 1) & 1, k2 = (p + 1 - b2) >> 1;
            if (k2 < NR && ncol(b2) > 0) prefetch_src(b2, a.n_hi - 1 - k2, (p + 1) & 1);
            if (work) {
                // half A: lamV <- lamV + dt Asv^T lamS + 2 C^T r^{n+1}
                split_phase<KI, false, false, true>(cluster, op, Xb, ownb, compb, gown, gown, Xb, dt, Wa, Kp,
                                                    row0, H, peer0, q, j, warp, lane, nullptr, Kown, ncol(b),
                                                    srcS + (size_t)(p & 1) * Wa * kOwnStride);
            }
        } else if (work) {
            // the block's df/dT table every kAdjTab of its steps
            if (k % kAdjTab == 0) {
                for (int idx = tid; idx < kAdjTab * ncol(b); idx += kThreads) {
                    const int i = idx / ncol(b), c = idx % ncol(b);
                    if (n - i >= a.n_lo)
                        dfT[(b * kAdjTab + i) * Wa + c] =
                            wavelet_dT_eval<float>(a.wavelet, (long long)a.n0 + n - i, a.dt, Tcol[b * Wa + c]);
                }
                __syncthreads();
            }
            // half B: lamS <- lamS + dt Avs^T lamV (the new lamV of block b)
            split_phase<KI, false, false>(cluster, op, Xb, ownb, compb, gown, gown, Xb, dt, Wa, Kp, row0, H,
                                          peer0, q, j, warp, lane, nullptr, Kown, ncol(b));
            // period gradient of step n over this slab's rows of the same new
            // lamV: dt (g_slab . a_V[:, c]) df/dT(t_n; T_c), fixed order
            const float* dfn = dfT + (b * kAdjTab + (k % kAdjTab)) * Wa;
            for (int c = warp; c < ncol(b); c += kSplitWarps) {
                const float* av = Xb + (size_t)c * Kp + row0;
                float sg = gown[lane] * av[lane];
                sg = __fmaf_rn(gown[lane + 32], av[lane + 32], sg);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
                if (lane == 0) gTacc[b * Wa + c] = __fmaf_rn(dt * sg, dfn[c], gTacc[b * Wa + c]);
            }
        }
        cluster.sync();
    }

    // ---- write back the owned rows, carries and the period-gradient partials
    float* out = vrole ? a.lamV : a.lamS;
    float* cout_ = vrole ? a.compV : a.compS;
    int bad = 0;
    for (int b = 0; b < 2; ++b) {
        for (int idx = tid; idx < ncol(b) * kSplitRows; idx += kThreads) {
            const int c = idx / kSplitRows, rl = idx % kSplitRows, row = row0 + rl;
            if (row < Kown) {
                const float x = own[(size_t)b * Wa * kOwnStride + c * kOwnStride + rl];
                out[(size_t)(gc0(b) + c) * Kown + row] = x;
                cout_[(size_t)(gc0(b) + c) * Kown + row] = comp[(size_t)b * Wa * kOwnStride + c * kOwnStride + rl];
                bad |= !is_finite(x);
            }
        }
        for (int c = tid; c < ncol(b); c += kThreads) a.gTpart[(size_t)crank * M + gc0(b) + c] = gTacc[b * Wa + c];
    }
    bad = __syncthreads_or(bad);
    if (bad && tid == 0 && a.status) atomicCAS(a.status, 0, 6 /* ROM_E_NONFINITE */);
}

}  // namespace romk
