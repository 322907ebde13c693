// Split-role, two-block pipelined cluster kernel for the rank-2 leapfrog (FP32).
//
// Sec. 3.1's leapfrog makes every half-step depend on the previous one, so a
// single column block keeps only half of a cluster busy if velocity and stress
// rows live on different CTAs.  This kernel gives each cluster TWO independent
// column blocks A and B (columns are independent realizations, Sec. 2.4) and
// runs them half a step apart:
//
//   phase p   V-role CTAs: V(A)^{n+1} = V(A)^n + dt (Avs S(A)^n + g f_n^T)   (p even)
//                          V(B)^{n+1}                                        (p odd)
//             S-role CTAs: S(B)^{n}   = S(B)^{n-1} + dt Asv V(B)^{n}          (p even)
//                          S(A)^{n+1} = S(A)^n + dt Asv V(A)^{n+1}            (p odd)
//
// so both roles work in every phase.  The cluster has 2H CTAs (H = Kp / 64):
// CTA s < H holds rows [64 s, 64 s + 64) of Avs in registers and owns those
// rows of V for both blocks; CTA H + s holds the same rows of Asv and owns
// those rows of S.  Each CTA keeps the full operand of both blocks (S for the
// velocity role, V for the stress role) in shared memory; after its epilogue a
// warp pushes its freshly updated 8 x 4 tile straight into the other role's
// operand copies through distributed shared memory (every lane carries one
// 16-byte piece to one or two peers), overlapping the transfer with the next
// column group's products.  One cluster barrier per phase publishes the pushes.
//
// Register tiling: thread (row quad q, chunk j) holds Avs/Asv rows 4q..4q+3 at
// k = 64 i + 4 j + t (i < KI, t < 4): every 16-byte shared load of the operand
// feeds 16 FMAs.  A butterfly reduce-scatter over the 16 chunk lanes leaves
// each lane one (row, column) sum for the fused epilogue: the Ricker forcing
// g f_n^T (Sec. 2.2, 3.2), the Kahan-compensated update, the push.  Receiver
// traces y = C V (Sec. 4.5.2) are computed by the stress role, which holds the
// full new V.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "rank2_simt.cuh"
#include "rom_internal.h"

namespace romk {

constexpr int kSplitRows = 64;   // rows of one operator per CTA
constexpr int kOwnStride = 72;   // padded column stride of the own-row buffers
constexpr int kSplitCB = 4;      // columns per register group
constexpr int kSplitWarps = kThreads / 32;

struct SplitSmem {
    size_t X, own, comp, C, f, T, Tpre, g, total;
};

__host__ __device__ inline SplitSmem split_smem_layout(int Wa, int Kp, int rpc) {
    SplitSmem s{};
    size_t o = 0;
    s.X = o;    o += align16((size_t)2 * Wa * Kp * sizeof(float));
    s.own = o;  o += align16((size_t)2 * Wa * kOwnStride * sizeof(float));
    s.comp = o; o += align16((size_t)2 * Wa * kOwnStride * sizeof(float));
    s.C = o;    o += align16((size_t)rpc * Kp * sizeof(float));
    s.f = o;    o += align16((size_t)2 * Wa * sizeof(float));
    s.T = o;    o += align16((size_t)2 * Wa * sizeof(float));
    s.Tpre = o; o += align16((size_t)2 * Wa * 2 * sizeof(double));
    s.g = o;    o += align16((size_t)kSplitRows * sizeof(float));
    s.total = o;
    return s;
}

template <int KI>
__device__ __forceinline__ void load_op_quad(float (&op)[4][4 * KI], const float* __restrict__ A,
                                             int Kp, int row, int j) {
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
#pragma unroll
        for (int i = 0; i < KI; ++i) {
            float x[4];
            load4_ro(A + (size_t)(row + rr) * Kp + 64 * i + 4 * j, x);
#pragma unroll
            for (int t = 0; t < 4; ++t) op[rr][4 * i + t] = x[t];
        }
    }
}

// One phase of one role on block b: own rows += dt (op . X_b [+ g f^T] [+ Xref]),
// pushing every finished 8 x 4 warp tile to the H peer CTAs of the other role.
// With XR, Xref points at block b's first column of the role's reduced
// reference state (Krows x columns); each lane fetches its epilogue's value
// before the products.  XR is a template flag so that runs without the term
// compile to exactly the code they had without it.  ADJ (the reverse-time
// adjoint's half A): own rows += dt (op . X_b) + 2 C_own^T r, with asrc
// block b's C_own^T r for this step ([Wa][kOwnStride], precomputed).
template <int KI, bool FORCED, bool XR, bool ADJ = false>
__device__ __forceinline__ void split_phase(cg::cluster_group& cluster, const float (&op)[4][4 * KI],
                                            const float* __restrict__ X, float* __restrict__ own,
                                            float* __restrict__ comp, const float* __restrict__ gown,
                                            const float* __restrict__ fcol, float* remote_X_b,
                                            const float dt, const int Wa, const int Kp,
                                            const int row0, const int H, const int peer0,
                                            const int q, const int j, const int warp,
                                            const int lane, const float* __restrict__ Xref,
                                            const int Krows, const int ncol,
                                            const float* __restrict__ asrc = nullptr) {
    constexpr int CB = kSplitCB;
    for (int c0 = 0; c0 < Wa; c0 += CB) {
        float xr = 0.f;
        if constexpr (XR) {
            // Xref is null for a role whose part of the term is not given
            const int si = rs16_slot<4 * CB>(j);
            const int rl = 4 * q + si / CB, c = c0 + si % CB;
            if (Xref && c < ncol && row0 + rl < Krows) xr = Xref[(size_t)c * Krows + row0 + rl];
        }
        float acc[4][CB];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int cc = 0; cc < CB; ++cc) acc[r][cc] = 0.f;
#pragma unroll
        for (int i = 0; i < KI; ++i) {
            float x[CB][4];
#pragma unroll
            for (int cc = 0; cc < CB; ++cc) load4(X + (size_t)(c0 + cc) * Kp + 64 * i + 4 * j, x[cc]);
#pragma unroll
            for (int t = 0; t < 4; ++t)
#pragma unroll
                for (int cc = 0; cc < CB; ++cc)
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        acc[r][cc] = __fmaf_rn(op[r][4 * i + t], x[cc][t], acc[r][cc]);
        }
        float v[4 * CB];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int cc = 0; cc < CB; ++cc) v[r * CB + cc] = acc[r][cc];
        int vi;
        bool active;
        const float tot = reduce_scatter16<float, 4 * CB>(v, j, vi, active);
        {
            const int rl = 4 * q + vi / CB;
            const int c = c0 + vi % CB;
            float inc = tot;
            if constexpr (ADJ) {
                const float src = asrc[c * kOwnStride + rl];
                inc = __fmaf_rn(tot, dt, 2.f * src);
            } else {
                if (FORCED) inc = __fmaf_rn(gown[rl], fcol[c], inc);
                if constexpr (XR) inc = inc + xr;
                inc = inc * dt;
            }
            float* yp = own + c * kOwnStride + rl;
            *yp = kahan_add(*yp, inc, comp[c * kOwnStride + rl]);
        }
        __syncwarp();
        // this warp's tile: rows 8 warp .. 8 warp + 7, columns c0 .. c0 + 3, as
        // eight 16-byte pieces; lane L carries piece L % 8 to peers L/8, L/8 + 4
        {
            const int piece = lane & 7, cc = piece >> 1, half = piece & 1;
            const int c = c0 + cc;
            const int rloc = 8 * warp + 4 * half;
            const float4 val = *reinterpret_cast<const float4*>(own + c * kOwnStride + rloc);
            float4* dst_local = reinterpret_cast<float4*>(remote_X_b + (size_t)c * Kp + row0 + rloc);
            for (int d = lane >> 3; d < H; d += 4) {
                float4* dst = cluster.map_shared_rank(dst_local, peer0 + d);
                *dst = val;
            }
        }
    }
}

// One stage of a 32-lane reduce-scatter of 16 values: lanes with bit `o`
// set keep the upper H entries, the others the lower H, each adding its
// partner's copy of the entries it keeps.
template <int H>
__device__ __forceinline__ void rs32_stage(float (&v)[16], int lane, int o) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float send = up ? v[i] : v[i + H];
        const float keep = up ? v[i + H] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
}

// Receiver traces y = C V^{n+1} of one block (Sec. 4.5.2): out[c R + jj] for
// this CTA's nj receiver rows Cown (row-major, Kp wide) and the nc columns of
// the new V in Xb (column-major, Kp rows).  A warp takes a tile of 4
// receivers x 4 columns over the whole K: each lane sums 4-wide stripes of k
// into 16 independent accumulators, then a 32-lane reduce-scatter (fixed
// order) leaves entry lane / 2 of the tile in lanes 2e and 2e + 1.
__device__ __forceinline__ void split_traces(const float* __restrict__ Cown, const float* __restrict__ Xb,
                                             int Kp, int nj, int nc, int warp, int lane,
                                             float* __restrict__ out, int R) {
    const int tcn = (nc + 3) >> 2;
    const int ntile = ((nj + 3) >> 2) * tcn;
    for (int t = warp; t < ntile; t += kSplitWarps) {
        const int tj = t / tcn;
        const int j0 = 4 * tj, c0 = 4 * (t - tj * tcn);
        float acc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = 0.f;
#pragma unroll 1
        for (int k = 4 * lane; k < Kp; k += 128) {
            float cv[4][4], xv[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                load4(Cown + (size_t)min(j0 + u, nj - 1) * Kp + k, cv[u]);
                load4(Xb + (size_t)min(c0 + u, nc - 1) * Kp + k, xv[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[4 * u + w] = __fmaf_rn(cv[u][q], xv[w][q], acc[4 * u + w]);
        }
        rs32_stage<8>(acc, lane, 16);
        rs32_stage<4>(acc, lane, 8);
        rs32_stage<2>(acc, lane, 4);
        rs32_stage<1>(acc, lane, 2);
        acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
        const int e = lane >> 1, jj = j0 + (e >> 2), c = c0 + (e & 3);
        if ((lane & 1) == 0 && jj < nj && c < nc) out[(size_t)c * R + jj] = acc[0];
    }
}

// The split kernel's work on one item: column blocks A = [gc0_0, gc0_0 + nc0)
// and B = [gc0_0 + Wv, gc0_0 + Wv + nc1) of the caller's arrays, operator
// `gop` of the table (MODE 2) or the launch's own operator.
template <int KI, int MODE>
__device__ __forceinline__ void split_body(cg::cluster_group& cluster, const Rank2Args& a,
                                           const GroupOp* gop, const int gc0_0, const int nc0,
                                           const int nc1) {
    constexpr bool XR = MODE == 1;
    constexpr bool GROUPED = MODE == 2;
    const int cs = (int)cluster.num_blocks();
    const int H = cs / 2;
    const int crank = (int)cluster.block_rank();
    const bool vrole = crank < H;
    const int s = vrole ? crank : crank - H;  // row slab
    const int row0 = s * kSplitRows;
    const int peer0 = vrole ? H : 0;          // first CTA of the other role
    const int Wa = a.Wa, Kp = a.Kp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = lane & 15;
    const int q = warp * 2 + (lane >> 4);     // row quad
    const float dt = (float)a.dt;

    extern __shared__ __align__(16) unsigned char smem[];
    const SplitSmem L = split_smem_layout(Wa, Kp, a.rpc);
    float* X = reinterpret_cast<float*>(smem + L.X);        // [2][Wa][Kp]
    float* own = reinterpret_cast<float*>(smem + L.own);    // [2][Wa][72]
    float* comp = reinterpret_cast<float*>(smem + L.comp);  // [2][Wa][72]
    float* Cown = reinterpret_cast<float*>(smem + L.C);     // [rpc][Kp]
    float* fcol = reinterpret_cast<float*>(smem + L.f);     // [2][Wa]
    float* Tcol = reinterpret_cast<float*>(smem + L.T);     // [2][Wa]
    double* Tpre = reinterpret_cast<double*>(smem + L.Tpre);  // [2][Wa][-1.5 T, pi / T]
    float* gown = reinterpret_cast<float*>(smem + L.g);     // [64]

    // column ranges of the two blocks, kept in scalars so that runtime block
    // indices do not force a local-memory array
    const int gc0_1 = gc0_0 + a.Wv;
    auto gc0 = [&](int b) { return b ? gc0_1 : gc0_0; };
    auto ncol = [&](int b) { return b ? nc1 : nc0; };

    const float* Vin = static_cast<const float*>(a.V);
    const float* Sin = static_cast<const float*>(a.S);
    const int Kown = vrole ? a.Kv : a.Ks;             // rows of the owned state
    const float* own_in = vrole ? Vin : Sin;
    const float* comp_in = static_cast<const float*>(vrole ? a.compV : a.compS);

    // ---- initial state.  V role: operand = full S^0, own = V^0 rows.
    //      S role: operand is filled by the first V pushes; own = S^0 rows.
    for (int idx = tid; idx < 2 * Wa * Kp; idx += kThreads) {
        const int b = idx / (Wa * Kp);
        const int rem = idx - b * Wa * Kp;
        const int c = rem / Kp, k = rem - (rem / Kp) * Kp;
        float v = 0.f;
        if (vrole && c < ncol(b) && k < a.Ks) v = Sin[(size_t)(gc0(b) + c) * a.Ks + k];
        X[idx] = v;
    }
    for (int idx = tid; idx < 2 * Wa * kOwnStride; idx += kThreads) {
        const int b = idx / (Wa * kOwnStride);
        const int rem = idx - b * Wa * kOwnStride;
        const int c = rem / kOwnStride, rl = rem % kOwnStride, row = row0 + rl;
        const bool ok = rl < kSplitRows && c < ncol(b) && row < Kown;
        own[idx] = ok ? own_in[(size_t)(gc0(b) + c) * Kown + row] : 0.f;
        comp[idx] = (ok && comp_in) ? comp_in[(size_t)(gc0(b) + c) * Kown + row] : 0.f;
    }
    const float* Cp = static_cast<const float*>(GROUPED ? gop->C_p : a.C_p);
    if (!vrole) {
        for (int idx = tid; idx < a.rpc * Kp; idx += kThreads) {
            const int jj = idx / Kp, k = idx % Kp, jr = s * a.rpc + jj;
            Cown[idx] = (Cp && jr < a.R) ? Cp[(size_t)jr * Kp + k] : 0.f;
        }
    }
    if (tid < kSplitRows) gown[tid] = vrole ? static_cast<const float*>(GROUPED ? gop->g_p : a.g_p)[row0 + tid] : 0.f;
    for (int idx = tid; idx < 2 * Wa; idx += kThreads) {
        const int b = idx / Wa, c = idx % Wa;
        Tcol[idx] = (a.Tper && c < ncol(b)) ? static_cast<const float*>(a.Tper)[gc0(b) + c] : 1.f;
        Tpre[2 * idx] = -1.5 * (double)Tcol[idx];
        Tpre[2 * idx + 1] = 3.14159265358979323846 / (double)Tcol[idx];
    }
    __syncthreads();
    // forcing of the first V phase (block A, step 0)
    if (vrole) {
        for (int c = tid; c < Wa; c += kThreads) {
            float f = 0.f;
            if (c < ncol(0)) {
                if (a.ftab) f = static_cast<const float*>(a.ftab)[gc0(0) + c];
                else if (a.Tper) f = wavelet_eval_pre(a.wavelet, (long long)a.n0, a.dt, Tpre[2 * c], Tpre[2 * c + 1]);
            }
            fcol[c] = f;
        }
    }

    float op[4][4 * KI];
    load_op_quad<KI>(op, static_cast<const float*>(vrole ? (GROUPED ? gop->Avs_rm : a.Avs_rm)
                                                         : (GROUPED ? gop->Asv_rm : a.Asv_rm)),
                     Kp, row0 + 4 * q, j);
    // every CTA's copies must be initialised before any peer pushes into them
    cluster.sync();

    float* traces = static_cast<float*>(a.traces);
    const float* Xrole = static_cast<const float*>(vrole ? a.Xv : a.Xs);
    const int N = a.nsteps;
    const int nphase = 2 * N + 1;
    for (int p = 0; p < nphase; ++p) {
        int b, n;
        if (vrole) { b = p & 1; n = (p - b) >> 1; }
        else { b = (p & 1) ^ 1; n = (p - 1 - b) >> 1; }
        const bool work = n >= 0 && n < N && ncol(b) > 0;
        if (work) {
            float* Xb = X + (size_t)b * Wa * Kp;
            float* ownb = own + (size_t)b * Wa * kOwnStride;
            float* compb = comp + (size_t)b * Wa * kOwnStride;
            const float* Xr = Xrole ? Xrole + (size_t)gc0(b) * Kown : nullptr;
            if (vrole) {
                split_phase<KI, true, XR>(cluster, op, Xb, ownb, compb, gown, fcol + b * Wa, Xb, dt, Wa,
                                          Kp, row0, H, peer0, q, j, warp, lane, Xr, Kown, ncol(b));
            } else {
                split_phase<KI, false, XR>(cluster, op, Xb, ownb, compb, gown, fcol, Xb, dt, Wa, Kp,
                                           row0, H, peer0, q, j, warp, lane, Xr, Kown, ncol(b));
                // receiver traces of V^{n+1} (the full new V of block b is in Xb)
                if (traces && ((n + 1) % a.r) == 0) {
                    const int rec = (n + 1) / a.r - 1;
                    const int nj = min(a.rpc, a.R - s * a.rpc);  // this CTA's receivers
                    split_traces(Cown, Xb, Kp, nj > 0 ? nj : 0, ncol(b), warp, lane,
                                 traces + ((size_t)rec * a.Mtot + gc0(b)) * a.R + s * a.rpc, a.R);
                }
            }
        }
        // forcing for this role's next phase (V role: block b' = (p+1)&1, step n')
        if (vrole) {
            const int b2 = (p + 1) & 1;
            const int n2 = (p + 1 - b2) >> 1;
            if (n2 < N) {
                for (int c = tid; c < Wa; c += kThreads) {
                    float f = 0.f;
                    if (c < ncol(b2)) {
                        if (a.ftab) f = static_cast<const float*>(a.ftab)[(size_t)n2 * a.Mtot + gc0(b2) + c];
                        else if (a.Tper) {
                            const double* tp = Tpre + 2 * (b2 * Wa + c);
                            f = wavelet_eval_pre(a.wavelet, (long long)a.n0 + n2, a.dt, tp[0], tp[1]);
                        }
                    }
                    fcol[b2 * Wa + c] = f;
                }
            }
        }
        cluster.sync();
    }

    // ---- write back the owned rows and carries
    float* out = static_cast<float*>(vrole ? a.V : a.S);
    float* cout_ = static_cast<float*>(vrole ? a.compV : a.compS);
    int bad = 0;
    for (int b = 0; b < 2; ++b) {
        for (int idx = tid; idx < ncol(b) * kSplitRows; idx += kThreads) {
            const int c = idx / kSplitRows, rl = idx % kSplitRows, row = row0 + rl;
            if (row < Kown) {
                const float x = own[(size_t)b * Wa * kOwnStride + c * kOwnStride + rl];
                out[(size_t)(gc0(b) + c) * Kown + row] = x;
                if (cout_) cout_[(size_t)(gc0(b) + c) * Kown + row] =
                    comp[(size_t)b * Wa * kOwnStride + c * kOwnStride + rl];
                bad |= !is_finite(x);
            }
        }
    }
    bad = __syncthreads_or(bad);
    if (bad && tid == 0 && a.status) atomicCAS(a.status, 0, 6 /* ROM_E_NONFINITE */);
}


// MODE: 0 plain; 1 adds the reduced reference state (a.Xv / a.Xs); 2 is the
// rank-3 grouped launch (operator table a.group).  A template parameter, so
// that each instance compiles to exactly the code its runs need.
template <int KI, int MODE>
__global__ void __launch_bounds__(kThreads, 1) rank2_split_kernel(const Rank2Args a) {
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    // rank-3 grouped launch: operator `job` of the table, cluster `clu` of it
    const int job = MODE == 2 ? (int)(blockIdx.x / cs) / a.group_cpj : 0;
    const int clu = MODE == 2 ? (int)(blockIdx.x / cs) % a.group_cpj : (int)(blockIdx.x / cs);
    const GroupOp* gop = MODE == 2 ? a.group + job : nullptr;
    const int gc0_0 = a.col_base + job * a.M + (2 * clu) * a.Wv;
    const int nr0 = a.M - (2 * clu) * a.Wv, nr1 = nr0 - a.Wv;
    const int nc0 = nr0 < 0 ? 0 : (nr0 > a.Wv ? a.Wv : nr0);
    const int nc1 = nr1 < 0 ? 0 : (nr1 > a.Wv ? a.Wv : nr1);
    split_body<KI, MODE>(cluster, a, gop, gc0_0, nc0, nc1);
}

}  // namespace romk
