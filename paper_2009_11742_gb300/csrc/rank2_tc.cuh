// Tensor-core (tcgen05) persistent rank-2 leapfrog with split-precision
// products (TF32x3, BF16x3, plain BF16) for reduced operators too large to
// stay on chip (K up to 1024).
//
// Work split.  A cluster of CS = Kp / 128 CTAs owns one block of W state
// columns for the whole run; CTA c owns rows [128 c, 128 c + 128) of V and S.
// A half-step is D = A_c . X (A_c: the CTA's 128-row slab of Avs or Asv, X:
// the full S or V of the block), an M = 128, N = W, K = Kp product that
// tcgen05.mma accumulates in tensor memory over Kp / KC k-chunks:
//   * warp 0 (one lane) streams each k-chunk of every operand term into a
//     ring of shared-memory stages with bulk copies (cp.async.bulk); operator
//     tiles are pre-split and pre-swizzled at rom_create time, state tiles are
//     written pre-split and pre-swizzled by the previous half-step's epilogue;
//   * warp 1 (one lane) issues the split products of each chunk
//     (e.g. A_hi X_hi + A_hi X_lo + A_lo X_hi for TF32x3) and releases the
//     stage with tcgen05.commit;
//   * all eight warps then read D from tensor memory (tcgen05.ld), fuse the
//     point-source forcing g f^T (Sec. 2.2, 3.2) and the Kahan-compensated
//     FP32 state update, write the new rows, and write them split and
//     swizzled into the exchange buffer the next half-step streams;
//   * a cluster barrier (after a generic->async proxy fence) publishes the
//     exchange buffer; receiver traces y = C V (Sec. 4.5.2) are taken by the
//     stress half-step from the published V.
// Every mbarrier wait is bounded; a timeout is made cluster-uniform at the
// next barrier, all CTAs stop together, drain their copies and free TMEM.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "rom_internal.h"
#include "tc_common.cuh"

namespace romk {

namespace cg = cooperative_groups;

constexpr int kTcThreads = 320;     // 10 warps: 0 producer, 1 MMA, 2..9 readout / epilogue
constexpr int kTcReadWarp0 = 2;
constexpr int kTcReadWarps = 8;
constexpr int kTcRows = 128;         // MMA M: rows per CTA
constexpr uint32_t kTileRowBytes = 128;  // K extent of one tile row (SW128)
constexpr uint32_t kATileBytes = kTcRows * kTileRowBytes;  // 16 KB

// Precision schemes: operand terms and the (a, x) term pairs multiplied.
template <int P> struct TcScheme;
template <> struct TcScheme<ROM_TF32X3> {
    static constexpr bool kTF32 = true;
    static constexpr int NA = 2, NX = 2, NP = 3;
    static constexpr int KC = 32;  // k per chunk (128 B of tf32)
    __device__ static constexpr int pa(int i) { return i == 2 ? 1 : 0; }
    __device__ static constexpr int px(int i) { return i == 1 ? 1 : 0; }
};
template <> struct TcScheme<ROM_BF16X3> {
    static constexpr bool kTF32 = false;
    static constexpr int NA = 3, NX = 2, NP = 5;
    static constexpr int KC = 64;  // k per chunk (128 B of bf16)
    // pairs (0,0) (0,1) (1,0) (1,1) (2,0)
    __device__ static constexpr int pa(int i) { return i < 2 ? 0 : (i < 4 ? 1 : 2); }
    __device__ static constexpr int px(int i) { return (i == 1 || i == 3) ? 1 : 0; }
};
template <> struct TcScheme<ROM_BF16> {
    static constexpr bool kTF32 = false;
    static constexpr int NA = 1, NX = 1, NP = 1;
    static constexpr int KC = 64;
    __device__ static constexpr int pa(int) { return 0; }
    __device__ static constexpr int px(int) { return 0; }
};

// Bytes of one k-chunk of one operator term for one 128-row tile / of one
// exchange term for W columns.
template <int P>
__host__ __device__ inline uint32_t tc_xtile_bytes(int W) { return (uint32_t)W * kTileRowBytes; }

template <int P>
__host__ __device__ inline size_t tc_stage_bytes(int W) {
    return (size_t)TcScheme<P>::NA * kATileBytes + (size_t)TcScheme<P>::NX * W * kTileRowBytes;
}

// Shared memory: stages (1024-aligned), then mbarriers and small arrays.
template <int P>
__host__ __device__ inline size_t tc_smem_bytes(int W, int stages, int rpc, int Kp) {
    size_t o = 1024;  // alignment slack
    o += (size_t)stages * tc_stage_bytes<P>(W);
    o += 8 * (2 * stages + 5);        // full[], empty[], dready[2], dempty[2], drain
    o += 32;                          // tmem slot, flags, chunk counter
    o += (size_t)W * 4 * 2;           // fcol, Tcol
    o += (size_t)kTcRows * 4;         // g rows
    o += 64;
    return o;
}

// Address in an exchange buffer (one term) of element (k = state row, j = column).
template <int P>
__device__ __forceinline__ size_t tc_xoffset(int k, int j, int W) {
    constexpr int KC = TcScheme<P>::KC;
    constexpr int ES = TcScheme<P>::kTF32 ? 4 : 2;
    const int kc = k / KC, kk = k - kc * KC;
    const int chunk16 = (kk * ES) >> 4, within = (kk * ES) & 15;
    return (size_t)kc * W * kTileRowBytes + sw128_offset((uint32_t)j, (uint32_t)chunk16) + within;
}

// Write the split terms of value x at (k, j) into the NX exchange terms.
template <int P>
__device__ __forceinline__ void tc_store_split(void* const* Xterms, size_t term_stride, int k, int j,
                                               int W, float x) {
    const size_t off = tc_xoffset<P>(k, j, W);
    unsigned char* base = static_cast<unsigned char*>(Xterms[0]);
    if constexpr (TcScheme<P>::kTF32) {
        float hi, lo;
        split_tf32_rn(x, hi, lo);
        *reinterpret_cast<float*>(base + off) = hi;
        *reinterpret_cast<float*>(base + term_stride + off) = lo;
    } else if constexpr (TcScheme<P>::NX == 2) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(base + term_stride + off) = l;
    } else {
        *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(x);
    }
}

template <int P, int W>
__global__ void __launch_bounds__(kTcThreads, 1) rank2_tc_kernel(const TcArgs a) {
    using Sch = TcScheme<P>;
    constexpr int NA = Sch::NA, NX = Sch::NX, NP = Sch::NP, KC = Sch::KC;
    constexpr int WH = W / 2;  // columns per readout warp
    constexpr uint32_t NCOLS = 2 * W <= 128 ? 128u : 256u;  // two accumulators of W columns
    cg::cluster_group cluster = cg::this_cluster();
    const int CS = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int blk = blockIdx.x / CS;
    const int Kp = a.Kp, STAGES = a.stages;
    const int col0 = blk * W;
    const int ncol = min(W, a.M - col0);
    const int row0 = crank * kTcRows;
    const int NKC = Kp / KC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float dt = (float)a.dt;
    const long long limit = a.spin_limit;
    const bool reader = warp >= kTcReadWarp0;
    const int quad = warp & 3;                            // TMEM lane quadrant of this warp
    const int chalf = (warp - kTcReadWarp0) / 4;          // column half of a readout warp
    const int rl = 32 * quad + lane;                      // row (within the slab) of a reader

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const size_t stage_bytes = tc_stage_bytes<P>(W);
    unsigned char* tail = smem + (size_t)STAGES * stage_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(tail);
    uint64_t* empty = full + STAGES;
    uint64_t* dready = empty + STAGES;   // [2]: an accumulator holds a finished chunk
    uint64_t* dempty = dready + 2;       // [2]: the readers have drained it
    uint64_t* drain = dempty + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* abort_all = reinterpret_cast<volatile int*>(tslot + 2);
    // abort flag as published for the cluster-wide decision: written after
    // the half-step's last wait, read by the peers after the barrier
    volatile int* abort_pub = reinterpret_cast<volatile int*>(tslot + 3);
    long long* consumed = reinterpret_cast<long long*>(tslot + 4);
    float* fcol = reinterpret_cast<float*>(tslot + 6);
    float* Tcol = fcol + W;
    float* grow = Tcol + W;

    if (tid == 0) {
        *abort_flag = 0;
        *abort_all = 0;
        *abort_pub = 0;
        for (int s = 0; s < STAGES; ++s) { mbarrier_init(&full[s], 1); mbarrier_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbarrier_init(&dready[b], 1); mbarrier_init(&dempty[b], kTcReadWarps); }
        mbarrier_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) { tmem_alloc(tslot, NCOLS); tmem_relinquish(); }
    for (int c = tid; c < W; c += kTcThreads) Tcol[c] = (a.Tper && c < ncol) ? a.Tper[col0 + c] : 1.f;
    if (tid < kTcRows) grow[tid] = a.g_p[row0 + tid];

    // ---- initial exchange tiles of S^0 (own rows) and the step-0 forcing
    const size_t xterm = (size_t)Kp * W * (Sch::kTF32 ? 4 : 2);  // bytes of one exchange term
    unsigned char* const Xblk0 = static_cast<unsigned char*>(a.X[0]) + (size_t)blk * NX * xterm;
    unsigned char* const Xblk1 = static_cast<unsigned char*>(a.X[1]) + (size_t)blk * NX * xterm;
    for (int idx = tid; idx < kTcRows * W; idx += kTcThreads) {
        const int j = idx / kTcRows, r = idx % kTcRows, row = row0 + r;
        const float x = (j < ncol && row < a.Ks) ? a.S[(size_t)(col0 + j) * a.Ks + row] : 0.f;
        void* xt[1] = {Xblk0};
        tc_store_split<P>(xt, xterm, row, j, W, x);
    }
    __syncthreads();
    for (int c = tid; c < W; c += kTcThreads) {
        float f = 0.f;
        if (c < ncol) {
            if (a.ftab) f = a.ftab[col0 + c];
            else if (a.Tper) f = wavelet_eval(a.wavelet, a.n0, a.dt, Tcol[c]);
        }
        fcol[c] = f;
    }
    fence_proxy_async_global();
    tc_fence_before();
    cluster.sync();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t idesc = mma_idesc(Sch::kTF32 ? kFmtTF32 : kFmtBF16, kTcRows, (uint32_t)W);
    const uint32_t xtile = tc_xtile_bytes<P>(W);
    const uint32_t chunk_bytes = NA * kATileBytes + NX * xtile;

    long long it_prod = 0, it_mma = 0, it_rd = 0;  // chunk counters of producer / MMA / readers
    // producer / MMA counters also as (ring stage, uses of that stage),
    // advanced by one so that the per-chunk loops do no 64-bit division
    int s_prod = 0, s_mma = 0;
    uint32_t u_prod = 0, u_mma = 0;
    const int N = a.nsteps;
    for (int n = 0; n < N && !*abort_all; ++n) {
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            const unsigned char* Aop = static_cast<const unsigned char*>(half ? a.Aop[1] : a.Aop[0]) +
                                       (size_t)crank * NKC * NA * kATileBytes;
            const unsigned char* Xsrc = half ? Xblk1 : Xblk0;
            float acc[WH];
#pragma unroll
            for (int i = 0; i < WH; ++i) acc[i] = 0.f;
            bool have = false;
            if (warp == 0) {
                if (lane == 0 && !*abort_flag) {
                    // ---- producer: stream every k-chunk's terms into the stage ring
                    for (int kc = 0; kc < NKC; ++kc) {
                        const int s = s_prod;
                        const uint32_t use = u_prod;
                        if (use > 0 && !mbarrier_wait(&empty[s], (use - 1) & 1, limit, abort_flag)) break;
                        unsigned char* st = smem + (size_t)s * stage_bytes;
                        mbarrier_arrive_expect_tx(&full[s], chunk_bytes);
                        for (int t = 0; t < NA; ++t)
                            bulk_g2s(st + t * kATileBytes, Aop + ((size_t)kc * NA + t) * kATileBytes,
                                     kATileBytes, &full[s]);
                        for (int t = 0; t < NX; ++t)
                            bulk_g2s(st + NA * kATileBytes + t * xtile,
                                     Xsrc + (size_t)t * xterm + (size_t)kc * xtile, xtile, &full[s]);
                        ++it_prod;
                        if (++s_prod == STAGES) { s_prod = 0; ++u_prod; }
                    }
                }
                __syncwarp();
            } else if (warp == 1) {
                if (lane == 0 && !*abort_flag) {
                    // ---- MMA issue: each chunk's split products into accumulator (chunk & 1)
                    for (int kc = 0; kc < NKC; ++kc) {
                        const int s = s_mma;
                        const uint32_t use = u_mma;
                        const int b = (int)(it_mma & 1);
                        const uint32_t ub = (uint32_t)(it_mma >> 1);
                        if (!mbarrier_wait(&full[s], use & 1, limit, abort_flag)) break;
                        if (ub > 0 && !mbarrier_wait(&dempty[b], (ub - 1) & 1, limit, abort_flag)) break;
                        tc_fence_after();
                        const uint32_t sA = cvta_shared(smem + (size_t)s * stage_bytes);
                        const uint32_t sX = sA + NA * kATileBytes;
                        const uint32_t dcol = tbase + (uint32_t)(b * W);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {  // four 32-byte K steps per 128-byte chunk
#pragma unroll
                            for (int p = 0; p < NP; ++p) {
                                const uint64_t ad = sw128_desc(sA + Sch::pa(p) * kATileBytes + 32u * ks);
                                const uint64_t xd = sw128_desc(sX + Sch::px(p) * xtile + 32u * ks);
                                mma_issue<Sch::kTF32>(dcol, ad, xd, idesc, (ks > 0 || p > 0) ? 1u : 0u);
                            }
                        }
                        mma_commit(&empty[s]);
                        mma_commit(&dready[b]);
                        ++it_mma;
                        if (++s_mma == STAGES) { s_mma = 0; ++u_mma; }
                    }
                }
                __syncwarp();
            } else if (reader) {
                // ---- readers: drain each chunk's partial products into FP32
                //      registers (round to nearest), so that the tensor core's
                //      accumulation never spans more than one chunk
                have = true;
                for (int kc = 0; kc < NKC; ++kc, ++it_rd) {
                    const int b = (int)(it_rd & 1);
                    const uint32_t ub = (uint32_t)(it_rd >> 1);
                    int gotl = 0;
                    if (lane == 0) gotl = (*abort_flag == 0) && mbarrier_wait(&dready[b], ub & 1, limit, abort_flag);
                    if (!__shfl_sync(0xffffffffu, gotl, 0)) { have = false; break; }
                    tc_fence_after();
                    const uint32_t taddr = tbase + ((uint32_t)(32 * quad) << 16) + (uint32_t)(b * W + chalf * WH);
#pragma unroll
                    for (int sl = 0; sl < WH / 32; ++sl) {
                        float v[32];
                        tmem_ld32(taddr + 32u * sl, v);
#pragma unroll
                        for (int i = 0; i < 32; ++i) acc[32 * sl + i] += v[i];
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbarrier_arrive(&dempty[b]);
                }
            }
            // ---- epilogue (readers): forcing, Kahan update, new state and its split tiles
            if (have) {
                const int row = row0 + rl;
                const int Kown = half == 0 ? a.Kv : a.Ks;
                float* Y = half == 0 ? a.V : a.S;
                float* Cy = half == 0 ? a.compV : a.compS;
                const float* Xref = half == 0 ? a.Xv : a.Xs;  // reduced reference state or null
                unsigned char* Xdst = half ? Xblk0 : Xblk1;  // V feeds the S half and vice versa
#pragma unroll
                for (int i = 0; i < WH; ++i) {
                    const int j = chalf * WH + i;
                    float y = 0.f;
                    if (j < ncol && row < Kown) {
                        const size_t gi = (size_t)(col0 + j) * Kown + row;
                        float inc = acc[i];
                        if (half == 0) inc = __fmaf_rn(grow[rl], fcol[j], inc);
                        if (Xref) inc = inc + Xref[gi];
                        inc = inc * dt;
                        float cc = Cy[gi];
                        y = kahan_add(Y[gi], inc, cc);
                        Y[gi] = y;
                        Cy[gi] = cc;
                    }
                    void* xt[1] = {Xdst};
                    tc_store_split<P>(xt, xterm, row, j, W, y);
                }
            }
            fence_proxy_async_global();
            // forcing of the next step (read by the next velocity epilogue)
            if (half == 1 && n + 1 < N) {
                for (int c = tid; c < W; c += kTcThreads) {
                    float f = 0.f;
                    if (c < ncol) {
                        if (a.ftab) f = a.ftab[(size_t)(n + 1) * a.Mtot + col0 + c];
                        else if (a.Tper) f = wavelet_eval(a.wavelet, a.n0 + n + 1, a.dt, Tcol[c]);
                    }
                    fcol[c] = f;
                }
            }
            __syncthreads();  // every wait of this half-step is over
            if (tid == 0) *abort_pub = *abort_flag;
            tc_fence_before();
            cluster.sync();
            tc_fence_after();
            // cluster-uniform abort decision from the published flags
            if (tid == 0) {
                int any = 0;
                for (int q = 0; q < CS; ++q) {
                    const int* pf = cluster.map_shared_rank(const_cast<int*>(abort_pub), q);
                    any |= *reinterpret_cast<volatile const int*>(pf);
                }
                *abort_all = any;
            }
            __syncthreads();
            if (*abort_all) break;
            // ---- receiver traces of V^{n+1} (after the velocity half is published)
            if (half == 0 && a.traces && ((n + 1) % a.r) == 0) {
                const int rec = (n + 1) / a.r - 1;
                const int npair = a.rpc * ncol;
                for (int pr = warp; pr < npair; pr += kTcThreads / 32) {
                    const int jj = pr / ncol, c = pr % ncol, jr = crank * a.rpc + jj;
                    if (jr >= a.R) continue;
                    const float* vcol = a.V + (size_t)(col0 + c) * a.Kv;
                    const float* crow = a.C_p + (size_t)jr * Kp;
                    float tacc = 0.f;
                    for (int k = lane; k < a.Kv; k += 32) tacc = __fmaf_rn(crow[k], __ldcg(vcol + k), tacc);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) tacc += __shfl_xor_sync(0xffffffffu, tacc, o);
                    if (lane == 0) a.traces[((size_t)rec * a.Mtot + col0 + c) * a.R + jr] = tacc;
                }
            }
        }
    }
    // ---- teardown: copies in flight complete, MMAs complete, TMEM freed
    if (warp == 1 && lane == 0) *consumed = it_mma;
    __syncthreads();
    if (warp == 0 && lane == 0) {
        for (long long it = *consumed; it < it_prod; ++it) {
            const int s = (int)(it % STAGES);
            mbarrier_wait(&full[s], (uint32_t)((it / STAGES) & 1), limit, abort_flag);
        }
    }
    if (warp == 1 && lane == 0) {
        mma_commit(drain);
        mbarrier_wait(drain, 0, limit, abort_flag);
    }
    if (*abort_flag && tid == 0 && a.status) atomicCAS(a.status, 0, 5 /* ROM_E_TIMEOUT */);
    tc_fence_before();
    __syncthreads();
    cluster.sync();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tbase, NCOLS);
}

}  // namespace romk
