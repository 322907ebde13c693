// Tensor-core rank-2 leapfrog with exact sliced-integer BF16 products
// (ROM_BF16S).
//
// The FP32 accumulator of tcgen05.mma does not round to nearest, so the
// split schemes of rank2_tc.cuh (TF32x3, BF16x3) carry a small bias of one
// sign in every product; over 10^4 leapfrog steps (Sec. 3.1) that bias
// dominates the error.  This scheme removes every rounding from the tensor
// core instead of splitting finer:
//   * operator row r is stored as 2^(eA_r - 7) (a0 + 2^-8 a1 + 2^-16 a2) and
//     state column j as 2^(eX_j - 7) (x0 + 2^-8 x1 + 2^-16 x2), with integer
//     digits in [-128, 128] (exact in BF16) and |A| < 2^eA_r over the row,
//     |X| < 2^eX_j over the whole column (all Kp rows of the cluster);
//   * the six digit products of weight 1, 2^-8 and 2^-16 go to four TMEM
//     accumulators: T0 = sum a0 x0 (|T0| <= Kp 2^14 <= 2^24), T1a / T1b =
//     sum a0 x1 + a1 x0 over k < 512 / k >= 512 (each <= 2^24), and
//     T2 = sum a0 x2 + a1 x1 + a2 x0.  Products of integers below 2^7 in
//     magnitude are exact, and every partial sum of T0 and T1 is an integer
//     of magnitude at most 2^24, so the tensor core computes them exactly;
//     T2 carries weight 2^-16, so whatever it rounds is below 2^-32 of the
//     result;
//   * the readers load the accumulators once per half-step and form
//     A.X = 2^(eA_r + eX_j - 14) (T0 + 2^-8 (T1a + T1b) + 2^-16 T2) in FP32
//     with round-to-nearest; the terms of weight 2^-24 and below that the
//     digits leave out are not biased either.
// The state's column exponent needs the column maximum over all rows, which
// the CTAs of a cluster agree on through distributed shared memory with one
// extra cluster barrier per half-step.  Work split, pipeline and bounded
// waits follow rank2_tc.cuh: lane 0 of warp 0 streams operator and state
// digit tiles into a ring of stages, lane 0 of warp 1 issues the MMAs, and
// then all eight warps read out, fuse the forcing g f^T (Sec. 2.2, 3.2) and
// the Kahan-compensated update, and slice the new state into the exchange
// tiles of the next half-step.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "rank2_tc.cuh"
#include "rom_internal.h"
#include "tc_common.cuh"

namespace romk {

constexpr int kTcsTerms = 3;    // digits per operand
constexpr int kTcsKC = 64;      // k per chunk (128 bytes of bf16)
constexpr int kTcsMaxCS = 8;    // CTAs per cluster (Kp <= 1024)
constexpr int kTcsThreads = 256;  // 8 warps, all read out; lane 0 of warps 0 / 1 also produce / issue MMAs
constexpr int kTcsTraceR = 64;  // receiver rows handled on chip (partial C.V per CTA)
constexpr int kTcsTStride = 132;  // padded row stride (floats) of the on-chip trace operands

// On-chip receiver traces reuse the stage ring during the epilogue: the new
// rows Ys[W][132], the CTA's slab of C, Cs[64][132], and the partial traces
// P[64][W] of this CTA's 128 rows.
__host__ __device__ inline size_t tcs_trace_scratch_bytes(int W) {
    return ((size_t)W * kTcsTStride + (size_t)kTcsTraceR * kTcsTStride + (size_t)kTcsTraceR * W) * 4;
}

// Integer digits of xs (|xs| <= 128): xs = d0 + 2^-8 d1 + 2^-16 d2 + e with
// |e| <= 2^-17 and every d in [-128, 128].  Each operation is exact in FP32:
// xs - d0 is a Sterbenz difference or has d0 = 0, and the scalings are by
// powers of two.
__host__ __device__ __forceinline__ void slice_digits(float xs, float& d0, float& d1, float& d2) {
    d0 = rintf(xs);
    const float r1 = (xs - d0) * 256.f;
    d1 = rintf(r1);
    const float r2 = (r1 - d1) * 256.f;
    d2 = rintf(r2);
}

// Exponent e with |x| < 2^e for every x of a set whose largest magnitude is
// mx (0 for an all-zero set).
__device__ __forceinline__ int bound_exponent(float mx) {
    int e = 0;
    if (mx > 0.f && isfinite(mx)) frexpf(mx, &e);
    return e;
}

// Column stride of the accumulators in tensor memory; after the four
// accumulators the new state of each readout warp (W columns in all) is
// parked between the update and the slicing.  Allocation: next power of two.
__host__ __device__ constexpr int tcs_acc_stride(int W) { return ((W + 31) / 32) * 32; }
__host__ __device__ constexpr uint32_t tcs_tmem_cols(int W) {
    return 4 * tcs_acc_stride(W) + W <= 128 ? 128u : (4 * tcs_acc_stride(W) + W <= 256 ? 256u : 512u);
}

__host__ __device__ inline size_t tcs_stage_bytes(int W) {
    return (size_t)kTcsTerms * kATileBytes + (size_t)kTcsTerms * W * kTileRowBytes;
}

__host__ __device__ inline size_t tcs_smem_bytes(int W, int stages) {
    size_t o = 1024;                                    // alignment slack
    o += (size_t)stages * tcs_stage_bytes(W);
    o += 8 * (2 * stages + 2);                          // full[], empty[], dready, drain
    o += 32;                                            // tmem slot, flags, chunk counter
    o += (size_t)W * 4 * 4;                             // fcol, Tcol, xsc, xinv
    o += (size_t)kTcRows * 4 * 3;                       // g rows, row scales of Avs and Asv
    o += (size_t)4 * W * 4;                             // column maxima per TMEM quadrant
    o += (size_t)kTcsMaxCS * W * 4;                     // block maxima of every CTA
    o += 64;
    return o;
}

// Byte offset of state element (k, j) in one digit term of an exchange block.
__device__ __forceinline__ size_t tcs_xoffset(int k, int j, int W) {
    const int kc = k / kTcsKC, kk = k - kc * kTcsKC;
    return (size_t)kc * W * kTileRowBytes + sw128_offset((uint32_t)j, (uint32_t)((kk * 2) >> 4)) +
           ((kk * 2) & 15);
}

__device__ __forceinline__ void tcs_store_digits(unsigned char* base, size_t term_stride, size_t off,
                                                 float xs) {
    float d0, d1, d2;
    slice_digits(xs, d0, d1, d2);
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(d0);
    *reinterpret_cast<__nv_bfloat16*>(base + term_stride + off) = __float2bfloat16_rn(d1);
    *reinterpret_cast<__nv_bfloat16*>(base + 2 * term_stride + off) = __float2bfloat16_rn(d2);
}

// Eight TMEM columns of this warp's 32 lanes, without waiting.
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
// Wait for outstanding tensor-memory loads; the registers pass through the
// statement so that no use of them is scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld4(uint32_t (&a)[8], uint32_t (&b)[8], uint32_t (&c)[8],
                                              uint32_t (&d)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]),
                   "+r"(a[7]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]),
                   "+r"(b[6]), "+r"(b[7]), "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3]), "+r"(c[4]),
                   "+r"(c[5]), "+r"(c[6]), "+r"(c[7]), "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]),
                   "+r"(d[4]), "+r"(d[5]), "+r"(d[6]), "+r"(d[7])
                 :
                 : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])),
                   "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])),
                   "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    tmem_ld8_nowait(taddr, r);
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

// The six digit products of one 16-deep k-step, issued from one asm block:
// d0 += a0 x0, d1 += a0 x1 + a1 x0, d2 += a0 x2 + a1 x1 + a2 x0.  The
// operands are given as the low words of their SW128 descriptors (the high
// word, hi, is the same for every tile); acc0 / acc1 = 0 start d0 and d2 /
// d1 afresh.
__device__ __forceinline__ void tcs_mma6(uint32_t d0, uint32_t d1, uint32_t d2, uint32_t hi, uint32_t a0,
                                         uint32_t a1, uint32_t a2, uint32_t x0, uint32_t x1, uint32_t x2,
                                         uint32_t idesc, uint32_t acc0, uint32_t acc1) {
    asm volatile(
        "{\n\t.reg .pred p0, p1;\n\t.reg .b64 da0, da1, da2, dx0, dx1, dx2;\n\t"
        "setp.ne.b32 p0, %11, 0;\n\tsetp.ne.b32 p1, %12, 0;\n\t"
        "mov.b64 da0, {%4, %3};\n\tmov.b64 da1, {%5, %3};\n\tmov.b64 da2, {%6, %3};\n\t"
        "mov.b64 dx0, {%7, %3};\n\tmov.b64 dx1, {%8, %3};\n\tmov.b64 dx2, {%9, %3};\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], da0, dx0, %10, p0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%1], da0, dx1, %10, p1;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%1], da1, dx0, %10, 1;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%2], da0, dx2, %10, p0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%2], da1, dx1, %10, 1;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%2], da2, dx0, %10, 1;\n\t}"
        ::"r"(d0), "r"(d1), "r"(d2), "r"(hi), "r"(a0), "r"(a1), "r"(a2), "r"(x0), "r"(x1), "r"(x2),
          "r"(idesc), "r"(acc0), "r"(acc1)
        : "memory");
}

// Old state and carries of 8 columns of one row (zero outside the valid range).
__device__ __forceinline__ void load_group8(const float* __restrict__ Y, const float* __restrict__ Cy,
                                            int Kown, int col_first, int ncol_left, bool rowok,
                                            float (&y)[8], float (&c)[8]) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const bool ok = rowok && q < ncol_left;
        const size_t gi = (size_t)(col_first + q) * Kown;
        y[q] = ok ? Y[gi] : 0.f;
        c[q] = ok ? Cy[gi] : 0.f;
    }
}

// Maximum over the 32 lanes of each of 8 values (|y| bits of 8 columns, one
// row per lane), as a butterfly reduce-scatter: afterwards lane l holds the
// maximum for column 4 b16 + 2 b8 + b4 (b_o = bit o of l), every lane of a
// group of four the same.
__device__ __forceinline__ unsigned colmax8(unsigned (&v)[8], int lane, int& col) {
    int base = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int o = 16 >> s;
        const int half = 4 >> s;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const unsigned send = up ? v[k] : v[k + half];
            const unsigned keep = up ? v[k + half] : v[k];
            v[k] = max(keep, __shfl_xor_sync(0xffffffffu, send, o));
        }
        base += up ? half : 0;
    }
    v[0] = max(v[0], __shfl_xor_sync(0xffffffffu, v[0], 2));
    v[0] = max(v[0], __shfl_xor_sync(0xffffffffu, v[0], 1));
    col = base;
    return v[0];
}


// Shared memory for the reduced reference state of one half-step: WH values
// per reader thread, [WH][256] so that a warp's accesses are consecutive.
__host__ __device__ inline size_t tcs_xref_bytes(int W) {
    return (size_t)(W / 2) * kTcsThreads * 4;
}

__device__ __forceinline__ void reader_bar_sync() {
    asm volatile("bar.sync 1, %0;" ::"r"(kTcsThreads) : "memory");
}

// XR: add the reduced reference state (a template flag, so that runs without
// it compile to the code they had without it).
template <int W, bool XR>
__global__ void __launch_bounds__(kTcsThreads, 1) rank2_tcs_kernel(const TcArgs a) {
    constexpr int WH = W / 2;                       // columns per readout warp
    constexpr int AST = tcs_acc_stride(W);          // accumulator column stride
    constexpr uint32_t NCOLS = tcs_tmem_cols(W);
    static_assert(W % 16 == 0 && W >= 32 && W <= 80 && WH % 8 == 0, "unsupported block width");
    cg::cluster_group cluster = cg::this_cluster();
    const int CS = (int)cluster.num_blocks();
    const int crank = (int)cluster.block_rank();
    const int blk = blockIdx.x / CS;
    const int Kp = a.Kp, STAGES = a.stages;
    const int col0 = blk * W;
    const int ncol = min(W, a.M - col0);
    const int row0 = crank * kTcRows;
    const int NKC = Kp / kTcsKC;
    // receiver traces from on-chip data when C has at most 64 rows and the
    // scratch fits in the stage ring (decided identically on the host)
    const bool chip_tr = a.traces && a.R <= kTcsTraceR &&
                         tcs_trace_scratch_bytes(W) <= (size_t)STAGES * tcs_stage_bytes(W);
    const int KC_T1B = 512 / kTcsKC;                // first chunk accumulated into T1b
    const bool two_t1 = Kp > 512;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float dt = (float)a.dt;
    const long long limit = a.spin_limit;
    const int quad = warp & 3;                      // TMEM lane quadrant of this warp
    const int chalf = warp / 4;                     // column half of a readout warp
    const int rl = 32 * quad + lane;                // row (within the slab) of a reader
    const int ridx = tid;                           // reader index 0..255

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const size_t stage_bytes = tcs_stage_bytes(W);
    unsigned char* tail = smem + (size_t)STAGES * stage_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(tail);
    uint64_t* empty = full + STAGES;
    uint64_t* dready = empty + STAGES;
    uint64_t* drain = dready + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    volatile int* abort_all = reinterpret_cast<volatile int*>(tslot + 2);
    // abort flag as published for the cluster-wide decision: written between
    // the two barriers of a half-step, where no wait can change abort_flag
    volatile int* abort_pub = reinterpret_cast<volatile int*>(tslot + 3);
    long long* consumed = reinterpret_cast<long long*>(tslot + 4);
    float* fcol = reinterpret_cast<float*>(tslot + 8);
    float* Tcol = fcol + W;
    float* xsc = Tcol + W;                          // 2^(eX_j - 7) of the current B operand
    float* xinv = xsc + W;                          // 2^(7 - eX_j)
    float* grow = xinv + W;
    float* arow = grow + kTcRows;                   // [2][128]: 2^(eA_r - 7) of Avs, Asv
    unsigned* colmax = reinterpret_cast<unsigned*>(arow + 2 * kTcRows);  // [4][W] |y| bits
    float* gmax = reinterpret_cast<float*>(colmax + 4 * W);             // [CS][W]
    float* xst = gmax + (size_t)kTcsMaxCS * W;  // [WH][256] reference state (only when given)
    float* Ys = reinterpret_cast<float*>(smem);                         // trace scratch (stage ring)
    float* Cs = Ys + (size_t)W * kTcsTStride;
    float* Pt = Cs + (size_t)kTcsTraceR * kTcsTStride;

    if (tid == 0) {
        *abort_flag = 0;
        *abort_all = 0;
        *abort_pub = 0;
        for (int s = 0; s < STAGES; ++s) { mbarrier_init(&full[s], 1); mbarrier_init(&empty[s], 1); }
        mbarrier_init(dready, 1);
        mbarrier_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) { tmem_alloc(tslot, NCOLS); tmem_relinquish(); }
    for (int c = tid; c < W; c += kTcsThreads) Tcol[c] = (a.Tper && c < ncol) ? a.Tper[col0 + c] : 1.f;
    if (tid < kTcRows) {
        grow[tid] = a.g_p[row0 + tid];
        arow[tid] = a.Ascale[0][row0 + tid];
        arow[kTcRows + tid] = a.Ascale[1][row0 + tid];
    }
    for (int i = tid; i < 4 * W; i += kTcsThreads) colmax[i] = 0u;
    __syncthreads();

    // ---- column maxima of S^0 over the own rows, agreed across the cluster
    for (int idx = tid; idx < kTcRows * W; idx += kTcsThreads) {
        const int j = idx / kTcRows, r = idx % kTcRows, row = row0 + r;
        const float x = (j < ncol && row < a.Ks) ? a.S[(size_t)(col0 + j) * a.Ks + row] : 0.f;
        atomicMax(&colmax[j], __float_as_uint(fabsf(x)));
    }
    cluster.sync();  // every CTA runs and is initialised before remote stores
    for (int j = tid; j < W; j += kTcsThreads) {
        const float bm = __uint_as_float(colmax[j]);
        for (int q = 0; q < CS; ++q) *cluster.map_shared_rank(gmax + crank * W + j, q) = bm;
    }
    cluster.sync();
    int bad = 0;
    for (int j = tid; j < W; j += kTcsThreads) {
        float mx = 0.f;
        for (int q = 0; q < CS; ++q) mx = fmaxf(mx, gmax[q * W + j]);
        bad |= !isfinite(mx);
        const int e = bound_exponent(mx);
        xsc[j] = ldexpf(1.f, e - 7);
        xinv[j] = ldexpf(1.f, 7 - e);
    }
    __syncthreads();
    const size_t xterm = (size_t)Kp * W * 2;  // bytes of one digit term of one block
    unsigned char* const Xblk0 = static_cast<unsigned char*>(a.X[0]) + (size_t)blk * kTcsTerms * xterm;
    unsigned char* const Xblk1 = static_cast<unsigned char*>(a.X[1]) + (size_t)blk * kTcsTerms * xterm;
    for (int idx = tid; idx < kTcRows * W; idx += kTcsThreads) {
        const int j = idx / kTcRows, r = idx % kTcRows, row = row0 + r;
        const float x = (j < ncol && row < a.Ks) ? a.S[(size_t)(col0 + j) * a.Ks + row] : 0.f;
        tcs_store_digits(Xblk0, xterm, tcs_xoffset(row, j, W), x * xinv[j]);
    }
    for (int c = tid; c < W; c += kTcsThreads) {
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
    const uint32_t idesc = mma_idesc(kFmtBF16, kTcRows, (uint32_t)W);
    const uint32_t xtile = (uint32_t)W * kTileRowBytes;
    const uint32_t chunk_bytes = kTcsTerms * kATileBytes + kTcsTerms * xtile;

    long long it_prod = 0, it_mma = 0;  // chunk counters of producer / MMA
    // the same counters as (ring stage, uses of that stage), advanced by one
    // so that the per-chunk loops do no 64-bit division
    int s_prod = 0, s_mma = 0;
    uint32_t u_prod = 0, u_mma = 0;
    int hs = 0;                         // half-steps done (parity of dready)
    const int N = a.nsteps;
    for (int n = 0; n < N && !*abort_all; ++n) {
#pragma unroll 1
        for (int half = 0; half < 2; ++half, ++hs) {
            const unsigned char* Aop = static_cast<const unsigned char*>(half ? a.Aop[1] : a.Aop[0]) +
                                       (size_t)crank * NKC * kTcsTerms * kATileBytes;
            const unsigned char* Xsrc = half ? Xblk1 : Xblk0;
            const bool tr_step = half == 0 && a.traces && ((n + 1) % a.r) == 0;
            const bool chip_step = tr_step && chip_tr;
            bool have = false;
            // ---- readout warps first start loading their old rows and carries
            const int row = row0 + rl;
            const int Kown = half == 0 ? a.Kv : a.Ks;
            float* Y = (half == 0 ? a.V : a.S) + row;
            float* Cy = (half == 0 ? a.compV : a.compS) + row;
            const bool rowok = row < Kown;
            const int jbase = chalf * WH;
            constexpr int NG = WH / 8;
            float ya[8], ca[8], yb[8], cb[8];
            load_group8(Y, Cy, Kown, col0 + jbase, ncol - jbase, rowok, ya, ca);
            if (NG > 1) load_group8(Y, Cy, Kown, col0 + jbase + 8, ncol - jbase - 8, rowok, yb, cb);
            // this thread's values of the reduced reference state, copied
            // asynchronously while the products run (no registers, no stall)
            const float* Xref = half == 0 ? a.Xv : a.Xs;
            if (XR && Xref) {
#pragma unroll 1
                for (int i = 0; i < WH; ++i) {
                    const int j = jbase + i;
                    const bool ok = rowok && j < ncol;
                    cp_async4(xst + (size_t)i * kTcsThreads + ridx,
                              ok ? Xref + (size_t)(col0 + j) * Kown + row : Xref, ok ? 4 : 0);
                }
            }
            if (warp == 0) {
                if (lane == 0 && !*abort_flag) {
                    // ---- producer: stream every k-chunk's digit tiles into the stage ring
                    for (int kc = 0; kc < NKC; ++kc) {
                        const int s = s_prod;
                        const uint32_t use = u_prod;
                        if (use > 0 && !mbarrier_wait(&empty[s], (use - 1) & 1, limit, abort_flag)) break;
                        unsigned char* st = smem + (size_t)s * stage_bytes;
                        mbarrier_arrive_expect_tx(&full[s], chunk_bytes);
                        for (int t = 0; t < kTcsTerms; ++t)
                            bulk_g2s(st + t * kATileBytes, Aop + ((size_t)kc * kTcsTerms + t) * kATileBytes,
                                     kATileBytes, &full[s]);
                        for (int t = 0; t < kTcsTerms; ++t)
                            bulk_g2s(st + kTcsTerms * kATileBytes + t * xtile,
                                     Xsrc + (size_t)t * xterm + (size_t)kc * xtile, xtile, &full[s]);
                        ++it_prod;
                        if (++s_prod == STAGES) { s_prod = 0; ++u_prod; }
                    }
                }
                __syncwarp();
            } else if (warp == 1) {
                if (lane == 0 && !*abort_flag) {
                    // ---- MMA issue: the six digit products of every chunk.  The
                    //      descriptors differ only in their start-address field, so
                    //      their low words are formed by adding tile offsets (in
                    //      16-byte units) to that of the ring's first tile.
                    bool ok = true;
                    const uint64_t dring = sw128_desc(cvta_shared(smem));
                    const uint32_t dhi = (uint32_t)(dring >> 32), dlo = (uint32_t)dring;
                    const uint32_t ta = kATileBytes >> 4, tx = xtile >> 4;
                    const uint32_t tstage = (uint32_t)(stage_bytes >> 4);
                    for (int kc = 0; kc < NKC; ++kc) {
                        const int s = s_mma;
                        const uint32_t use = u_mma;
                        if (!mbarrier_wait(&full[s], use & 1, limit, abort_flag)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t la = dlo + (uint32_t)s * tstage;
                        const uint32_t lx = la + kTcsTerms * ta;
                        const bool t1b = two_t1 && kc >= KC_T1B;
                        const uint32_t d0 = tbase;
                        const uint32_t d1 = tbase + (uint32_t)((t1b ? 2 : 1) * AST);
                        const uint32_t d2 = tbase + (uint32_t)(3 * AST);
                        const bool first0 = kc == 0;
                        const bool first1 = kc == (t1b ? KC_T1B : 0);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {  // four 16-deep K steps per 128-byte chunk
                            const uint32_t o = 2u * ks;     // 32 bytes
                            tcs_mma6(d0, d1, d2, dhi, la + o, la + ta + o, la + 2 * ta + o, lx + o, lx + tx + o,
                                     lx + 2 * tx + o, idesc, (first0 && ks == 0) ? 0u : 1u,
                                     (first1 && ks == 0) ? 0u : 1u);
                        }
                        mma_commit(&empty[s]);
                        ++it_mma;
                        if (++s_mma == STAGES) { s_mma = 0; ++u_mma; }
                    }
                    if (ok) mma_commit(dready);
                }
                __syncwarp();
            }
            {
                // ---- readers: one readout of the four accumulators, the fused
                //      forcing and Kahan update, the column maxima of the new
                //      state.  The old rows and carries are loaded two 8-column
                //      groups ahead (the first two while the MMAs run); the new
                //      rows wait in spare tensor-memory columns for the slicing.
                int gotl = 0;
                if (lane == 0) gotl = (*abort_flag == 0) && mbarrier_wait(dready, (uint32_t)(hs & 1), limit, abort_flag);
                have = __shfl_sync(0xffffffffu, gotl, 0) != 0;
                tc_fence_after();
                if constexpr (XR) cp_async_wait_all();  // this thread's own copies only
                const float ars = arow[half * kTcRows + rl];
                const float grw = grow[rl];
                const uint32_t tl = tbase + ((uint32_t)(32 * quad) << 16) + (uint32_t)jbase;
                // one 8-column group: readout, update, new state parked in TMEM,
                // loads of the group two ahead into the same buffers
                // accumulator registers of one group, double-buffered: the next
                // group's loads are issued before the current group's update
                struct Acc8 { uint32_t r0[8], r1a[8], r1b[8], r2[8]; };
                auto acc_issue = [&](const int g, Acc8& t) {
                    if (!have) return;
                    const int i0 = 8 * g;
                    tmem_ld8_nowait(tl + (uint32_t)i0, t.r0);
                    tmem_ld8_nowait(tl + (uint32_t)(AST + i0), t.r1a);
                    if (two_t1) tmem_ld8_nowait(tl + (uint32_t)(2 * AST + i0), t.r1b);
                    tmem_ld8_nowait(tl + (uint32_t)(3 * AST + i0), t.r2);
                };
                auto acc_wait = [&](Acc8& t) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (!have) { t.r0[q] = 0u; t.r1a[q] = 0u; t.r2[q] = 0u; }
                        if (!have || !two_t1) t.r1b[q] = 0u;
                    }
                    if (have) tmem_wait_ld4(t.r0, t.r1a, t.r1b, t.r2);
                };
                auto group = [&](const int g, Acc8& cur, Acc8& nxt, float (&yg)[8], float (&cg_)[8]) {
                    const int i0 = 8 * g;
                    if (g + 1 < NG) acc_issue(g + 1, nxt);
                    const uint32_t(&r0)[8] = cur.r0;
                    const uint32_t(&r1a)[8] = cur.r1a;
                    const uint32_t(&r1b)[8] = cur.r1b;
                    const uint32_t(&r2)[8] = cur.r2;
                    float ynew[8], scl[8], fq[8];
                    unsigned ybits[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {  // shared-memory operands before any global store
                        scl[q] = ars * xsc[jbase + i0 + q];
                        fq[q] = half == 0 ? fcol[jbase + i0 + q] : 0.f;
                    }
                    // branch-free update of the 8 columns (the valid entries are
                    // selected afterwards), so that their dependency chains interleave
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float t1 = __fadd_rn(__uint_as_float(r1a[q]), __uint_as_float(r1b[q]));
                        const float u = __fmaf_rn(__uint_as_float(r2[q]), 1.f / 65536.f, t1 * (1.f / 256.f));
                        const float R = __fadd_rn(__uint_as_float(r0[q]), u);
                        float inc = R * scl[q];
                        inc = half == 0 ? __fmaf_rn(grw, fq[q], inc) : inc;
                        if (XR && Xref) inc = inc + xst[(size_t)(i0 + q) * kTcsThreads + ridx];
                        inc = inc * dt;
                        float c = cg_[q];
                        const float y = kahan_add(yg[q], inc, c);
                        const bool ok = have && rowok && jbase + i0 + q < ncol;
                        ynew[q] = ok ? y : yg[q];
                        cg_[q] = ok ? c : cg_[q];
                        ybits[q] = __float_as_uint(fabsf(ynew[q]));
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int j = jbase + i0 + q;
                        if (have && rowok && j < ncol) {
                            const size_t gi = (size_t)(col0 + j) * Kown;
                            Y[gi] = ynew[q];
                            Cy[gi] = cg_[q];
                        }
                        if (chip_step) Ys[(size_t)j * kTcsTStride + rl] = ynew[q];
                    }
                    {
                        int cq;
                        const unsigned m = colmax8(ybits, lane, cq);
                        if ((lane & 3) == 0) colmax[quad * W + jbase + i0 + cq] = m;
                    }
                    tmem_st8(tl + (uint32_t)(4 * AST + i0), ynew);
                    if (g + 2 < NG)
                        load_group8(Y, Cy, Kown, col0 + jbase + i0 + 16, ncol - jbase - i0 - 16, rowok, yg, cg_);
                    if (g + 1 < NG) acc_wait(nxt);
                };
                Acc8 accA, accB;
                acc_issue(0, accA);
                acc_wait(accA);
#pragma unroll 1
                for (int g = 0; g < NG; g += 2) {
                    group(g, accA, accB, ya, ca);
                    if (g + 1 < NG) group(g + 1, accB, accA, yb, cb);
                }
                tmem_wait_st();
                tc_fence_before();
                if (chip_step) {
                    // this CTA's 128 columns of C (rows jr < 64; zero beyond R)
                    for (int idx = ridx; idx < kTcsTraceR * kTcRows; idx += kTcsThreads) {
                        const int jr = idx / kTcRows, r = idx % kTcRows;
                        Cs[(size_t)jr * kTcsTStride + r] = jr < a.R ? a.C_p[(size_t)jr * Kp + row0 + r] : 0.f;
                    }
                }
                reader_bar_sync();
                if (chip_step) {
                    // partial traces over the own rows, P[jr][c] = sum_r Cs[jr][r] Ys[c][r]
                    // (fixed order): reader t computes jr = 4 (t / 16) + 0..3 and
                    // columns (t % 16) * (W / 16) + 0..W/16-1
                    constexpr int CB = W / 16;
                    const int cgp = ridx % 16, jg = ridx / 16;
                    float pacc[4][CB];
#pragma unroll
                    for (int t = 0; t < 4; ++t)
#pragma unroll
                        for (int i = 0; i < CB; ++i) pacc[t][i] = 0.f;
#pragma unroll 2
                    for (int r = 0; r < kTcRows; r += 4) {
                        float4 cv4[4], yv4[CB];
#pragma unroll
                        for (int t = 0; t < 4; ++t)
                            cv4[t] = *reinterpret_cast<const float4*>(Cs + (size_t)(4 * jg + t) * kTcsTStride + r);
#pragma unroll
                        for (int i = 0; i < CB; ++i)
                            yv4[i] = *reinterpret_cast<const float4*>(Ys + (size_t)(cgp * CB + i) * kTcsTStride + r);
#pragma unroll
                        for (int t = 0; t < 4; ++t)
#pragma unroll
                            for (int i = 0; i < CB; ++i) {
                                pacc[t][i] = __fmaf_rn(cv4[t].x, yv4[i].x, pacc[t][i]);
                                pacc[t][i] = __fmaf_rn(cv4[t].y, yv4[i].y, pacc[t][i]);
                                pacc[t][i] = __fmaf_rn(cv4[t].z, yv4[i].z, pacc[t][i]);
                                pacc[t][i] = __fmaf_rn(cv4[t].w, yv4[i].w, pacc[t][i]);
                            }
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t)
#pragma unroll
                        for (int i = 0; i < CB; ++i) Pt[(size_t)(4 * jg + t) * W + cgp * CB + i] = pacc[t][i];
                }
                // block maxima of this CTA, stored into every CTA of the cluster
                if (ridx < W) {
                    const unsigned bm = max(max(colmax[ridx], colmax[W + ridx]),
                                            max(colmax[2 * W + ridx], colmax[3 * W + ridx]));
                    for (int q = 0; q < CS; ++q)
                        *cluster.map_shared_rank(gmax + crank * W + ridx, q) = __uint_as_float(bm);
                }
            }
            cluster.sync();
            // ---- column exponents of the new state (the B operand of the next half-step)
            for (int j = tid; j < W; j += kTcsThreads) {
                float mx = 0.f;
                for (int q = 0; q < CS; ++q) mx = fmaxf(mx, gmax[q * W + j]);
                bad |= !isfinite(mx);
                const int e = bound_exponent(mx);
                xsc[j] = ldexpf(1.f, e - 7);
                xinv[j] = ldexpf(1.f, 7 - e);
            }
            __syncthreads();
            if (chip_step) {
                // receiver rows crank*rpc .. : sum of the CTAs' partials in rank order
                const int rec = (n + 1) / a.r - 1;
                const int npair = a.rpc * ncol;
                for (int pr = tid; pr < npair; pr += kTcsThreads) {
                    const int c = pr / a.rpc, jj = pr % a.rpc, jr = crank * a.rpc + jj;
                    if (jr >= a.R) continue;
                    float tsum = 0.f;
                    for (int q = 0; q < CS; ++q) tsum += *cluster.map_shared_rank(Pt + (size_t)jr * W + c, q);
                    a.traces[((size_t)rec * a.Mtot + col0 + c) * a.R + jr] = tsum;
                }
                fence_proxy_async_shared();  // scratch writes before the next bulk copies into the ring
            }
            {
                unsigned char* Xdst = half ? Xblk0 : Xblk1;  // V feeds the S half and vice versa
                const uint32_t ts = tbase + ((uint32_t)(32 * quad) << 16) + (uint32_t)(4 * AST + chalf * WH);
                tc_fence_after();
#pragma unroll 1
                for (int i0 = 0; i0 < WH; i0 += 8) {
                    float yn[8], xi[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) xi[q] = xinv[chalf * WH + i0 + q];  // before any store
                    tmem_ld8(ts + (uint32_t)i0, yn);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int j = chalf * WH + i0 + q;
                        tcs_store_digits(Xdst, xterm, tcs_xoffset(row, j, W), yn[q] * xi[q]);
                    }
                }
                tc_fence_before();
            }
            fence_proxy_async_global();
            // forcing of the next step (read by the next velocity epilogue)
            if (half == 1 && n + 1 < N) {
                for (int c = tid; c < W; c += kTcsThreads) {
                    float f = 0.f;
                    if (c < ncol) {
                        if (a.ftab) f = a.ftab[(size_t)(n + 1) * a.Mtot + col0 + c];
                        else if (a.Tper) f = wavelet_eval(a.wavelet, a.n0 + n + 1, a.dt, Tcol[c]);
                    }
                    fcol[c] = f;
                }
            }
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
            if (tr_step && !chip_step) {
                const int rec = (n + 1) / a.r - 1;
                const int npair = a.rpc * ncol;
                for (int pr = warp; pr < npair; pr += kTcsThreads / 32) {
                    const int jj = pr / ncol, c = pr % ncol, jr = crank * a.rpc + jj;
                    if (jr >= a.R) continue;
                    const float* vcol = a.V + (size_t)(col0 + c) * a.Kv;
                    const float* crow = a.C_p + (size_t)jr * Kp;
                    float tacc = 0.f;
#pragma unroll 4
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
    bad = __syncthreads_or(bad);
    if (tid == 0 && a.status) {
        if (*abort_flag) atomicCAS(a.status, 0, 5 /* ROM_E_TIMEOUT */);
        else if (bad) atomicCAS(a.status, 0, 6 /* ROM_E_NONFINITE */);
    }
    tc_fence_before();
    __syncthreads();
    cluster.sync();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tbase, NCOLS);
}

}  // namespace romk
