// Split-role, two-block DATAFLOW cluster kernel for the rank-2 leapfrog (FP32).
//
// Same work split as rank2_split.cuh; instead of one cluster barrier per
// phase, consumers wait on per-block mbarriers fed by asynchronous stores.
//
// Sec. 3.1's leapfrog makes every half-step depend on the previous one.  This
// kernel gives each thread-block cluster TWO independent column blocks A and
// B (columns are independent realizations, Sec. 2.4) and runs them half a
// step apart, so velocity and stress work always overlap:
//
//   V-role CTAs: V(A)^1, V(B)^1, V(A)^2, V(B)^2, ...   (V += dt (Avs S + g f^T))
//   S-role CTAs:   S(A)^1, S(B)^1, S(A)^2, ...        (S += dt Asv V, new V)
//
// The cluster has 2H CTAs (H = Kp / 64).  CTA s < H keeps rows
// [64 s, 64 s + 64) of Avs in registers and owns those rows of V for both
// blocks; CTA H + s keeps the same rows of Asv and owns those rows of S.  Each
// CTA holds the full operand of both blocks (S for the velocity role, V for
// the stress role) in shared memory.
//
// Synchronisation is dataflow, not phase barriers: the operand of each
// (block, 4-column group) has an mbarrier in every consumer CTA.  A producer
// warp that finishes its 8 x 4 tile writes it into the H consumer CTAs with
// asynchronous distributed-shared-memory stores (st.async, spread over all 32
// lanes) that count their bytes against the consumer's mbarrier; the consumer
// arms each phase with the bytes it expects and waits on it (acquire,
// bounded) before reading that group.  No fence or remote atomic is needed.  Every reuse of a
// buffer or an mbarrier phase is ordered by the same per-group causality: a
// producer can only produce step n+2 of group g after every consumer warp
// has pushed step n+1 of group g, which each does only after it finished
// reading step n+1.  A wait that runs out (see Rank2Args::spin_limit) records
// ROM_E_TIMEOUT, stops the CTA's work and leaves through the final cluster
// barrier, so no CTA exits while a peer may still write to it.
//
// Register tiling: thread (row quad q, chunk j) holds rows 4q..4q+3 of its
// operator at k = 64 i + 4 j + t (i < KI, t < 4): every 16-byte shared load of
// the operand feeds 16 FMAs.  A butterfly reduce-scatter over the 16 chunk
// lanes leaves each lane one (row, column) sum for the fused epilogue: the
// Ricker forcing g f_n^T (Sec. 2.2, 3.2, evaluated by four lanes and
// shuffled), the Kahan-compensated FP32 update, the push.  Receiver traces
// y = C V (Sec. 4.5.2) are produced by the stress role from the full new V,
// group by group, before the group is released.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "rank2_simt.cuh"
#include "rank2_split.cuh"
#include "rom_internal.h"

namespace romk {

struct DataflowSmem {
    size_t X, own, comp, C, T, g, mbar, flag, sent, total;
};

// Largest number of producer CTAs of one role (H = Kp / 64 <= 16).
constexpr int kDataflowMaxH = 16;

__host__ __device__ inline DataflowSmem dataflow_smem_layout(int Wa, int Kp, int rpc) {
    DataflowSmem s{};
    size_t o = 0;
    s.X = o;    o += align16((size_t)2 * Wa * Kp * sizeof(float));
    s.own = o;  o += align16((size_t)2 * Wa * kOwnStride * sizeof(float));
    s.comp = o; o += align16((size_t)2 * Wa * kOwnStride * sizeof(float));
    s.C = o;    o += align16((size_t)rpc * Kp * sizeof(float));
    s.T = o;    o += align16((size_t)2 * Wa * sizeof(float));
    s.g = o;    o += align16((size_t)kSplitRows * sizeof(float));
    s.mbar = o; o += align16((size_t)2 * sizeof(unsigned long long));
    s.flag = o; o += 16;
    // bytes each producer slab of the other role sent per block [H][2], the
    // phases armed per block [2], and this CTA's own sent bytes per block [2]
    s.sent = o; o += align16((size_t)(kDataflowMaxH * 2 + 4) * sizeof(unsigned));
    s.total = o;
    return s;
}

// ---- mbarrier / cluster primitives (PTX, sm_90+ semantics)
__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init_cluster() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arrive on a local mbarrier and add `bytes` to the transaction count its
// current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Count `bytes` as arrived on the current phase of a local mbarrier without
// an asynchronous copy (used to retire bytes a producer will never send).
__device__ __forceinline__ void mbar_complete_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: returns false (and raises the CTA's abort flag) if the phase
// did not complete within `limit` clock cycles or another warp aborted.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  long long limit, volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            return false;
        }
    }
}

template <int KI>
__global__ void __launch_bounds__(kThreads, 1) rank2_dataflow_kernel(const Rank2Args a) {
    constexpr int CB = kSplitCB;
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = (int)cluster.num_blocks();
    const int H = cs / 2;
    const int crank = (int)cluster.block_rank();
    const bool vrole = crank < H;
    const int s = vrole ? crank : crank - H;  // row slab
    const int row0 = s * kSplitRows;
    const int peer0 = vrole ? H : 0;          // first CTA of the other role
    const int clu = blockIdx.x / cs;
    const int Wa = a.Wa, Kp = a.Kp;
    const int G = Wa / CB;                    // column groups per block
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = lane & 15;
    const int q = warp * 2 + (lane >> 4);     // row quad
    const float dt = (float)a.dt;
    const long long limit = a.spin_limit;

    extern __shared__ __align__(16) unsigned char smem[];
    const DataflowSmem L = dataflow_smem_layout(Wa, Kp, a.rpc);
    float* X = reinterpret_cast<float*>(smem + L.X);        // [2][Wa][Kp] operand copies
    float* own = reinterpret_cast<float*>(smem + L.own);    // [2][Wa][72] owned rows
    float* comp = reinterpret_cast<float*>(smem + L.comp);  // [2][Wa][72] Kahan carries
    float* Cown = reinterpret_cast<float*>(smem + L.C);     // [rpc][Kp] receiver rows
    float* Tcol = reinterpret_cast<float*>(smem + L.T);     // [2][Wa] periods
    float* gown = reinterpret_cast<float*>(smem + L.g);     // [64] source row
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + L.mbar);  // [2]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.flag);
    unsigned* sent_in = reinterpret_cast<unsigned*>(smem + L.sent);  // [H][2], written by peers
    unsigned* armed = sent_in + 2 * kDataflowMaxH;                    // [2]
    unsigned* sent_out = armed + 2;                                   // [2]

    // column ranges of the two blocks, kept in scalars
    const int gc0_0 = a.col_base + (2 * clu) * a.Wv;
    const int gc0_1 = gc0_0 + a.Wv;
    const int nr0 = a.M - (2 * clu) * a.Wv, nr1 = nr0 - a.Wv;
    const int nc0 = nr0 < 0 ? 0 : (nr0 > a.Wv ? a.Wv : nr0);
    const int nc1 = nr1 < 0 ? 0 : (nr1 > a.Wv ? a.Wv : nr1);
    auto gc0 = [&](int b) { return b ? gc0_1 : gc0_0; };
    auto ncol = [&](int b) { return b ? nc1 : nc0; };

    const float* Vin = static_cast<const float*>(a.V);
    const float* Sin = static_cast<const float*>(a.S);
    const int Kown = vrole ? a.Kv : a.Ks;
    const float* own_in = vrole ? Vin : Sin;
    const float* comp_in = static_cast<const float*>(vrole ? a.compV : a.compS);

    // ---- initial state.  V role: operand = full S^0, own = V^0 rows.
    //      S role: operand arrives with the first velocity pushes; own = S^0 rows.
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
    const float* Cp = static_cast<const float*>(a.C_p);
    if (!vrole) {
        for (int idx = tid; idx < a.rpc * Kp; idx += kThreads) {
            const int jj = idx / Kp, k = idx % Kp, jr = s * a.rpc + jj;
            Cown[idx] = (Cp && jr < a.R) ? Cp[(size_t)jr * Kp + k] : 0.f;
        }
    }
    if (tid < kSplitRows) gown[tid] = vrole ? static_cast<const float*>(a.g_p)[row0 + tid] : 0.f;
    for (int idx = tid; idx < 2 * Wa; idx += kThreads) {
        const int b = idx / Wa, c = idx % Wa;
        Tcol[idx] = (a.Tper && c < ncol(b)) ? static_cast<const float*>(a.Tper)[gc0(b) + c] : 1.f;
    }
    // bytes of one block's operand: H producer CTAs x 64 rows x Wa columns
    const unsigned block_bytes = (unsigned)(H * kSplitRows * Wa * sizeof(float));
    if (tid == 0) {
        *abort_flag = 0;
        for (int i = 0; i < 2 * kDataflowMaxH + 4; ++i) sent_in[i] = 0u;
        for (int i = 0; i < 2; ++i) mbar_init(&mbar[i], 1u);
        fence_mbar_init_cluster();
        for (int i = 0; i < 2; ++i) mbar_arrive_expect_tx(&mbar[i], block_bytes);
        armed[0] = armed[1] = 1u;
    }

    float op[4][4 * KI];
    load_op_quad<KI>(op, static_cast<const float*>(vrole ? a.Avs_rm : a.Asv_rm), Kp, row0 + 4 * q, j);
    // shared::cluster windows of the (at most two) peers this lane writes to
    unsigned rX[2] = {0u, 0u}, rB[2] = {0u, 0u};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int d = (lane >> 3) + 4 * e;
        if (d < H) {
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rX[e]) : "r"(smem_addr(X)), "r"(peer0 + d));
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rB[e]) : "r"(smem_addr(mbar)), "r"(peer0 + d));
        }
    }
    // every CTA's buffers and mbarriers exist before any peer writes to them
    cluster.sync();

    float* traces = static_cast<float*>(a.traces);
    const float* ftab = static_cast<const float*>(a.ftab);
    const int N = a.nsteps;
    const int nphase = 2 * N + 1;
    const bool stall_test = a.debug_skip_push && crank == 0;
    const float* Xrole = static_cast<const float*>(vrole ? a.Xv : a.Xs);  // reference state or null
    // column groups this warp pushed per block (every push carries 128 bytes
    // to each consumer CTA): retires unsent bytes after a timeout, see below
    unsigned pushed0 = 0u, pushed1 = 0u;
    for (int p = 0; p < nphase; ++p) {
        int b, n;
        if (vrole) { b = p & 1; n = (p - b) >> 1; }
        else { b = (p & 1) ^ 1; n = (p - 1 - b) >> 1; }
        if (n < 0 || n >= N || ncol(b) == 0) continue;
        if (*abort_flag) break;
        float* Xb = X + (size_t)b * Wa * Kp;
        float* ownb = own + (size_t)b * Wa * kOwnStride;
        float* compb = comp + (size_t)b * Wa * kOwnStride;
        unsigned long long* mb = mbar + b;
        // the operand of this phase arrived as completion (n-1) of the V role's
        // mbarriers (S^n, n >= 1; S^0 is local) or completion n of the S role's (V^{n+1})
        const bool need_wait = vrole ? (n >= 1) : true;
        const unsigned parity = vrole ? (unsigned)((n - 1) & 1) : (unsigned)(n & 1);
        const bool record = !vrole && traces && ((n + 1) % a.r) == 0;
        const int rec = (n + 1) / (a.r > 0 ? a.r : 1) - 1;
        if (need_wait) {
            // lane 0 spins (bounded); the verdict is shared so the warp stays
            // converged, then every lane takes its own acquire of the phase
            int got = 1;
            if (lane == 0) got = mbar_wait_bounded(mb, parity, limit, abort_flag) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            mbar_try_wait(mb, parity);
            // arm the next completion of this mbarrier (the V role also
            // receives S^N, which it drains before leaving)
            const int k = vrole ? n - 1 : n;
            if (warp == 0 && lane == 0 && k + 1 <= N - 1) {
                mbar_arrive_expect_tx(mb, block_bytes);
                armed[b] += 1u;
            }
        }
        for (int g = 0; g < G; ++g) {
            const int c0 = g * CB;
            // this lane's reference-state value, fetched before the products
            float xr = 0.f;
            if (Xrole) {
                const int si = rs16_slot<4 * CB>(j);
                const int rl = 4 * q + si / CB, c = c0 + si % CB;
                if (c < ncol(b) && row0 + rl < Kown) xr = Xrole[(size_t)(gc0(b) + c) * Kown + row0 + rl];
            }
            // ---- products of this group
            float acc[4][CB];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int cc = 0; cc < CB; ++cc) acc[r][cc] = 0.f;
#pragma unroll
            for (int i = 0; i < KI; ++i) {
                float x[CB][4];
#pragma unroll
                for (int cc = 0; cc < CB; ++cc) load4(Xb + (size_t)(c0 + cc) * Kp + 64 * i + 4 * j, x[cc]);
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int cc = 0; cc < CB; ++cc)
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            acc[r][cc] = __fmaf_rn(op[r][4 * i + t], x[cc][t], acc[r][cc]);
            }
            // ---- receiver traces of V^{n+1} for this group (stress role), taken
            //      before the group is released back to the velocity role
            if (record) {
                const int npair = a.rpc * CB;
                for (int pr = warp; pr < npair; pr += kSplitWarps) {
                    const int jj = pr / CB, cc = pr % CB, jr = s * a.rpc + jj, c = c0 + cc;
                    if (jr >= a.R || c >= ncol(b)) continue;
                    float tacc = 0.f;
                    for (int k = 4 * lane; k < Kp; k += 128) {
                        float cx[4], vx[4];
                        load4(Cown + (size_t)jj * Kp + k, cx);
                        load4(Xb + (size_t)c * Kp + k, vx);
#pragma unroll
                        for (int t = 0; t < 4; ++t) tacc = __fmaf_rn(cx[t], vx[t], tacc);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) tacc += __shfl_xor_sync(0xffffffffu, tacc, o);
                    if (lane == 0) traces[((size_t)rec * a.Mtot + gc0(b) + c) * a.R + jr] = tacc;
                }
            }
            // ---- reduce-scatter, fused epilogue
            float v[4 * CB];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int cc = 0; cc < CB; ++cc) v[r * CB + cc] = acc[r][cc];
            int vi;
            bool active;
            const float tot = reduce_scatter16<float, 4 * CB>(v, j, vi, active);
            const int rl = 4 * q + vi / CB;
            const int c = c0 + vi % CB;
            float inc = tot;
            if (vrole) {
                // forcing f_n of the group's four columns, evaluated by lanes 0..3
                float f = 0.f;
                if (lane < CB) {
                    const int cl = c0 + lane;
                    if (cl < ncol(b)) {
                        if (ftab) f = ftab[(size_t)n * a.Mtot + gc0(b) + cl];
                        else if (a.Tper) f = wavelet_eval(a.wavelet, (long long)a.n0 + n, a.dt, Tcol[b * Wa + cl]);
                    }
                }
                f = __shfl_sync(0xffffffffu, f, vi % CB);
                inc = __fmaf_rn(gown[rl], f, inc);
            }
            if (Xrole) inc = inc + xr;
            inc = inc * dt;
            float* yp = ownb + c * kOwnStride + rl;
            *yp = kahan_add(*yp, inc, compb[c * kOwnStride + rl]);
            __syncwarp();
            // ---- push this warp's 8 x 4 tile (rows 8 warp .. 8 warp + 7) to the
            //      other role; lane L carries tile L % 8 to peers L / 8, L / 8 + 4, ...
            if (!stall_test) {
                const int tile = lane & 7, cc = tile >> 1, half = tile & 1;
                const int rloc = 8 * warp + 4 * half;
                const float4 val = *reinterpret_cast<const float4*>(ownb + (c0 + cc) * kOwnStride + rloc);
                const unsigned xoff = (unsigned)(((size_t)b * Wa * Kp + (size_t)(c0 + cc) * Kp + row0 + rloc) * sizeof(float));
                const unsigned boff = (unsigned)(b * sizeof(unsigned long long));
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if ((lane >> 3) + 4 * e < H) {
                        asm volatile(
                            "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
                            ::"r"(rX[e] + xoff), "f"(val.x), "f"(val.y), "f"(val.z), "f"(val.w), "r"(rB[e] + boff)
                            : "memory");
                    }
                }
                if (b) ++pushed1; else ++pushed0;
            }
        }
    }
    // the V role also received S^N (the stress role's last push): wait for it,
    // so that no asynchronous store is still in flight when the CTA leaves
    if (vrole && N >= 1 && !*abort_flag) {
        for (int b = 0; b < 2; ++b) {
            if (ncol(b) == 0) continue;
            int got = 1;
            if (lane == 0) got = mbar_wait_bounded(&mbar[b], (unsigned)((N - 1) & 1), limit, abort_flag) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
        }
    }
    const bool aborted = *abort_flag != 0;
    if (aborted && tid == 0 && a.status) atomicCAS(a.status, 0, 5 /* ROM_E_TIMEOUT */);
    // ---- drain.  Stores a peer issued before it stopped may still be in
    // flight into this CTA's shared memory.  Every CTA (a timeout or not, so
    // the barriers stay cluster-uniform) tells each consumer how many bytes it
    // sent per block; past the barrier no CTA issues another store.  Each
    // consumer then retires, on the phase it armed last, the bytes that will
    // never come (armed phases x block bytes - bytes sent), so that phase
    // completes exactly when every byte sent has landed, and waits for it
    // (bounded).  After a complete run nothing is outstanding and the wait
    // returns at once.
    if (lane == 0) {
        atomicAdd(&sent_out[0], pushed0 * 128u);
        atomicAdd(&sent_out[1], pushed1 * 128u);
    }
    __syncthreads();
    if (tid < H) {
        unsigned dst;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                     : "=r"(dst) : "r"(smem_addr(sent_in + 2 * s)), "r"(peer0 + tid));
        asm volatile("st.shared::cluster.v2.u32 [%0], {%1, %2};"
                     ::"r"(dst), "r"(sent_out[0]), "r"(sent_out[1]) : "memory");
    }
    cluster.sync();
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            unsigned got = 0u;
            for (int d = 0; d < H; ++d) got += sent_in[2 * d + b];
            const unsigned expect = armed[b] * block_bytes;
            if (expect > got) mbar_complete_tx(&mbar[b], expect - got);
            const unsigned parity = (armed[b] - 1u) & 1u;
            const long long t0 = clock64();
            while (!mbar_try_wait(&mbar[b], parity)) {
                if (clock64() - t0 > limit) {
                    if (a.status) atomicCAS(a.status, 0, 5 /* ROM_E_TIMEOUT */);
                    break;
                }
            }
        }
    }
    __syncthreads();

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

}  // namespace romk
