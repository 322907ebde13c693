// Rank-2 full-order model (FOM) of the paper's test case on the GPU: the
// axisymmetric elastic shear-wave system of Sec. 3, Eq. (fom_asym), in
// velocity-stress form, advanced by the velocity-first leapfrog for M forcing
// realizations at once (the rank-2 FOM of Eq. (shwave_ode_tensor)).
//
// Discretization: second-order staggered grid in flux form on
// r_cmb <= r <= r_earth, 0 <= theta <= pi, Nr x Nt intervals:
//     v        at (r_{i+1/2}, theta_j),       i in [0, Nr), j in [1, Nt)
//     sigma_rp at (r_i, theta_j),             i in [1, Nr), j in [1, Nt)
//     sigma_tp at (r_{i+1/2}, theta_{j+1/2}), i in [0, Nr), j in [1, Nt - 1)
//     rho v_t      = r^-3 (r^3 sigma_rp)_r + (r sin^2)^-1 (sin^2 sigma_tp)_theta + f
//     (sigma_rp)_t = mu r (v / r)_r,  (sigma_tp)_t = mu (sin / r)(v / sin)_theta
// with v = 0 on the axis and sigma_rp = 0 on the axis and on both free
// surfaces (Sec. 3), and sigma_tp = 0 at the two half points next to the axis
// (v / sin(theta) extrapolated to the axis with zero slope).  Each velocity
// row has at most four non-zeros and each stress row two.
//
// Layout: unknown-major, M realizations contiguous per unknown:
//     V[k * M + m], k = i (Nt - 1) + (j - 1);  S1[k * M + m], k = (i - 1)(Nt - 1) + (j - 1);
//     S2[k * M + m], k = i (Nt - 2) + (j - 1).
// A warp reads whole M-vectors of its stencil neighbours, so every access
// is coalesced and the stencil's reuse stays in L1/L2.  The run is bound by
// HBM: 12 M bytes per unknown per step in FP32 (read V, S and write V in the
// velocity pass; read V, S and write S in the stress pass).
//
// Per step: velocity kernel, point source, receiver record (on record
// steps), stress kernel, and a one-thread tick of the device step counter.  The kernels
// read the step from that counter, so a CUDA graph of kFomGraphSteps steps is
// captured once per argument set and replayed; steps past nsteps are no-ops.
#include <cuda_runtime.h>
#include <math.h>

#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "dev_common.cuh"
#include "rom_internal.h"

namespace romk {

constexpr int kFomThreads = 256;
constexpr int kFomGraphSteps = 64;
constexpr int kFomSegRows = 32;  // radial rows per block of the fused pass

struct FomCtl {
    long long step, nsteps, n0;
};

// Per-row factors of the stencils (all divided out of the inner loop).
template <typename T>
struct FomTables {
    const T* cr_p;   // [Nr]  r_{i+1}^3 / (rho r_{i+1/2}^3 dr), 0 at i = Nr - 1
    const T* cr_m;   // [Nr]  r_i^3 / (rho r_{i+1/2}^3 dr), 0 at i = 0
    const T* inv_rh; // [Nr]  1 / r_{i+1/2}
    const T* pt_p;   // [Nt]  sin^2 theta_{j+1/2} / (rho sin^2 theta_j dth), 0 at j = Nt - 1
    const T* pt_m;   // [Nt]  sin^2 theta_{j-1/2} / (rho sin^2 theta_j dth), 0 at j = 1
    const T* q_u;    // [Nr]  mu r_i / (r_{i+1/2} dr)
    const T* q_d;    // [Nr]  mu r_i / (r_{i-1/2} dr)
    const T* w_p;    // [Nt]  mu sin theta_{j+1/2} / (sin theta_{j+1} dth)
    const T* w_m;    // [Nt]  mu sin theta_{j+1/2} / (sin theta_j dth)
};

template <typename T>
struct FomArgs {
    FomTables<T> tb;
    T* V;
    T* S1;
    T* S2;
    const T* Tper;   // M periods, or null
    const int* recv; // nrecv velocity unknowns, or null
    T* traces;       // records of nrecv x M, or null
    const FomCtl* ctl;
    int Nr, Nt, M, src, nrecv, r, wavelet;
    double dt, rho;
    // fused single pass: second buffer set (ping-pong by step parity), the
    // source's grid point and the radial rows per block
    T* V2;
    T* S12;
    T* S22;
    int fused, src_i, src_j, seg_rows;
};

// Vector of VW consecutive realizations (16-byte loads when VW > 1).
template <typename T, int VW> struct FomVec;
template <> struct FomVec<float, 1> { using type = float; };
template <> struct FomVec<float, 4> { using type = float4; };
template <> struct FomVec<double, 1> { using type = double; };
template <> struct FomVec<double, 2> { using type = double2; };

template <typename T, int VW>
__device__ __forceinline__ void fom_load(const T* p, T (&x)[VW]) {
    const typename FomVec<T, VW>::type v = *reinterpret_cast<const typename FomVec<T, VW>::type*>(p);
    const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int q = 0; q < VW; ++q) x[q] = e[q];
}
template <typename T, int VW>
__device__ __forceinline__ void fom_store(T* p, const T (&x)[VW]) {
    typename FomVec<T, VW>::type v;
    T* e = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int q = 0; q < VW; ++q) e[q] = x[q];
    *reinterpret_cast<typename FomVec<T, VW>::type*>(p) = v;
}

// Thread layout of the two passes: persistent blocks stride over tiles of
// (radial index i, blockDim.y polar points j); in a tile threadIdx.y picks j
// and threadIdx.x runs over the realizations in groups of VW (a warp reads
// whole M-vectors with 16-byte loads).  The step word is read once per block.
template <typename T, int VW>
__global__ void __launch_bounds__(kFomThreads) fom_velocity_kernel(const FomArgs<T> a) {
    const long long n = a.ctl->step;
    if (n >= a.ctl->nsteps) return;
    const int Nt1 = a.Nt - 1, Nt2 = a.Nt - 2, M = a.M;
    const T dt = (T)a.dt;
    const int gx = (Nt1 + blockDim.y - 1) / blockDim.y;
    const long long tiles = (long long)a.Nr * gx;
    const T* __restrict__ S1 = a.S1;
    const T* __restrict__ S2 = a.S2;
    T* __restrict__ Vv = a.V;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int i = (int)(t / gx);
        const int j = (int)(t - (long long)i * gx) * blockDim.y + threadIdx.y + 1;
        if (j >= a.Nt) continue;
        const T cp = a.tb.cr_p[i], cm = a.tb.cr_m[i], ir = a.tb.inv_rh[i];
        const T pp = a.tb.pt_p[j], pm = a.tb.pt_m[j];
        const bool hp = i + 1 < a.Nr, hm = i >= 1, h2p = j <= Nt2, h2m = j >= 2;
        const size_t kv = (size_t)i * Nt1 + (j - 1);
        // stencil neighbours (the pointers of absent ones are never read)
        const T* s1p = S1 + (hp ? kv : 0) * M;                                  // sigma_rp (i + 1, j)
        const T* s1m = S1 + (hm ? (size_t)(i - 1) * Nt1 + (j - 1) : 0) * M;     // sigma_rp (i, j)
        const T* s2p = S2 + (h2p ? (size_t)i * Nt2 + (j - 1) : 0) * M;          // sigma_tp (i + 1/2, j + 1/2)
        const T* s2m = S2 + (h2m ? (size_t)i * Nt2 + (j - 2) : 0) * M;          // sigma_tp (i + 1/2, j - 1/2)
        T* v = Vv + kv * M;
        for (int m = threadIdx.x * VW; m < M; m += blockDim.x * VW) {
            T x1p[VW], x1m[VW], x2p[VW], x2m[VW], y[VW];
#pragma unroll
            for (int q = 0; q < VW; ++q) x1p[q] = x1m[q] = x2p[q] = x2m[q] = T(0);
            if (hp) fom_load<T, VW>(s1p + m, x1p);
            if (hm) fom_load<T, VW>(s1m + m, x1m);
            if (h2p) fom_load<T, VW>(s2p + m, x2p);
            if (h2m) fom_load<T, VW>(s2m + m, x2m);
            fom_load<T, VW>(v + m, y);
#pragma unroll
            for (int q = 0; q < VW; ++q)
                y[q] = y[q] + dt * (cp * x1p[q] - cm * x1m[q] + ir * (pp * x2p[q] - pm * x2m[q]));
            fom_store<T, VW>(v + m, y);
        }
    }
}

// The point source of the step, after the velocity pass (one row):
// v[src] += (dt / rho) f(t_n; T_m).
template <typename T>
__global__ void __launch_bounds__(kFomThreads) fom_source_kernel(const FomArgs<T> a) {
    const long long n = a.ctl->step;
    if (n >= a.ctl->nsteps) return;
    const T c = (T)(a.dt / a.rho);
    T* v = a.V + (size_t)a.src * a.M;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < a.M; m += gridDim.x * blockDim.x)
        v[m] = v[m] + c * (T)wavelet_eval(a.wavelet, a.ctl->n0 + n, a.dt, a.Tper[m]);
}

template <typename T>
__global__ void __launch_bounds__(kFomThreads) fom_record_kernel(const FomArgs<T> a) {
    const long long n = a.ctl->step;
    if (n >= a.ctl->nsteps || ((n + 1) % a.r) != 0) return;
    const long long rec = (n + 1) / a.r - 1;
    const int tot = a.nrecv * a.M;
    const T* V = (a.fused && !(n & 1)) ? a.V2 : a.V;  // the buffer this step wrote
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += gridDim.x * blockDim.x) {
        const int kk = idx / a.M, m = idx - kk * a.M;
        a.traces[(rec * a.nrecv + kk) * a.M + m] = V[(long long)a.recv[kk] * a.M + m];
    }
}

// Fused single pass of one step.  Reads the old state and writes the new
// one into the other buffer set (step parity picks which), so neighbouring
// blocks never see each other's writes within a step.  Block = a strip of
// TJ = blockDim.y - 1 polar columns (thread row ty; ty = TJ is a halo column
// whose new velocity the strip's last stress sigma_tp needs) times a segment
// of seg_rows radial rows, marched outward in r: the lower sigma_rp face and
// the previous row's new velocity stay in registers, the row's new velocity
// goes through shared memory to the left neighbour.  The segment starts one
// row early to recompute the new velocity below it.  Every state value is
// read once and written once per step (plus the halo column and row), 8 M
// bytes per unknown in FP32, against 12 M for the two passes.  The halo
// values are computed by the same arithmetic as their owners' (forcing
// included), so they are bitwise the owners' values.
template <typename T, int VW>
__global__ void __launch_bounds__(kFomThreads) fom_fused_kernel(const FomArgs<T> a) {
    const long long n = a.ctl->step;
    if (n >= a.ctl->nsteps) return;
    const bool odd = (n & 1) != 0;
    const T* __restrict__ Vo = odd ? a.V2 : a.V;
    const T* __restrict__ S1o = odd ? a.S12 : a.S1;
    const T* __restrict__ S2o = odd ? a.S22 : a.S2;
    T* __restrict__ Vn = odd ? a.V : a.V2;
    T* __restrict__ S1n = odd ? a.S1 : a.S12;
    T* __restrict__ S2n = odd ? a.S2 : a.S22;
    const int Nt1 = a.Nt - 1, Nt2 = a.Nt - 2, M = a.M;
    const int TJ = (int)blockDim.y - 1;
    const int nstrip = (Nt1 + TJ - 1) / TJ;
    const int strip = (int)blockIdx.x % nstrip, seg = (int)blockIdx.x / nstrip;
    const int ia = seg * a.seg_rows;
    const int ib = min(a.Nr, ia + a.seg_rows);
    const int ty = threadIdx.y, tx = threadIdx.x;
    const int j = strip * TJ + ty + 1;            // polar index of this thread's column
    const bool act = j <= Nt1;                    // a velocity column
    const bool own = act && ty < TJ;              // written by this block
    const T dt = (T)a.dt;
    const T pp = act ? a.tb.pt_p[j] : T(0), pm = act ? a.tb.pt_m[j] : T(0);
    const bool has_s2 = own && j <= Nt2;
    const T wp = has_s2 ? a.tb.w_p[j] : T(0), wm = has_s2 ? a.tb.w_m[j] : T(0);
    const bool src_col = a.Tper && act && j == a.src_j;
    const T csrc = (T)(a.dt / a.rho);
    extern __shared__ __align__(16) unsigned char fom_smem[];
    T* row = reinterpret_cast<T*>(fom_smem);      // [blockDim.y][blockDim.x * VW] new velocity
    const int i0 = ia > 0 ? ia - 1 : 0;
    const int chunk = (int)blockDim.x * VW;
    for (int mb = 0; mb < M; mb += chunk) {       // same trip count in every thread
        const int m0 = mb + tx * VW;
        const bool lane = act && m0 < M;
        T prev_s1[VW], prev_v[VW];
#pragma unroll
        for (int q = 0; q < VW; ++q) prev_s1[q] = prev_v[q] = T(0);
        if (lane && i0 >= 1) fom_load<T, VW>(S1o + ((size_t)(i0 - 1) * Nt1 + (j - 1)) * M + m0, prev_s1);
        for (int i = i0; i < ib; ++i) {
            T s1u[VW], s2r[VW], s2l[VW], vo[VW], vn[VW];
#pragma unroll
            for (int q = 0; q < VW; ++q) s1u[q] = s2r[q] = s2l[q] = vo[q] = T(0);
            if (lane) {
                if (i + 1 <= a.Nr - 1) fom_load<T, VW>(S1o + ((size_t)i * Nt1 + (j - 1)) * M + m0, s1u);
                if (j <= Nt2) fom_load<T, VW>(S2o + ((size_t)i * Nt2 + (j - 1)) * M + m0, s2r);
                if (j >= 2) fom_load<T, VW>(S2o + ((size_t)i * Nt2 + (j - 2)) * M + m0, s2l);
                fom_load<T, VW>(Vo + ((size_t)i * Nt1 + (j - 1)) * M + m0, vo);
            }
            const T cp = a.tb.cr_p[i], cm = a.tb.cr_m[i], ir = a.tb.inv_rh[i];
#pragma unroll
            for (int q = 0; q < VW; ++q) vn[q] = vo[q] + dt * (cp * s1u[q] - cm * prev_s1[q] + ir * (pp * s2r[q] - pm * s2l[q]));
            if (lane && src_col && i == a.src_i) {
#pragma unroll
                for (int q = 0; q < VW; ++q)
                    vn[q] = vn[q] + csrc * (T)wavelet_eval(a.wavelet, a.ctl->n0 + n, a.dt, a.Tper[m0 + q]);
            }
            if (i >= ia) {                        // block-uniform
                if (own && m0 < M) fom_store<T, VW>(Vn + ((size_t)i * Nt1 + (j - 1)) * M + m0, vn);
#pragma unroll
                for (int q = 0; q < VW; ++q) row[(ty * blockDim.x + tx) * VW + q] = vn[q];
                __syncthreads();
                if (own && m0 < M) {
                    if (i >= 1) {
                        const T qu = a.tb.q_u[i], qd = a.tb.q_d[i];
                        T s1[VW];
#pragma unroll
                        for (int q = 0; q < VW; ++q) s1[q] = prev_s1[q] + dt * (qu * vn[q] - qd * prev_v[q]);
                        fom_store<T, VW>(S1n + ((size_t)(i - 1) * Nt1 + (j - 1)) * M + m0, s1);
                    }
                    if (has_s2) {
                        T s2[VW];
#pragma unroll
                        for (int q = 0; q < VW; ++q) {
                            const T vr = row[((ty + 1) * blockDim.x + tx) * VW + q];
                            s2[q] = s2r[q] + dt * ir * (wp * vr - wm * vn[q]);
                        }
                        fom_store<T, VW>(S2n + ((size_t)i * Nt2 + (j - 1)) * M + m0, s2);
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int q = 0; q < VW; ++q) {
                prev_s1[q] = s1u[q];
                prev_v[q] = vn[q];
            }
        }
    }
}

template <typename T, int VW>
__global__ void __launch_bounds__(kFomThreads) fom_stress_kernel(const FomArgs<T> a) {
    const long long n = a.ctl->step;
    if (n >= a.ctl->nsteps) return;
    const int Nt1 = a.Nt - 1, Nt2 = a.Nt - 2, M = a.M;
    const T dt = (T)a.dt;
    const int gx = (Nt1 + blockDim.y - 1) / blockDim.y;
    const long long tiles1 = (long long)(a.Nr - 1) * gx;   // sigma_rp: i in [1, Nr)
    const long long tiles = tiles1 + (long long)a.Nr * gx;  // then sigma_tp: i in [0, Nr)
    const T* __restrict__ Vv = a.V;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        if (t < tiles1) {
            // sigma_rp (i, j), i in [1, Nr), j in [1, Nt)
            const int i = (int)(t / gx) + 1;
            const int j = (int)(t - (long long)(i - 1) * gx) * blockDim.y + threadIdx.y + 1;
            if (j >= a.Nt) continue;
            const T qu = a.tb.q_u[i], qd = a.tb.q_d[i];
            const T* vu = Vv + ((size_t)i * Nt1 + (j - 1)) * M;        // v (i + 1/2, j)
            const T* vd = Vv + ((size_t)(i - 1) * Nt1 + (j - 1)) * M;  // v (i - 1/2, j)
            T* s = a.S1 + ((size_t)(i - 1) * Nt1 + (j - 1)) * M;
            for (int m = threadIdx.x * VW; m < M; m += blockDim.x * VW) {
                T xu[VW], xd[VW], y[VW];
                fom_load<T, VW>(vu + m, xu);
                fom_load<T, VW>(vd + m, xd);
                fom_load<T, VW>(s + m, y);
#pragma unroll
                for (int q = 0; q < VW; ++q) y[q] = y[q] + dt * (qu * xu[q] - qd * xd[q]);
                fom_store<T, VW>(s + m, y);
            }
        } else {
            // sigma_tp (i + 1/2, j + 1/2), i in [0, Nr), j in [1, Nt - 1)
            const long long t2 = t - tiles1;
            const int i = (int)(t2 / gx);
            const int j = (int)(t2 - (long long)i * gx) * blockDim.y + threadIdx.y + 1;
            if (j >= a.Nt - 1) continue;
            const T ir = a.tb.inv_rh[i], wp = a.tb.w_p[j], wm = a.tb.w_m[j];
            const T* vr = Vv + ((size_t)i * Nt1 + j) * M;              // v (i + 1/2, j + 1)
            const T* vl = Vv + ((size_t)i * Nt1 + (j - 1)) * M;        // v (i + 1/2, j)
            T* s = a.S2 + ((size_t)i * Nt2 + (j - 1)) * M;
            for (int m = threadIdx.x * VW; m < M; m += blockDim.x * VW) {
                T xr[VW], xl[VW], y[VW];
                fom_load<T, VW>(vr + m, xr);
                fom_load<T, VW>(vl + m, xl);
                fom_load<T, VW>(s + m, y);
#pragma unroll
                for (int q = 0; q < VW; ++q) y[q] = y[q] + dt * ir * (wp * xr[q] - wm * xl[q]);
                fom_store<T, VW>(s + m, y);
            }
        }
    }
}

__global__ void fom_tick_kernel(FomCtl* ctl) {
    if (ctl->step < ctl->nsteps) ctl->step = ctl->step + 1;
}

__global__ void fom_set_kernel(FomCtl* ctl, long long nsteps, long long n0) {
    ctl->step = 0;
    ctl->nsteps = nsteps;
    ctl->n0 = n0;
}

}  // namespace romk

using namespace romk;

struct rom_fom_s {
    int Nr = 0, Nt = 0;
    double r_cmb = 0, r_earth = 0, rho = 0, vs = 0, dt = 0;
    void* tables[2] = {nullptr, nullptr};  // [0] f64, [1] f32: 9 arrays of max(Nr, Nt) + 1
    size_t tlen = 0;
    FomCtl* ctl = nullptr;
    cudaStream_t cap = nullptr;
    std::mutex mu;
    std::map<std::vector<long long>, cudaGraphExec_t> graphs;
    int passes = 1;          // 1: fused single pass (default), 2: velocity and stress passes
    void* ws = nullptr;      // second state buffer set of the fused pass
    size_t ws_bytes = 0;
};

namespace {

template <typename T>
FomTables<T> tables_of(const rom_fom_s* f) {
    const T* b = static_cast<const T*>(f->tables[sizeof(T) == 8 ? 0 : 1]);
    const size_t L = f->tlen;
    return {b, b + L, b + 2 * L, b + 3 * L, b + 4 * L, b + 5 * L, b + 6 * L, b + 7 * L, b + 8 * L};
}

template <typename T>
cudaError_t capture_steps(rom_fom_s* f, const FomArgs<T>& a, long long nv, long long ns,
                          cudaGraphExec_t* out) {
    // 16-byte vectors along m when every row starts on a 16-byte boundary
    constexpr int VWIDE = 16 / (int)sizeof(T);
    bool wide = a.M % VWIDE == 0;
    for (const void* p : {(const void*)a.V, (const void*)a.S1, (const void*)a.S2, (const void*)a.V2,
                          (const void*)a.S12, (const void*)a.S22})
        wide = wide && ((uintptr_t)p % 16 == 0);
    const int vw = wide ? VWIDE : 1;
    // block: bx realization groups x by polar points; persistent grid of
    // blocks_per_sm blocks on every SM striding over the tiles
    int bx = 1;
    while (bx * vw < a.M && bx < 32) bx *= 2;
    const int by = kFomThreads / bx;
    const dim3 blk(bx, by, 1);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    auto grid_for = [&](const void* fn, long long tiles) {
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kFomThreads, 0) != cudaSuccess || per < 1)
            per = 1;
        const long long g = (long long)nsm * per;
        return (unsigned)(tiles < g ? (tiles < 1 ? 1 : tiles) : g);
    };
    const long long gx = (a.Nt - 1 + by - 1) / by;
    const void* fv = wide ? (const void*)fom_velocity_kernel<T, VWIDE> : (const void*)fom_velocity_kernel<T, 1>;
    const void* fs = wide ? (const void*)fom_stress_kernel<T, VWIDE> : (const void*)fom_stress_kernel<T, 1>;
    const unsigned gv = grid_for(fv, (long long)a.Nr * gx);
    const unsigned gs = grid_for(fs, (long long)(2 * a.Nr - 1) * gx);
    auto blocks = [&](long long work) {
        const long long b = (work + kFomThreads - 1) / kFomThreads;
        return (unsigned)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
    };
    // fused pass: strips of by - 1 polar columns x segments of seg_rows radial rows
    const unsigned gfused = (unsigned)(((a.Nt - 1 + by - 2) / (by - 1)) * ((a.Nr + a.seg_rows - 1) / a.seg_rows));
    const size_t fsmem = (size_t)by * bx * vw * sizeof(T);
    cudaError_t e = cudaStreamBeginCapture(f->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int s = 0; s < kFomGraphSteps && e == cudaSuccess && a.fused; ++s) {
        if (wide) fom_fused_kernel<T, VWIDE><<<gfused, blk, fsmem, f->cap>>>(a);
        else fom_fused_kernel<T, 1><<<gfused, blk, fsmem, f->cap>>>(a);
        if (a.traces) fom_record_kernel<T><<<blocks((long long)a.nrecv * a.M), kFomThreads, 0, f->cap>>>(a);
        fom_tick_kernel<<<1, 1, 0, f->cap>>>(const_cast<FomCtl*>(a.ctl));
        e = cudaGetLastError();
    }
    for (int s = 0; s < kFomGraphSteps && e == cudaSuccess && !a.fused; ++s) {
        if (wide) fom_velocity_kernel<T, VWIDE><<<gv, blk, 0, f->cap>>>(a);
        else fom_velocity_kernel<T, 1><<<gv, blk, 0, f->cap>>>(a);
        if (a.Tper) fom_source_kernel<T><<<blocks(a.M), kFomThreads, 0, f->cap>>>(a);
        if (a.traces) fom_record_kernel<T><<<blocks((long long)a.nrecv * a.M), kFomThreads, 0, f->cap>>>(a);
        if (wide) fom_stress_kernel<T, VWIDE><<<gs, blk, 0, f->cap>>>(a);
        else fom_stress_kernel<T, 1><<<gs, blk, 0, f->cap>>>(a);
        fom_tick_kernel<<<1, 1, 0, f->cap>>>(const_cast<FomCtl*>(a.ctl));
        e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(f->cap, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

}  // namespace

extern "C" {

rom_status rom_fom_create(int Nr, int Ntheta, double r_cmb, double r_earth, double rho, double vs,
                          double dt, rom_fom_t* out) {
    if (!out) return ROM_E_INVAL;
    *out = nullptr;
    if (Nr < 2 || Nr > 65535 || Ntheta < 3 || !(r_cmb > 0.0) || !(r_earth > r_cmb) || !(rho > 0.0) || !(vs > 0.0) ||
        !(dt > 0.0) || !isfinite(r_earth) || !isfinite(rho) || !isfinite(vs) || !isfinite(dt))
        return ROM_E_INVAL;
    const long long nv = (long long)Nr * (Ntheta - 1);
    if (nv * 3 > (1LL << 31)) return ROM_E_INVAL;  // unknown indices stay below 2^31 per field
    rom_fom_s* f = new (std::nothrow) rom_fom_s();
    if (!f) return ROM_E_NOMEM;
    f->Nr = Nr;
    f->Nt = Ntheta;
    f->r_cmb = r_cmb;
    f->r_earth = r_earth;
    f->rho = rho;
    f->vs = vs;
    f->dt = dt;
    const size_t L = (size_t)(Nr > Ntheta ? Nr : Ntheta) + 1;
    f->tlen = L;
    // the stencil factors in FP64 on the host (see the header comment)
    const double dr = (r_earth - r_cmb) / Nr, dth = 3.14159265358979323846 / Ntheta;
    const double mu = rho * vs * vs;
    std::vector<double> t(9 * L, 0.0);
    double *cr_p = &t[0], *cr_m = &t[L], *inv_rh = &t[2 * L], *pt_p = &t[3 * L], *pt_m = &t[4 * L];
    double *q_u = &t[5 * L], *q_d = &t[6 * L], *w_p = &t[7 * L], *w_m = &t[8 * L];
    for (int i = 0; i < Nr; ++i) {
        const double rm = r_cmb + i * dr, rp = r_cmb + (i + 1) * dr, rh = r_cmb + (i + 0.5) * dr;
        const double rh3 = rh * rh * rh;
        cr_p[i] = i + 1 < Nr ? rp * rp * rp / (rho * rh3 * dr) : 0.0;
        cr_m[i] = i >= 1 ? rm * rm * rm / (rho * rh3 * dr) : 0.0;
        inv_rh[i] = 1.0 / rh;
        if (i >= 1) {
            const double rl = r_cmb + (i - 0.5) * dr;
            q_u[i] = mu * rm / (rh * dr);
            q_d[i] = mu * rm / (rl * dr);
        }
    }
    for (int j = 1; j < Ntheta; ++j) {
        const double s = sin(j * dth), sp = sin((j + 0.5) * dth), sm = sin((j - 0.5) * dth);
        pt_p[j] = j <= Ntheta - 2 ? sp * sp / (rho * s * s * dth) : 0.0;
        pt_m[j] = j >= 2 ? sm * sm / (rho * s * s * dth) : 0.0;
        if (j <= Ntheta - 2) {
            w_p[j] = mu * sp / (sin((j + 1) * dth) * dth);
            w_m[j] = mu * sp / (s * dth);
        }
    }
    std::vector<float> tf(t.begin(), t.end());
    cudaError_t e = cudaMalloc(&f->tables[0], t.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&f->tables[1], tf.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(f->tables[0], t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f->tables[1], tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&f->ctl, sizeof(FomCtl));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(f->tables[0]);
        cudaFree(f->tables[1]);
        cudaFree(f->ctl);
        if (f->cap) cudaStreamDestroy(f->cap);
        delete f;
        set_last_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? ROM_E_NOMEM : ROM_E_CUDA;
    }
    *out = f;
    return ROM_OK;
}

rom_status rom_fom_destroy(rom_fom_t f) {
    if (!f) return ROM_E_INVAL;
    cudaDeviceSynchronize();
    for (auto& kv : f->graphs) cudaGraphExecDestroy(kv.second);
    cudaFree(f->tables[0]);
    cudaFree(f->tables[1]);
    cudaFree(f->ctl);
    cudaFree(f->ws);
    if (f->cap) cudaStreamDestroy(f->cap);
    delete f;
    return ROM_OK;
}

rom_status rom_fom_set_passes(rom_fom_t f, int passes) {
    if (!f || (passes != 1 && passes != 2)) return ROM_E_INVAL;
    std::lock_guard<std::mutex> lk(f->mu);
    f->passes = passes;
    return ROM_OK;
}

rom_status rom_fom_dims(rom_fom_t f, int* nv, int* n1, int* n2) {
    if (!f) return ROM_E_INVAL;
    if (nv) *nv = f->Nr * (f->Nt - 1);
    if (n1) *n1 = (f->Nr - 1) * (f->Nt - 1);
    if (n2) *n2 = f->Nr * (f->Nt - 2);
    return ROM_OK;
}

rom_status rom_fom_run(rom_fom_t f, void* V, void* S1, void* S2, int M, int nsteps, long n0,
                       int src, const void* T, int wavelet, const int* recv, int nrecv, int r,
                       void* traces, int prec, void* stream) {
    if (!f || !V || !S1 || !S2 || M < 1 || nsteps < 0 || n0 < 0) return ROM_E_INVAL;
    if (prec != ROM_FP32 && prec != ROM_FP64) return ROM_E_UNSUPPORTED;
    if (wavelet != ROM_WAVELET_RICKER && wavelet != ROM_WAVELET_GAUSS1) return ROM_E_INVAL;
    const long long nv = (long long)f->Nr * (f->Nt - 1);
    const long long ns = (long long)(f->Nr - 1) * (f->Nt - 1) + (long long)f->Nr * (f->Nt - 2);
    if (src >= nv || (T && src < 0)) return ROM_E_INVAL;
    if (traces && (r < 1 || nrecv < 1 || !recv)) return ROM_E_INVAL;
    if ((long long)M * (nv > ns ? nv : ns) > (1LL << 40)) return ROM_E_INVAL;
    cudaPointerAttributes at;
    for (const void* p : {(const void*)V, (const void*)S1, (const void*)S2, T, (const void*)recv,
                          (const void*)traces}) {
        if (!p) continue;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            set_last_error("rom_fom_run: device buffers only");
            return ROM_E_INVAL;
        }
    }
    if (nsteps == 0) return ROM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(f->mu);
    // the fused pass writes every other step into a second buffer set
    const bool fused = f->passes == 1;
    const size_t es = prec == ROM_FP64 ? 8 : 4;
    const size_t need = (size_t)(nv + ns) * (size_t)M * es + 64;
    if (fused && f->ws_bytes < need) {
        cudaStreamSynchronize(st);
        cudaDeviceSynchronize();
        for (auto& kv : f->graphs) cudaGraphExecDestroy(kv.second);
        f->graphs.clear();
        cudaFree(f->ws);
        f->ws = nullptr;
        f->ws_bytes = 0;
        cudaError_t em = cudaMalloc(&f->ws, need);
        if (em != cudaSuccess) {
            set_last_error(cudaGetErrorString(em));
            return em == cudaErrorMemoryAllocation ? ROM_E_NOMEM : ROM_E_CUDA;
        }
        f->ws_bytes = need;
    }
    char* w = static_cast<char*>(f->ws);
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    void* V2 = fused ? w : nullptr;
    void* S12 = fused ? w + al((size_t)nv * M * es) : nullptr;
    void* S22 = fused ? w + al((size_t)nv * M * es) + al((size_t)(f->Nr - 1) * (f->Nt - 1) * M * es) : nullptr;
    if (fused && (size_t)((char*)S22 - w) + (size_t)f->Nr * (f->Nt - 2) * M * es > f->ws_bytes) {
        // the aligned layout needs a little more than `need`: grow once more
        cudaDeviceSynchronize();
        for (auto& kv : f->graphs) cudaGraphExecDestroy(kv.second);
        f->graphs.clear();
        cudaFree(f->ws);
        f->ws_bytes = 0;
        const size_t need2 = need + 1024;
        cudaError_t em = cudaMalloc(&f->ws, need2);
        if (em != cudaSuccess) {
            f->ws = nullptr;
            set_last_error(cudaGetErrorString(em));
            return em == cudaErrorMemoryAllocation ? ROM_E_NOMEM : ROM_E_CUDA;
        }
        f->ws_bytes = need2;
        w = static_cast<char*>(f->ws);
        V2 = w;
        S12 = w + al((size_t)nv * M * es);
        S22 = w + al((size_t)nv * M * es) + al((size_t)(f->Nr - 1) * (f->Nt - 1) * M * es);
    }
    const int src_i = src >= 0 ? (int)(src / (f->Nt - 1)) : -1;
    const int src_j = src >= 0 ? (int)(src % (f->Nt - 1)) + 1 : -1;
    const std::vector<long long> key = {(long long)(uintptr_t)V, (long long)(uintptr_t)S1,
                                        (long long)(uintptr_t)S2, M, src, (long long)(uintptr_t)T,
                                        wavelet, (long long)(uintptr_t)recv, nrecv, traces ? r : 0,
                                        (long long)(uintptr_t)traces, prec, fused,
                                        (long long)(uintptr_t)V2};
    auto it = f->graphs.find(key);
    if (it == f->graphs.end()) {
        cudaGraphExec_t ge = nullptr;
        cudaError_t e;
        if (prec == ROM_FP64) {
            FomArgs<double> a = {tables_of<double>(f), static_cast<double*>(V), static_cast<double*>(S1),
                                 static_cast<double*>(S2), static_cast<const double*>(T), recv,
                                 static_cast<double*>(traces), f->ctl, f->Nr, f->Nt, M, src, nrecv,
                                 traces ? r : 1, wavelet, f->dt, f->rho,
                                 static_cast<double*>(V2), static_cast<double*>(S12), static_cast<double*>(S22),
                                 fused ? 1 : 0, src_i, src_j, kFomSegRows};
            e = capture_steps<double>(f, a, nv, ns, &ge);
        } else {
            FomArgs<float> a = {tables_of<float>(f), static_cast<float*>(V), static_cast<float*>(S1),
                                static_cast<float*>(S2), static_cast<const float*>(T), recv,
                                static_cast<float*>(traces), f->ctl, f->Nr, f->Nt, M, src, nrecv,
                                traces ? r : 1, wavelet, f->dt, f->rho,
                                static_cast<float*>(V2), static_cast<float*>(S12), static_cast<float*>(S22),
                                fused ? 1 : 0, src_i, src_j, kFomSegRows};
            e = capture_steps<float>(f, a, nv, ns, &ge);
        }
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return ROM_E_CUDA;
        }
        if (f->graphs.size() >= 16) {  // keep the cache small
            cudaStreamSynchronize(st);
            for (auto& kv : f->graphs) cudaGraphExecDestroy(kv.second);
            f->graphs.clear();
        }
        it = f->graphs.emplace(key, ge).first;
    }
    fom_set_kernel<<<1, 1, 0, st>>>(f->ctl, nsteps, n0);
    cudaError_t e = cudaGetLastError();
    const int reps = (nsteps + kFomGraphSteps - 1) / kFomGraphSteps;
    for (int k = 0; k < reps && e == cudaSuccess; ++k) e = cudaGraphLaunch(it->second, st);
    if (e == cudaSuccess && fused && (nsteps & 1)) {
        // an odd number of fused steps leaves the result in the second buffer set
        e = cudaMemcpyAsync(V, V2, (size_t)nv * M * es, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S1, S12, (size_t)(f->Nr - 1) * (f->Nt - 1) * M * es, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S2, S22, (size_t)f->Nr * (f->Nt - 2) * M * es, cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return ROM_E_CUDA;
    }
    return ROM_OK;
}

}  // extern "C"
