// Rank-1 ensemble GEMV kernel, FP64 power iteration, FP64 error norms and
// operator layout copies.
#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "rom_internal.h"

namespace romk {

// ---------------------------------------------------------------------------
// Rank-1 ensemble: one CTA advances one realization (Eq. (rom_ode), Sec. 2.2)
// through all steps.  Each half-step is a GEMV that streams the whole
// column-major operator from memory: thread (row group gq, k-split ks) reads
// four consecutive rows of every column k = ks (mod KS) as one 16-byte load,
// so a warp reads contiguous 512-byte segments.  No operator value is reused
// across realizations: this is the bandwidth-bound rank-1 formulation of
// Sec. 2.3, run M times side by side.
//
// The stream is latency-bound: its rate is the bytes each SM keeps in flight,
// i.e. the loads of its resident warps.  The CTA therefore takes NT = 256, 512
// or 1024 threads, the most that still keeps all M CTAs resident in one wave
// (64 registers a thread, so NT * CTAs per SM <= 1024), with at most 8
// k-splits so that the per-row sum of the partials stays short.  Co-resident
// CTAs read the same operator lines at about the same time and share them
// in L1.
// ---------------------------------------------------------------------------
constexpr int kEnsMaxSplit = 8;

__host__ __device__ inline int ens_ksplit(int NT, int Kp) {
    const int G = Kp / 4;
    const int ks = NT / G;
    return ks < 1 ? 1 : (ks > kEnsMaxSplit ? kEnsMaxSplit : ks);
}

// XR: add the reduced reference state (a template flag, so that runs without
// it compile to the code they had without it).
template <typename T, int NT, bool XR>
__global__ void __launch_bounds__(NT, 1024 / NT) rank1_ensemble_kernel(const Rank1EnsArgs a) {
    const int m = blockIdx.x;
    const int Kp = a.Kp;
    const int G = Kp / 4;                 // row groups of 4
    const int KS = ens_ksplit(NT, Kp);
    const int tid = threadIdx.x;
    const int gq = tid % G;
    const int ks = tid / G;
    const bool act = ks < KS;
    extern __shared__ __align__(16) unsigned char smem[];
    T* v = reinterpret_cast<T*>(smem);
    T* s = v + Kp;
    T* part = s + Kp;  // KS x Kp partial sums
    const T* Vin = static_cast<const T*>(a.V);
    const T* Sin = static_cast<const T*>(a.S);
    for (int k = tid; k < Kp; k += NT) {
        v[k] = k < a.Kv ? Vin[(size_t)m * a.Kv + k] : T(0);
        s[k] = k < a.Ks ? Sin[(size_t)m * a.Ks + k] : T(0);
    }
    const T* __restrict__ Avs = static_cast<const T*>(a.Avs_cm);
    const T* __restrict__ Asv = static_cast<const T*>(a.Asv_cm);
    const T* __restrict__ gp = static_cast<const T*>(a.g_p);
    const T* __restrict__ Cc = static_cast<const T*>(a.C_cm);
    const T Tm = a.Tper ? static_cast<const T*>(a.Tper)[m] : T(1);
    const T dt = (T)a.dt;
    // reduced reference state (velocity, stress parts) or null
    const T* XrV = static_cast<const T*>(a.Xv);
    const T* XrS = static_cast<const T*>(a.Xs);
    float cv[4] = {0.f, 0.f, 0.f, 0.f}, cs[4] = {0.f, 0.f, 0.f, 0.f};
    T* traces = static_cast<T*>(a.traces);
    __syncthreads();
    for (int n = 0; n < a.nsteps; ++n) {
        const T f = a.Tper ? (T)wavelet_eval(a.wavelet, (long long)a.n0 + n, a.dt, Tm) : T(0);
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            const T* A = half == 0 ? Avs : Asv;
            const T* x = half == 0 ? s : v;
            T* y = half == 0 ? v : s;
            T acc[4] = {T(0), T(0), T(0), T(0)};
            if (act) {
#pragma unroll 4
                for (int k = ks; k < Kp; k += KS) {
                    T av[4];
                    load4_ro(A + (size_t)k * Kp + 4 * gq, av);
                    const T xk = x[k];
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] += av[q] * xk;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) part[(size_t)ks * Kp + 4 * gq + q] = acc[q];
            }
            __syncthreads();
            if (act && ks == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int row = 4 * gq + q;
                    T tot = part[row];
                    for (int k2 = 1; k2 < KS; ++k2) tot += part[(size_t)k2 * Kp + row];
                    if (half == 0) tot += gp[row] * f;
                    if constexpr (XR) {
                        const T* xh = half == 0 ? XrV : XrS;
                        const int kh = half == 0 ? a.Kv : a.Ks;
                        if (xh && row < kh) tot += xh[(size_t)m * kh + row];
                    }
                    const T inc = tot * dt;
                    if constexpr (sizeof(T) == 4) {
                        y[row] = kahan_add(y[row], inc, half == 0 ? cv[q] : cs[q]);
                    } else {
                        y[row] = y[row] + inc;
                    }
                }
            }
            __syncthreads();
        }
        if (traces && ((n + 1) % a.r) == 0) {
            const int rec = (n + 1) / a.r - 1;
            for (int jr = tid; jr < a.R; jr += NT) {
                T acc = T(0);
                for (int k = 0; k < a.Kv; ++k) acc += Cc[(size_t)k * a.R + jr] * v[k];
                traces[((size_t)rec * a.M + m) * a.R + jr] = acc;
            }
        }
    }
    T* Vout = static_cast<T*>(a.V);
    T* Sout = static_cast<T*>(a.S);
    int bad = 0;
    for (int k = tid; k < Kp; k += NT) {
        if (k < a.Kv) { Vout[(size_t)m * a.Kv + k] = v[k]; bad |= !is_finite(v[k]); }
        if (k < a.Ks) { Sout[(size_t)m * a.Ks + k] = s[k]; bad |= !is_finite(s[k]); }
    }
    bad = __syncthreads_or(bad);
    if (bad && tid == 0 && a.status) atomicCAS(a.status, 0, 6 /* ROM_E_NONFINITE */);
}

template <typename T, int NT>
static cudaError_t launch_ens_nt(const Rank1EnsArgs& a, cudaStream_t st) {
    const int KS = ens_ksplit(NT, a.Kp);
    const size_t smem = sizeof(T) * (size_t)(2 * a.Kp + KS * a.Kp);
    auto fn = (a.Xv || a.Xs) ? rank1_ensemble_kernel<T, NT, true> : rank1_ensemble_kernel<T, NT, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<a.M, NT, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_ens(const Rank1EnsArgs& a, cudaStream_t st) {
    if (a.Kp <= 0 || a.Kp % 64 != 0 || a.Kp > 1024 || a.M <= 0) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) return cudaErrorInvalidDevice;
    int NT = a.M <= nsm ? 1024 : (a.M <= 2 * nsm ? 512 : 256);
    while (NT > 256 && NT / (a.Kp / 4) > kEnsMaxSplit) NT /= 2;
    if (NT == 1024) return launch_ens_nt<T, 1024>(a, st);
    if (NT == 512) return launch_ens_nt<T, 512>(a, st);
    return launch_ens_nt<T, 256>(a, st);
}

cudaError_t launch_rank1_ensemble_f32(const Rank1EnsArgs& a, cudaStream_t st) { return launch_ens<float>(a, st); }
cudaError_t launch_rank1_ensemble_f64(const Rank1EnsArgs& a, cudaStream_t st) { return launch_ens<double>(a, st); }

// ---------------------------------------------------------------------------
// FP64 power iteration pieces (dt-stability check).
// ---------------------------------------------------------------------------
// y = A x, A row-major rows x cols with leading dimension ld; one warp per row.
__global__ void matvec_f64_kernel(const double* __restrict__ A, int rows, int cols, int ld,
                                  const double* __restrict__ x, double* __restrict__ y) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= rows) return;
    double acc = 0.0;
    for (int k = lane; k < cols; k += 32) acc = __fma_rn(A[(size_t)warp * ld + k], x[k], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[warp] = acc;
}

cudaError_t launch_matvec_f64(const double* A_rm, int rows, int cols, int ld, const double* x,
                              double* y, cudaStream_t st) {
    const int threads = 256;
    const int blocks = (rows * 32 + threads - 1) / threads;
    matvec_f64_kernel<<<blocks, threads, 0, st>>>(A_rm, rows, cols, ld, x, y);
    return cudaGetLastError();
}

// One block: lam = |x.y| / x.x, x <- y / ||y||, lam_out[it] = lam.
__global__ void power_step_kernel(const double* __restrict__ y, double* __restrict__ x, int n,
                                  double* __restrict__ lam_out, int it) {
    __shared__ double red[3][32];
    double xy = 0.0, xx = 0.0, yy = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        xy += x[i] * y[i];
        xx += x[i] * x[i];
        yy += y[i] * y[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        xy += __shfl_xor_sync(0xffffffffu, xy, o);
        xx += __shfl_xor_sync(0xffffffffu, xx, o);
        yy += __shfl_xor_sync(0xffffffffu, yy, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = xy; red[1][w] = xx; red[2][w] = yy; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        xy = l < nw ? red[0][l] : 0.0;
        xx = l < nw ? red[1][l] : 0.0;
        yy = l < nw ? red[2][l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            xy += __shfl_xor_sync(0xffffffffu, xy, o);
            xx += __shfl_xor_sync(0xffffffffu, xx, o);
            yy += __shfl_xor_sync(0xffffffffu, yy, o);
        }
        if (l == 0) { red[0][0] = xy; red[1][0] = xx; red[2][0] = yy; }
    }
    __syncthreads();
    xy = red[0][0];
    xx = red[1][0];
    yy = red[2][0];
    const double inv = yy > 0.0 ? 1.0 / sqrt(yy) : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = y[i] * inv;
    if (threadIdx.x == 0) lam_out[it] = xx > 0.0 ? fabs(xy) / xx : 0.0;
}

cudaError_t launch_power_step(const double* y, double* x, int n, double* lam_out, int it,
                              cudaStream_t st) {
    power_step_kernel<<<1, 1024, 0, st>>>(y, x, n, lam_out, it);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 relative-error accumulation: acc2[0] += sum (x - ref)^2, acc2[1] += sum ref^2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double load_as_f64(const void* p, int dt, size_t i) {
    return dt == 0 ? static_cast<const double*>(p)[i] : (double)static_cast<const float*>(p)[i];
}

__global__ void rel_l2_kernel(const void* __restrict__ x, int xd, const void* __restrict__ ref,
                              int rd, size_t n, double* acc2) {
    double d2 = 0.0, r2 = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double xv = load_as_f64(x, xd, i), rv = load_as_f64(ref, rd, i);
        d2 += (xv - rv) * (xv - rv);
        r2 += rv * rv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    }
    __shared__ double red[2][32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = d2; red[1][w] = r2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += red[0][i]; b += red[1][i]; }
        atomicAdd(&acc2[0], a);
        atomicAdd(&acc2[1], b);
    }
}

cudaError_t launch_rel_l2(const void* x, int xd, const void* ref, int rd, size_t n, double* acc2,
                          cudaStream_t st) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 1216) blocks = 1216;  // 8 per SM on 152 SMs
    if (blocks == 0) blocks = 1;
    rel_l2_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, xd, ref, rd, n, acc2);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Zero-padded, re-laid-out copies of a column-major rows x cols source.
// ---------------------------------------------------------------------------
__global__ void pad_copy_kernel(const void* __restrict__ src, int sd, int rows, int cols, int Pr,
                                int Pc, int row_major_out, void* __restrict__ dst, int dd) {
    const size_t total = (size_t)Pr * Pc;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        int i, k;
        if (row_major_out) { i = (int)(idx / Pc); k = (int)(idx % Pc); }
        else { k = (int)(idx / Pr); i = (int)(idx % Pr); }
        double val = 0.0;
        if (i < rows && k < cols) val = load_as_f64(src, sd, (size_t)k * rows + i);
        if (dd == 0) static_cast<double*>(dst)[idx] = val;
        else static_cast<float*>(dst)[idx] = (float)val;
    }
}

cudaError_t launch_pad_copy(const void* src, int src_dtype, int rows, int cols, int Pr, int Pc,
                            bool row_major_out, void* dst, int dst_dtype, cudaStream_t st) {
    const size_t total = (size_t)Pr * Pc;
    size_t blocks = (total + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks == 0) return cudaSuccess;
    pad_copy_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, src_dtype, rows, cols, Pr, Pc,
                                                        row_major_out ? 1 : 0, dst, dst_dtype);
    return cudaGetLastError();
}

}  // namespace romk
