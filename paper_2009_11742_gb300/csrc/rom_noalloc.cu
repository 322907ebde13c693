// rom_spectral_radius_noalloc: the FP64 power iteration of rom_create for
// callers that must not allocate device memory (see include/rom.h).
//
// Its work vectors live in one file-scope device array instead of cudaMalloc'd
// buffers.  Host code may not use the array's name as a device address, so
// the address is taken once per device with cudaGetSymbolAddress and handed to
// the kernels.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "rom_internal.h"

namespace {

// Largest Kv / Ks the allocation-free entry point accepts.
constexpr int kNoallocMaxK = 4096;
// Estimates read back per host check of convergence.
constexpr int kNoallocChunk = 64;
// x (Kv), z (Ks), y (Kv) and a ring of kNoallocChunk eigenvalue estimates.
constexpr size_t kNoallocDoubles = 3 * (size_t)kNoallocMaxK + kNoallocChunk + 1;

// Shared by every call on a device; kept until the process exits.
static __device__ __align__(256) double g_power_scratch[kNoallocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

__global__ void fill_start_vector(double* x, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = 1.0 / sqrt((double)n);
}

// True for device (or managed) memory that the current device `dev` can read
// directly: plain device memory must belong to `dev` itself, since a peer's
// buffer would need peer access, which this entry point does not set up.
bool is_local_device_pointer(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" rom_status rom_spectral_radius_noalloc(const double* Avs, const double* Asv, int Kv,
                                                  int Ks, double* rho, void* stream) {
    if (!Avs || !Asv || !rho || Kv < 1 || Ks < 1) return ROM_E_INVAL;
    // the work area is fixed: larger operators are refused, never truncated
    if (Kv > kNoallocMaxK || Ks > kNoallocMaxK) return ROM_E_INVAL;
    int dev = 0;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return romk::cuda_fail(de, "rom_spectral_radius_noalloc");
    if (dev < 0 || dev >= kMaxDevices) {
        romk::set_last_error("rom_spectral_radius_noalloc: device ordinal beyond the supported 64");
        return ROM_E_CUDA;
    }
    if (!is_local_device_pointer(Avs, dev) || !is_local_device_pointer(Asv, dev)) return ROM_E_INVAL;
    double* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_power_scratch);
            if (e != cudaSuccess) return romk::cuda_fail(e, "rom_spectral_radius_noalloc setup");
            if (!p) {
                romk::set_last_error("rom_spectral_radius_noalloc setup: null symbol address");
                return ROM_E_CUDA;
            }
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        base = g_scratch_addr[dev];
    }
    double* x = base;
    double* z = base + kNoallocMaxK;
    double* y = base + 2 * kNoallocMaxK;
    double* lam = base + 3 * kNoallocMaxK;  // ring of kNoallocChunk + 1 estimates
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // The caller's column-major Avs (Kv x Ks) is the row-major Avs^T, and the
    // column-major Asv the row-major Asv^T, so the iteration below runs on
    // (Avs Asv)^T = Asv^T Avs^T, which has the same eigenvalues as Avs Asv.
    fill_start_vector<<<(Kv + 255) / 256, 256, 0, st>>>(x, Kv);
    cudaError_t e = cudaGetLastError();
    const int max_iter = 20000;
    const double tol = 1e-14;
    double hl[kNoallocChunk];
    double cur = 0.0, prev = -1.0;
    bool converged = false;
    for (int it0 = 1; e == cudaSuccess && it0 <= max_iter; it0 += kNoallocChunk) {
        const int it1 = it0 + kNoallocChunk - 1 <= max_iter ? it0 + kNoallocChunk - 1 : max_iter;
        for (int it = it0; it <= it1 && e == cudaSuccess; ++it) {
            e = romk::launch_matvec_f64(Avs, Ks, Kv, Kv, x, z, st);        // z = Avs^T x
            if (e == cudaSuccess) e = romk::launch_matvec_f64(Asv, Kv, Ks, Ks, z, y, st);  // y = Asv^T z
            if (e == cudaSuccess) e = romk::launch_power_step(y, x, Kv, lam, it - it0, st);
        }
        if (e != cudaSuccess) break;
        const int cnt = it1 - it0 + 1;
        e = cudaMemcpyAsync(hl, lam, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        for (int i = 0; i < cnt; ++i) {
            cur = hl[i];
            if (prev >= 0.0 && fabs(cur - prev) <= tol * cur) { converged = true; break; }
            prev = cur;
        }
        if (converged) break;
    }
    if (e != cudaSuccess) return romk::cuda_fail(e, "rom_spectral_radius_noalloc");
    *rho = sqrt(cur);
    // not converged: the estimate is only a lower bound on rho
    return converged ? ROM_OK : ROM_E_NOCONV;
}
