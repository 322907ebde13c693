// C ABI of librom: handles, argument checking, staging of host buffers and
// dispatch to the kernels.  Declarations and contracts: include/rom.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "rom_internal.h"

using namespace romk;

namespace {

thread_local char g_last_error[256] = "";

}  // namespace

void romk::set_last_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

rom_status romk::cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    // clear the runtime's record of a non-sticky error (a failed allocation),
    // so that a later call's launch check does not report it again
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? ROM_E_NOMEM : ROM_E_CUDA;
}

namespace {

#define ROM_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int pad64(int k) { return ((k + 63) / 64) * 64; }

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t ensure(size_t n) {
        if (n <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) bytes = n;
        return e;
    }
};

}  // namespace

struct rom_s {
    int device = 0;
    int Kv = 0, Ks = 0, R = 0, Kp = 0;
    double dt = 0.0, rho = 0.0;
    // Operator copies, zero padded to Kp x Kp.  rm: row-major, cm: column-major.
    void* Avs_rm[2] = {nullptr, nullptr};  // [0] = f64, [1] = f32
    void* Asv_rm[2] = {nullptr, nullptr};
    void* Avs_cm[2] = {nullptr, nullptr};
    void* Asv_cm[2] = {nullptr, nullptr};
    void* g_p[2] = {nullptr, nullptr};
    void* C_rm[2] = {nullptr, nullptr};  // R x Kp row-major
    void* C_cm[2] = {nullptr, nullptr};  // Kp x R  (column j = row j of C)
    int* status = nullptr;
    double* scalar = nullptr;  // small device scratch (rank-1 period)
    DevBuf stage;              // staging of host buffers
    // tensor-core path (prepared on first use of a split precision)
    int Kp_tc = 0;
    void* tc_ops[6][2] = {};   // [prec][0: Avs, 1: Asv] pre-split, pre-swizzled tiles
    float* g_tc = nullptr;     // Kp_tc
    float* C_tc = nullptr;     // R x Kp_tc
    DevBuf tc_ws;              // exchange tiles + Kahan carries of one call
    std::map<std::tuple<int, int, int>, TcPlan> tc_plans;
    int tc_cols = 0;           // columns per block pinned by rom_set_tc_columns (0 = planner)
    std::map<std::tuple<int, int, int, int, int>, Rank2Plan> plans;
    std::mutex mu;
    int kernel_choice = 0;  // ROM_KERNEL_AUTO
    long long wait_limit = 4000000000LL;  // device wait bound in SM clock cycles (~2 s)
    int inject_stall = 0;
    int wavelet = ROM_WAVELET_RICKER;  // source signal of the periods T
    // plans chosen by rom_autotune, per (precision, M): used while the kernel
    // and tensor-core column choices are on automatic
    std::map<std::pair<int, int>, Rank2Plan> tuned;
    std::map<std::pair<int, int>, TcPlan> tuned_tc;
    // reduced reference state (rom_set_reference): [0] f64, [1] f32 copies of
    // the velocity (Kv x xref_M) and stress (Ks x xref_M) parts; xref_M = 0: none
    void* xref[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int xref_M = 0;
    // streaming companion of the FP32 split kernel (rom_set_companion):
    // comp_cs 0 = the planner's choice, -1 = off, 2 / 4 = pinned with
    // comp_cols columns; a private stream and two events fork it off the
    // caller's stream and join it back
    int comp_cs = 0, comp_cols = 0;
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

void free_handle(rom_s* h) {
    if (!h) return;
    for (int t = 0; t < 2; ++t) {
        cudaFree(h->Avs_rm[t]);
        cudaFree(h->Asv_rm[t]);
        cudaFree(h->Avs_cm[t]);
        cudaFree(h->Asv_cm[t]);
        cudaFree(h->g_p[t]);
        cudaFree(h->C_rm[t]);
        cudaFree(h->C_cm[t]);
    }
    for (int p = 0; p < 6; ++p) {
        cudaFree(h->tc_ops[p][0]);
        cudaFree(h->tc_ops[p][1]);
    }
    cudaFree(h->g_tc);
    cudaFree(h->C_tc);
    cudaFree(h->status);
    cudaFree(h->scalar);
    for (int t = 0; t < 2; ++t) {
        cudaFree(h->xref[t][0]);
        cudaFree(h->xref[t][1]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->aux) cudaStreamDestroy(h->aux);
    delete h;
}

// Reference-state pointers of precision copy t (0 f64, 1 f32) for a run over
// M columns; ROM_E_INVAL when one is set for another number of columns.
rom_status xref_for(const rom_s* h, int t, int M, const void** Xv, const void** Xs) {
    *Xv = nullptr;
    *Xs = nullptr;
    if (h->xref_M == 0) return ROM_OK;
    if (M != h->xref_M) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "the reference state has %d columns, the run %d", h->xref_M, M);
        return ROM_E_INVAL;
    }
    *Xv = h->xref[t][0];
    *Xs = h->xref[t][1];
    return ROM_OK;
}

// FP64 power iteration for rho(Avs Asv) on the GPU.
rom_status power_iteration(rom_s* h, double* rho_out) {
    const int Kv = h->Kv, Ks = h->Ks, Kp = h->Kp;
    const int max_iter = 20000, chunk = 64;
    const double tol = 1e-14;
    double *x = nullptr, *z = nullptr, *y = nullptr, *lam = nullptr;
    cudaError_t e = cudaMalloc(&x, sizeof(double) * Kp);
    if (e == cudaSuccess) e = cudaMalloc(&z, sizeof(double) * Kp);
    if (e == cudaSuccess) e = cudaMalloc(&y, sizeof(double) * Kp);
    if (e == cudaSuccess) e = cudaMalloc(&lam, sizeof(double) * (max_iter + 1));
    if (e != cudaSuccess) {
        cudaFree(x); cudaFree(z); cudaFree(y); cudaFree(lam);
        return cuda_fail(e, "power_iteration alloc");
    }
    std::vector<double> hx(Kv, 1.0 / sqrt((double)Kv));
    std::vector<double> hl(chunk);
    rom_status st = ROM_OK;
    double cur = 0.0, prev = -1.0;
    bool converged = false;
    e = cudaMemcpy(x, hx.data(), sizeof(double) * Kv, cudaMemcpyHostToDevice);
    for (int it0 = 1; e == cudaSuccess && it0 <= max_iter; it0 += chunk) {
        const int it1 = it0 + chunk - 1 <= max_iter ? it0 + chunk - 1 : max_iter;
        for (int it = it0; it <= it1 && e == cudaSuccess; ++it) {
            e = launch_matvec_f64(static_cast<const double*>(h->Asv_rm[0]), Ks, Kv, Kp, x, z, 0);
            if (e == cudaSuccess)
                e = launch_matvec_f64(static_cast<const double*>(h->Avs_rm[0]), Kv, Ks, Kp, z, y, 0);
            if (e == cudaSuccess) e = launch_power_step(y, x, Kv, lam, it, 0);
        }
        if (e != cudaSuccess) break;
        const int cnt = it1 - it0 + 1;
        e = cudaMemcpy(hl.data(), lam + it0, sizeof(double) * cnt, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        for (int i = 0; i < cnt; ++i) {
            cur = hl[i];
            if (prev >= 0.0 && fabs(cur - prev) <= tol * cur) { converged = true; break; }
            prev = cur;
        }
        if (converged) break;
    }
    if (e != cudaSuccess) st = cuda_fail(e, "power_iteration");
    else if (!converged) st = ROM_E_NOCONV;
    cudaFree(x); cudaFree(z); cudaFree(y); cudaFree(lam);
    *rho_out = sqrt(cur);
    return st;
}

bool valid_prec(int prec) { return prec >= ROM_FP64 && prec <= ROM_BF16S; }
bool tc_prec(int prec) {
    return prec == ROM_TF32X3 || prec == ROM_BF16X3 || prec == ROM_BF16 || prec == ROM_BF16S;
}

// Forget cached batched graphs, and the tuned schedules of job lists, that
// reference handle h (defined with them below).
void drop_batch_graphs(rom_s* h);
// Forget cached rank-3 operator tables that reference handle h (defined below).
void drop_group_tables(rom_s* h);

}  // namespace

extern "C" {

int rom_version(void) { return 100; }

const char* rom_last_error(void) { return g_last_error; }

const char* rom_status_string(rom_status s) {
    switch (s) {
        case ROM_OK: return "ROM_OK";
        case ROM_E_INVAL: return "ROM_E_INVAL: invalid argument";
        case ROM_E_NOMEM: return "ROM_E_NOMEM: allocation failed";
        case ROM_E_CUDA: return "ROM_E_CUDA: CUDA runtime error";
        case ROM_E_UNSTABLE: return "ROM_E_UNSTABLE: dt * rho >= 2";
        case ROM_E_TIMEOUT: return "ROM_E_TIMEOUT: device wait ran out";
        case ROM_E_NONFINITE: return "ROM_E_NONFINITE: non-finite state";
        case ROM_E_UNSUPPORTED: return "ROM_E_UNSUPPORTED: shape/precision not provided";
        case ROM_E_NOCONV: return "ROM_E_NOCONV: power iteration did not converge";
    }
    return "unknown rom_status";
}

rom_status rom_create(const void* Avs, const void* Asv, const void* g, const void* C, int Kv,
                      int Ks, int R, double dt, int in_dtype, rom_t* out, double* rho_out) {
    if (!out) return ROM_E_INVAL;
    *out = nullptr;
    if (!Avs || !Asv || !g || Kv < 1 || Ks < 1 || Kv > 1024 || Ks > 1024 || R < 0 || R > 1024 ||
        (R > 0 && !C) || !(dt > 0.0) || !isfinite(dt) ||
        (in_dtype != ROM_IN_F64 && in_dtype != ROM_IN_F32))
        return ROM_E_INVAL;
    rom_s* h = new (std::nothrow) rom_s();
    if (!h) return ROM_E_NOMEM;
    cudaGetDevice(&h->device);
    h->Kv = Kv;
    h->Ks = Ks;
    h->R = R;
    h->dt = dt;
    h->Kp = pad64(Kv > Ks ? Kv : Ks);
    const int Kp = h->Kp;
    const size_t es = in_dtype == ROM_IN_F64 ? 8 : 4;
    // bring the inputs to the device (temporary copies when they are host data)
    const void* src[4] = {Avs, Asv, g, C};
    const size_t cnt[4] = {(size_t)Kv * Ks, (size_t)Ks * Kv, (size_t)Kv, (size_t)R * Kv};
    void* tmp[4] = {nullptr, nullptr, nullptr, nullptr};
    const void* dsrc[4] = {nullptr, nullptr, nullptr, nullptr};
    rom_status st = ROM_OK;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
        if (!src[i] || cnt[i] == 0) continue;
        if (is_device_ptr(src[i])) {
            dsrc[i] = src[i];
        } else {
            e = cudaMalloc(&tmp[i], cnt[i] * es);
            if (e == cudaSuccess) e = cudaMemcpy(tmp[i], src[i], cnt[i] * es, cudaMemcpyHostToDevice);
            dsrc[i] = tmp[i];
        }
    }
    const size_t kk = (size_t)Kp * Kp;
    for (int t = 0; t < 2 && e == cudaSuccess; ++t) {
        const size_t el = t == 0 ? 8 : 4;
        e = cudaMalloc(&h->Avs_rm[t], kk * el);
        if (e == cudaSuccess) e = cudaMalloc(&h->Asv_rm[t], kk * el);
        if (e == cudaSuccess) e = cudaMalloc(&h->Avs_cm[t], kk * el);
        if (e == cudaSuccess) e = cudaMalloc(&h->Asv_cm[t], kk * el);
        if (e == cudaSuccess) e = cudaMalloc(&h->g_p[t], (size_t)Kp * el);
        if (e == cudaSuccess && R > 0) e = cudaMalloc(&h->C_rm[t], (size_t)R * Kp * el);
        if (e == cudaSuccess && R > 0) e = cudaMalloc(&h->C_cm[t], (size_t)R * Kp * el);
        const int sd = in_dtype == ROM_IN_F64 ? 0 : 1;
        if (e == cudaSuccess) e = launch_pad_copy(dsrc[0], sd, Kv, Ks, Kp, Kp, true, h->Avs_rm[t], t, 0);
        if (e == cudaSuccess) e = launch_pad_copy(dsrc[1], sd, Ks, Kv, Kp, Kp, true, h->Asv_rm[t], t, 0);
        if (e == cudaSuccess) e = launch_pad_copy(dsrc[0], sd, Kv, Ks, Kp, Kp, false, h->Avs_cm[t], t, 0);
        if (e == cudaSuccess) e = launch_pad_copy(dsrc[1], sd, Ks, Kv, Kp, Kp, false, h->Asv_cm[t], t, 0);
        if (e == cudaSuccess) e = launch_pad_copy(dsrc[2], sd, Kv, 1, Kp, 1, false, h->g_p[t], t, 0);
        if (e == cudaSuccess && R > 0) e = launch_pad_copy(dsrc[3], sd, R, Kv, R, Kp, true, h->C_rm[t], t, 0);
        if (e == cudaSuccess && R > 0) e = launch_pad_copy(dsrc[3], sd, R, Kv, R, Kp, false, h->C_cm[t], t, 0);
    }
    if (e == cudaSuccess) e = cudaMalloc(&h->status, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&h->scalar, 64);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    for (int i = 0; i < 4; ++i) cudaFree(tmp[i]);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "rom_create");
        free_handle(h);
        return st;
    }
    double rho = 0.0;
    st = power_iteration(h, &rho);
    if (st != ROM_OK) {
        // not converged: the estimate is only a lower bound, so no handle
        if (st == ROM_E_NOCONV && rho_out) *rho_out = rho;
        free_handle(h);
        return st;
    }
    h->rho = rho;
    if (rho_out) *rho_out = rho;
    if (!(dt * rho < 2.0)) {
        free_handle(h);
        return ROM_E_UNSTABLE;
    }
    *out = h;
    return ROM_OK;
}

rom_status rom_destroy(rom_t h) {
    if (!h) return ROM_E_INVAL;
    cudaDeviceSynchronize();
    drop_batch_graphs(h);
    drop_group_tables(h);
    free_handle(h);
    return ROM_OK;
}

rom_status rom_spectral_radius(rom_t h, double* rho) {
    if (!h || !rho) return ROM_E_INVAL;
    *rho = h->rho;
    return ROM_OK;
}

rom_status rom_get_dims(rom_t h, int* Kv, int* Ks, int* R, double* dt) {
    if (!h) return ROM_E_INVAL;
    if (Kv) *Kv = h->Kv;
    if (Ks) *Ks = h->Ks;
    if (R) *R = h->R;
    if (dt) *dt = h->dt;
    return ROM_OK;
}

rom_status rom_sync_status(rom_t h, rom_status* device_status) {
    if (!h || !device_status) return ROM_E_INVAL;
    ROM_CUDA(cudaDeviceSynchronize());
    int v = 0;
    ROM_CUDA(cudaMemcpy(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    ROM_CUDA(cudaMemset(h->status, 0, sizeof(int)));
    *device_status = (rom_status)v;
    return ROM_OK;
}

}  // extern "C"

namespace {

// Device buffers of one integration call (caller's or staged).
struct RunBufs {
    void *V, *S, *T, *ftab, *compV, *compS, *traces;
};

rom_status get_plan(rom_s* h, int prec, int M, bool rank1, Rank2Plan* plan) {
    std::lock_guard<std::mutex> lk(h->mu);
    if (!rank1 && h->kernel_choice == ROM_KERNEL_AUTO) {
        auto tt = h->tuned.find(std::make_pair(prec == ROM_FP64 ? 0 : 1, M));
        if (tt != h->tuned.end()) {
            *plan = tt->second;
            return ROM_OK;
        }
    }
    const auto key = std::make_tuple(prec == ROM_FP64 ? 0 : 1, M, rank1 ? 1 : 0, h->R,
                                     h->kernel_choice);
    auto it = h->plans.find(key);
    if (it != h->plans.end()) {
        *plan = it->second;
        return ROM_OK;
    }
    bool ok = false;
    // FP32 with more than one realization: the two-block split-role kernel,
    // unless the caller pinned the one-block kernel.
    const bool two_block = prec != ROM_FP64 && !rank1 && h->kernel_choice != ROM_KERNEL_ONE_BLOCK;
    if (two_block && h->kernel_choice == ROM_KERNEL_DATAFLOW) {
        ok = plan_rank2_dataflow_f32(h->Kp, M, h->R, plan);
    } else if (two_block) {
        ok = plan_rank2_split_f32(h->Kp, M, h->R, plan);
        // the streaming companion on the SMs the split kernel's clusters
        // leave idle (automatic kernel choice only)
        if (ok && h->kernel_choice == ROM_KERNEL_AUTO) {
            Rank2Plan cp;
            if (h->comp_cs == 0 && plan_rank2_companion(h->Kp, M, h->R, &cp)) *plan = cp;
            else if ((h->comp_cs == 2 || h->comp_cs == 4) &&
                     plan_rank2_companion_pinned(h->Kp, M, h->R, h->comp_cs,
                                                 h->comp_cols < M ? h->comp_cols : M, &cp))
                *plan = cp;
        }
    }
    if (!ok && h->kernel_choice != ROM_KERNEL_TWO_BLOCK && h->kernel_choice != ROM_KERNEL_DATAFLOW) {
        ok = prec == ROM_FP64 ? plan_rank2_simt_f64(h->Kp, M, h->R, rank1, plan)
                              : plan_rank2_simt_f32(h->Kp, M, h->R, rank1, plan);
        if (ok) plan->variant = 1;
    }
    if (!ok) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "no SIMT rank-2 plan for Kp=%d M=%d (prec %d)", h->Kp, M, prec);
        return ROM_E_UNSUPPORTED;
    }
    h->plans[key] = *plan;
    return ROM_OK;
}

// Split operator tiles, padded g and C for the tensor-core path (once per precision).
rom_status tc_prepare(rom_s* h, int prec, cudaStream_t st) {
    if (h->tc_ops[prec][0]) return ROM_OK;
    const int Kp_tc = ((h->Kp + 127) / 128) * 128;
    if (Kp_tc > 1024) return ROM_E_UNSUPPORTED;
    if (!h->g_tc) {
        h->Kp_tc = Kp_tc;
        ROM_CUDA(cudaMalloc(&h->g_tc, sizeof(float) * Kp_tc));
        ROM_CUDA(tc_pad_rows(static_cast<const float*>(h->g_p[1]), 1, h->Kp, Kp_tc, h->g_tc, st));
        if (h->R > 0) {
            ROM_CUDA(cudaMalloc(&h->C_tc, sizeof(float) * (size_t)h->R * Kp_tc));
            ROM_CUDA(tc_pad_rows(static_cast<const float*>(h->C_rm[1]), h->R, h->Kp, Kp_tc, h->C_tc, st));
        }
    }
    const size_t bytes = tc_operator_bytes_for(prec, Kp_tc);
    void* ops[2] = {nullptr, nullptr};
    for (int o = 0; o < 2; ++o) {
        cudaError_t e = cudaMalloc(&ops[o], bytes);
        if (e == cudaSuccess)
            e = tc_prepare_operator(prec, static_cast<const float*>(o == 0 ? h->Avs_rm[1] : h->Asv_rm[1]),
                                    h->Kp, Kp_tc, ops[o], st);
        if (e != cudaSuccess) {
            cudaFree(ops[0]);
            cudaFree(ops[1]);
            return cuda_fail(e, "tensor-core operator split");
        }
    }
    h->tc_ops[prec][0] = ops[0];
    h->tc_ops[prec][1] = ops[1];
    return ROM_OK;
}

rom_status run_rank2_tc_plan(rom_s* h, const RunBufs& b, int M, int nsteps, long n0, int r, int prec,
                             const TcPlan& plan, cudaStream_t st);

rom_status run_rank2_tc(rom_s* h, const RunBufs& b, int M, int nsteps, long n0, int r, int prec,
                        cudaStream_t st) {
    rom_status s = tc_prepare(h, prec, st);
    if (s != ROM_OK) return s;
    TcPlan plan;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        const auto key = std::make_tuple(prec, M, h->tc_cols);
        auto it = h->tc_plans.find(key);
        auto tt = h->tuned_tc.find(std::make_pair(prec, M));
        if (h->tc_cols == 0 && tt != h->tuned_tc.end()) {
            plan = tt->second;
        } else if (it != h->tc_plans.end()) {
            plan = it->second;
        } else {
            if (!plan_rank2_tc(prec, h->Kp_tc, M, h->R, h->tc_cols, &plan)) {
                snprintf(g_last_error, sizeof(g_last_error),
                         "no tensor-core plan for Kp=%d M=%d prec=%d", h->Kp_tc, M, prec);
                return ROM_E_UNSUPPORTED;
            }
            h->tc_plans[key] = plan;
        }
    }
    return run_rank2_tc_plan(h, b, M, nsteps, n0, r, prec, plan, st);
}

rom_status run_rank2_tc_plan(rom_s* h, const RunBufs& b, int M, int nsteps, long n0, int r, int prec,
                             const TcPlan& plan, cudaStream_t st) {
    rom_status s = tc_prepare(h, prec, st);
    if (s != ROM_OK) return s;
    // workspace: exchange tiles of both states for every block, Kahan carries
    const size_t xterm = (size_t)h->Kp_tc * plan.W * tc_element_bytes(prec);
    const size_t xbytes = (size_t)plan.nclusters * tc_exchange_terms(prec) * xterm;
    const bool own_comp = b.compV == nullptr;
    const size_t cbytes = own_comp ? sizeof(float) * (size_t)(h->Kv + h->Ks) * M : 0;
    auto al = [](size_t x) { return (x + 1023) & ~size_t(1023); };
    ROM_CUDA(h->tc_ws.ensure(2 * al(xbytes) + al(cbytes)));
    char* ws = static_cast<char*>(h->tc_ws.p);
    TcArgs a = {};
    a.Aop[0] = h->tc_ops[prec][0];
    a.Aop[1] = h->tc_ops[prec][1];
    if (prec == ROM_BF16S) {
        const size_t so = tc_scale_offset(prec, h->Kp_tc);
        a.Ascale[0] = reinterpret_cast<const float*>(static_cast<const char*>(a.Aop[0]) + so);
        a.Ascale[1] = reinterpret_cast<const float*>(static_cast<const char*>(a.Aop[1]) + so);
    }
    a.X[0] = ws;
    a.X[1] = ws + al(xbytes);
    float* cw = reinterpret_cast<float*>(ws + 2 * al(xbytes));
    if (own_comp) ROM_CUDA(cudaMemsetAsync(cw, 0, cbytes, st));
    a.g_p = h->g_tc;
    a.C_p = h->C_tc;
    a.V = static_cast<float*>(b.V);
    a.S = static_cast<float*>(b.S);
    a.compV = own_comp ? cw : static_cast<float*>(b.compV);
    a.compS = own_comp ? cw + (size_t)h->Kv * M : static_cast<float*>(b.compS);
    a.Tper = b.ftab ? nullptr : static_cast<const float*>(b.T);
    a.ftab = static_cast<const float*>(b.ftab);
    a.traces = static_cast<float*>(b.traces);
    a.status = h->status;
    a.dt = h->dt;
    a.wavelet = h->wavelet;
    a.n0 = n0;
    a.spin_limit = h->wait_limit;
    {
        const void *xv, *xs;
        const rom_status xst = xref_for(h, 1, M, &xv, &xs);
        if (xst != ROM_OK) return xst;
        a.Xv = static_cast<const float*>(xv);
        a.Xs = static_cast<const float*>(xs);
    }
    a.Kv = h->Kv;
    a.Ks = h->Ks;
    a.Kp = h->Kp_tc;
    a.R = h->R;
    a.M = M;
    a.Mtot = M;
    a.nsteps = nsteps;
    a.r = b.traces ? r : 1;
    cudaError_t e = launch_rank2_tc(a, plan, st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core rank2 launch");
    return ROM_OK;
}

rom_status launch_simt_with_plan(rom_s* h, const RunBufs& b, int M, int nsteps, long n0, int r,
                                 int prec, const Rank2Plan& plan, cudaStream_t st);
rom_status launch_with_companion(rom_s* h, const Rank2Args& a, const Rank2Plan& plan, cudaStream_t st);

rom_status run_rank2_device(rom_s* h, const RunBufs& b, int M, int nsteps, long n0, int r,
                            int prec, bool rank1, cudaStream_t st) {
    if (tc_prec(prec)) {
        if (rank1) return ROM_E_UNSUPPORTED;
        return run_rank2_tc(h, b, M, nsteps, n0, r, prec, st);
    }
    if (prec != ROM_FP64 && prec != ROM_FP32) {
        snprintf(g_last_error, sizeof(g_last_error), "precision %d has no kernel in this build", prec);
        return ROM_E_UNSUPPORTED;
    }
    Rank2Plan plan;
    rom_status s = get_plan(h, prec, M, rank1, &plan);
    if (s != ROM_OK) return s;
    return launch_simt_with_plan(h, b, M, nsteps, n0, r, prec, plan, st);
}

rom_status launch_simt_with_plan(rom_s* h, const RunBufs& b, int M, int nsteps, long n0, int r,
                                 int prec, const Rank2Plan& plan, cudaStream_t st) {
    const int t = prec == ROM_FP64 ? 0 : 1;
    Rank2Args a = {};
    a.Avs_rm = h->Avs_rm[t];
    a.Asv_rm = h->Asv_rm[t];
    a.g_p = h->g_p[t];
    a.C_p = h->C_rm[t];
    a.V = b.V;
    a.S = b.S;
    a.compV = prec == ROM_FP64 ? nullptr : b.compV;
    a.compS = prec == ROM_FP64 ? nullptr : b.compS;
    a.Tper = b.ftab ? nullptr : b.T;
    a.ftab = b.ftab;
    a.traces = b.traces;
    a.status = h->status;
    a.dt = h->dt;
    a.wavelet = h->wavelet;
    a.n0 = n0;
    a.Kv = h->Kv;
    a.Ks = h->Ks;
    a.Kp = h->Kp;
    a.R = h->R;
    a.M = M;
    a.Mtot = M;
    a.col_base = 0;
    a.nsteps = nsteps;
    a.r = b.traces ? r : 1;
    a.spin_limit = h->wait_limit;
    a.debug_skip_push = h->inject_stall;
    {
        const rom_status xst = xref_for(h, t, M, &a.Xv, &a.Xs);
        if (xst != ROM_OK) return xst;
    }
    if (prec != ROM_FP64 && plan.variant == 2 && plan.comp_cols > 0) {
        if (a.Xv || a.Xs) {
            // the companion does not carry the reference state: split kernel alone
            Rank2Plan p2;
            if (!plan_rank2_split_f32(h->Kp, M, h->R, &p2)) return ROM_E_UNSUPPORTED;
            cudaError_t e = launch_rank2_split_f32(a, p2, st);
            return e == cudaSuccess ? ROM_OK : cuda_fail(e, "rank2 launch");
        }
        return launch_with_companion(h, a, plan, st);
    }
    cudaError_t e = prec == ROM_FP64   ? launch_rank2_simt_f64(a, plan, st)
                    : plan.variant >= 2 ? launch_rank2_split_f32(a, plan, st)
                                        : launch_rank2_simt_f32(a, plan, st);
    if (e != cudaSuccess) return cuda_fail(e, "rank2 launch");
    return ROM_OK;
}

// The split kernel on the caller's stream over columns [0, M - comp_cols) and
// the streaming companion over the rest on the handle's private stream,
// forked after the work already queued on the caller's stream and joined
// back before anything queued after this call.  The split kernel is issued
// first so that its large clusters are placed before the companion's.
rom_status launch_with_companion(rom_s* h, const Rank2Args& a, const Rank2Plan& plan, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (!h->aux) {
        e = cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "companion stream");
    }
    const int mc = plan.comp_cols;
    Rank2Args am = a;
    am.M = a.M - mc;
    Rank2Args ac = a;
    ac.col_base = a.col_base + (a.M - mc);
    ac.M = mc;
    e = cudaEventRecord(h->ev_fork, st);
    if (e == cudaSuccess && am.M > 0) e = launch_rank2_split_f32(am, plan, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->aux, h->ev_fork, 0);
    if (e == cudaSuccess) e = launch_rank2_stream_f32(ac, plan.comp_cs, plan.comp_W, plan.comp_n, h->aux);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->aux);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_join, 0);
    return e == cudaSuccess ? ROM_OK : cuda_fail(e, "rank2 launch with companion");
}

// Validates and runs a rank-2 style call; stages host buffers when V is host memory.
rom_status run_common(rom_s* h, void* V, void* S, const void* T, const void* ftab, void* compV,
                      void* compS, int M, int nsteps, long n0, int r, void* traces, int prec,
                      void* stream, bool ensemble) {
    if (!h || !V || !S || M < 1 || nsteps < 0 || r < 0 || !valid_prec(prec)) return ROM_E_INVAL;
    if (traces && (r < 1 || h->R < 1)) return ROM_E_INVAL;
    if (nsteps == 0) return ROM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t es = prec == ROM_FP64 ? 8 : 4;
    const int nrec = traces ? nsteps / r : 0;
    const bool host = !is_device_ptr(V);
    if (!host) {
        RunBufs b = {V, S, const_cast<void*>(T), const_cast<void*>(ftab), compV, compS,
                     nrec > 0 ? traces : nullptr};
        if (ensemble) {
            if (ftab || compV || compS) return ROM_E_UNSUPPORTED;
            const int t = prec == ROM_FP64 ? 0 : 1;
            Rank1EnsArgs a = {};
            a.Avs_cm = h->Avs_cm[t];
            a.Asv_cm = h->Asv_cm[t];
            a.g_p = h->g_p[t];
            a.C_cm = h->C_cm[t];
            a.V = V;
            a.S = S;
            a.Tper = T;
            a.traces = b.traces;
            a.status = h->status;
            a.dt = h->dt;
            a.wavelet = h->wavelet;
            {
                const rom_status xst = xref_for(h, t, M, &a.Xv, &a.Xs);
                if (xst != ROM_OK) return xst;
            }
            a.n0 = n0;
            a.Kv = h->Kv;
            a.Ks = h->Ks;
            a.Kp = h->Kp;
            a.R = h->R;
            a.M = M;
            a.nsteps = nsteps;
            a.r = b.traces ? r : 1;
            if (prec != ROM_FP64 && prec != ROM_FP32) return ROM_E_UNSUPPORTED;
            cudaError_t e = prec == ROM_FP64 ? launch_rank1_ensemble_f64(a, st)
                                             : launch_rank1_ensemble_f32(a, st);
            if (e != cudaSuccess) return cuda_fail(e, "rank1 ensemble launch");
            return ROM_OK;
        }
        return run_rank2_device(h, b, M, nsteps, n0, r, prec, false, st);
    }
    // host buffers: stage through library-owned device memory, synchronous
    const size_t nV = (size_t)h->Kv * M, nS = (size_t)h->Ks * M;
    const size_t nT = T ? (size_t)M : 0, nF = ftab ? (size_t)nsteps * M : 0;
    const size_t nC = compV ? nV + nS : 0;
    const size_t nTr = (size_t)nrec * h->R * M;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t bytes = al(nV * es) + al(nS * es) + al(nT * es) + al(nF * es) + al(nC * 4) +
                         al(nTr * es);
    ROM_CUDA(h->stage.ensure(bytes));
    char* base = static_cast<char*>(h->stage.p);
    size_t o = 0;
    RunBufs b = {};
    b.V = base + o; o += al(nV * es);
    b.S = base + o; o += al(nS * es);
    b.T = nT ? base + o : nullptr; o += al(nT * es);
    b.ftab = nF ? base + o : nullptr; o += al(nF * es);
    b.compV = nC ? base + o : nullptr;
    b.compS = nC ? base + o + nV * 4 : nullptr; o += al(nC * 4);
    b.traces = nTr ? base + o : nullptr;
    ROM_CUDA(cudaMemcpyAsync(b.V, V, nV * es, cudaMemcpyHostToDevice, st));
    ROM_CUDA(cudaMemcpyAsync(b.S, S, nS * es, cudaMemcpyHostToDevice, st));
    if (nT) ROM_CUDA(cudaMemcpyAsync(b.T, T, nT * es, cudaMemcpyHostToDevice, st));
    if (nF) ROM_CUDA(cudaMemcpyAsync(b.ftab, ftab, nF * es, cudaMemcpyHostToDevice, st));
    if (nC) {
        ROM_CUDA(cudaMemcpyAsync(b.compV, compV, nV * 4, cudaMemcpyHostToDevice, st));
        ROM_CUDA(cudaMemcpyAsync(b.compS, compS, nS * 4, cudaMemcpyHostToDevice, st));
    }
    rom_status s = run_common(h, b.V, b.S, b.T, b.ftab, b.compV, b.compS, M, nsteps, n0, r,
                              b.traces, prec, stream, ensemble);
    if (s != ROM_OK) return s;
    ROM_CUDA(cudaMemcpyAsync(V, b.V, nV * es, cudaMemcpyDeviceToHost, st));
    ROM_CUDA(cudaMemcpyAsync(S, b.S, nS * es, cudaMemcpyDeviceToHost, st));
    if (nC) {
        ROM_CUDA(cudaMemcpyAsync(compV, b.compV, nV * 4, cudaMemcpyDeviceToHost, st));
        ROM_CUDA(cudaMemcpyAsync(compS, b.compS, nS * 4, cudaMemcpyDeviceToHost, st));
    }
    if (nTr) ROM_CUDA(cudaMemcpyAsync(traces, b.traces, nTr * es, cudaMemcpyDeviceToHost, st));
    ROM_CUDA(cudaStreamSynchronize(st));
    return ROM_OK;
}

}  // namespace

extern "C" {

rom_status rom_set_wait_limit(rom_t h, long long cycles) {
    if (!h || cycles < 1) return ROM_E_INVAL;
    h->wait_limit = cycles;
    return ROM_OK;
}

rom_status rom_debug_inject_stall(rom_t h, int on) {
    if (!h) return ROM_E_INVAL;
    h->inject_stall = on ? 1 : 0;
    return ROM_OK;
}

rom_status rom_set_reference(rom_t h, const void* Xv, const void* Xs, int M, int in_dtype) {
    if (!h) return ROM_E_INVAL;
    std::lock_guard<std::mutex> lk(h->mu);
    if (!Xv && !Xs) {
        cudaDeviceSynchronize();  // earlier launches may still read the old copies
        for (int t = 0; t < 2; ++t)
            for (int part = 0; part < 2; ++part) {
                cudaFree(h->xref[t][part]);
                h->xref[t][part] = nullptr;
            }
        h->xref_M = 0;
        return ROM_OK;
    }
    if (M < 1 || (in_dtype != ROM_IN_F64 && in_dtype != ROM_IN_F32)) return ROM_E_INVAL;
    const size_t es = in_dtype == ROM_IN_F64 ? 8 : 4;
    const void* src[2] = {Xv, Xs};
    const int rows[2] = {h->Kv, h->Ks};
    void* tmp[2] = {nullptr, nullptr};
    const void* dsrc[2] = {nullptr, nullptr};
    void* fresh[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaError_t e = cudaSuccess;
    for (int part = 0; part < 2 && e == cudaSuccess; ++part) {
        if (!src[part]) continue;
        const size_t n = (size_t)rows[part] * M;
        if (is_device_ptr(src[part])) {
            dsrc[part] = src[part];
        } else {
            e = cudaMalloc(&tmp[part], n * es);
            if (e == cudaSuccess) e = cudaMemcpy(tmp[part], src[part], n * es, cudaMemcpyHostToDevice);
            dsrc[part] = tmp[part];
        }
        for (int t = 0; t < 2 && e == cudaSuccess; ++t) {
            e = cudaMalloc(&fresh[t][part], n * (t == 0 ? 8 : 4));
            if (e == cudaSuccess)
                e = launch_pad_copy(dsrc[part], in_dtype == ROM_IN_F64 ? 0 : 1, rows[part], M, rows[part], M,
                                    false, fresh[t][part], t, 0);
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    for (int part = 0; part < 2; ++part) cudaFree(tmp[part]);
    if (e != cudaSuccess) {
        for (int t = 0; t < 2; ++t)
            for (int part = 0; part < 2; ++part) cudaFree(fresh[t][part]);
        return e == cudaErrorMemoryAllocation ? ROM_E_NOMEM : cuda_fail(e, "rom_set_reference");
    }
    for (int t = 0; t < 2; ++t)
        for (int part = 0; part < 2; ++part) {
            cudaFree(h->xref[t][part]);
            h->xref[t][part] = fresh[t][part];
        }
    h->xref_M = M;
    return ROM_OK;
}

rom_status rom_set_wavelet(rom_t h, int wavelet) {
    if (!h || (wavelet != ROM_WAVELET_RICKER && wavelet != ROM_WAVELET_GAUSS1)) return ROM_E_INVAL;
    std::lock_guard<std::mutex> lk(h->mu);
    h->wavelet = wavelet;
    return ROM_OK;
}

rom_status rom_autotune(rom_t h, int prec, int M, int probe_steps, double* best_us, void* stream) {
    if (!h || M < 1 || probe_steps < 1 || !valid_prec(prec)) return ROM_E_INVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool f64 = prec == ROM_FP64;
    const bool tc = tc_prec(prec);
    // candidates
    std::vector<Rank2Plan> simt;
    std::vector<TcPlan> tcp;
    if (tc) {
        rom_status s = tc_prepare(h, prec, st);
        if (s != ROM_OK) return s;
        const int w_s[4] = {32, 48, 64, 80};
        const int w_o[2] = {64, 128};
        const int* ws = prec == ROM_BF16S ? w_s : w_o;
        const int nw = prec == ROM_BF16S ? 4 : 2;
        for (int i = 0; i < nw; ++i) {
            TcPlan p;
            if (plan_rank2_tc(prec, h->Kp_tc, M, h->R, ws[i], &p)) tcp.push_back(p);
        }
    } else if (f64) {
        Rank2Plan p;
        if (plan_rank2_simt_f64(h->Kp, M, h->R, false, &p)) { p.variant = 1; simt.push_back(p); }
    } else {
        Rank2Plan p0;
        int nact = 0;
        if (plan_rank2_split_f32(h->Kp, M, h->R, &p0)) nact = p0.max_active_clusters;
        else if (plan_rank2_simt_f32(h->Kp, M, h->R, false, &p0)) nact = p0.max_active_clusters;
        const int budgets[3] = {nact, nact / 2, nact / 4};
        for (int b : budgets) {
            if (b < 1) continue;
            Rank2Plan p;
            if (plan_rank2_split_f32(h->Kp, M, h->R, &p, b)) { p.variant = 2; simt.push_back(p); }
            if (plan_rank2_simt_f32(h->Kp, M, h->R, false, &p, b)) { p.variant = 1; simt.push_back(p); }
        }
        // above Kp = 512 the planner's own choice (clusters of Kp/64, 4 or 2
        // CTAs; the budgeted plans above keep Kp/64)
        if (h->Kp > 512 && nact > 0 && p0.variant == 1) simt.push_back(p0);
        // the saturated split kernel with 4, 8 or 12 fewer columns per block,
        // the freed columns on the streaming companion (clusters of 2 or 4)
        Rank2Plan ps;
        if (h->comp_cs >= 0 && plan_rank2_split_f32(h->Kp, M, h->R, &ps) &&
            ps.nclusters >= ps.max_active_clusters) {
            for (int csz : {2, 4}) {
                for (int d = 1; d <= 3; ++d) {
                    const int w = ps.Wa - 4 * d;
                    const int cols = M - 2 * ps.nclusters * w;
                    if (w < 4 || cols < 1) continue;
                    Rank2Plan p = ps;
                    Rank2Plan pc;
                    if (!plan_rank2_companion_pinned(h->Kp, M, h->R, csz, cols, &pc)) continue;
                    p.Wv = p.Wa = w;
                    p.comp_cs = pc.comp_cs;
                    p.comp_n = pc.comp_n;
                    p.comp_W = pc.comp_W;
                    p.comp_cols = pc.comp_cols;
                    simt.push_back(p);
                }
            }
        }
    }
    const size_t ncand = tc ? tcp.size() : simt.size();
    if (ncand == 0) {
        snprintf(g_last_error, sizeof(g_last_error), "rom_autotune: no plan fits Kp=%d M=%d", h->Kp, M);
        return ROM_E_UNSUPPORTED;
    }
    // probe buffers: zero state, every column with the period 45 dt
    const size_t es = f64 ? 8 : 4;
    void *V = nullptr, *S = nullptr, *T = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&V, es * (size_t)h->Kv * M);
    if (e == cudaSuccess) e = cudaMalloc(&S, es * (size_t)h->Ks * M);
    if (e == cudaSuccess) e = cudaMalloc(&T, es * (size_t)M);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    rom_status rs = ROM_OK;
    double best = -1.0;
    size_t bi = 0;
    if (e == cudaSuccess) {
        std::vector<char> hT(es * (size_t)M);
        for (int m = 0; m < M; ++m) {
            if (f64) reinterpret_cast<double*>(hT.data())[m] = 45.0 * h->dt;
            else reinterpret_cast<float*>(hT.data())[m] = (float)(45.0 * h->dt);
        }
        e = cudaMemcpyAsync(T, hT.data(), hT.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    for (size_t c = 0; c < ncand && e == cudaSuccess && rs == ROM_OK; ++c) {
        RunBufs b = {V, S, T, nullptr, nullptr, nullptr, nullptr};
        float ms = 0.f;
        for (int pass = 0; pass < 2 && rs == ROM_OK && e == cudaSuccess; ++pass) {  // warm-up, timed
            e = cudaMemsetAsync(V, 0, es * (size_t)h->Kv * M, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(S, 0, es * (size_t)h->Ks * M, st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e != cudaSuccess) break;
            const int n = pass == 0 ? (probe_steps < 20 ? probe_steps : 20) : probe_steps;
            rs = tc ? run_rank2_tc_plan(h, b, M, n, 0, 0, prec, tcp[c], st)
                    : launch_simt_with_plan(h, b, M, n, 0, 0, prec, simt[c], st);
            if (rs == ROM_OK) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess && rs == ROM_OK) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess && rs == ROM_OK) e = cudaEventElapsedTime(&ms, e0, e1);
        }
        if (e == cudaSuccess && rs == ROM_OK) {
            const double us = 1e3 * ms / probe_steps;
            if (best < 0.0 || us < best) { best = us; bi = c; }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(V);
    cudaFree(S);
    cudaFree(T);
    if (e != cudaSuccess) return cuda_fail(e, "rom_autotune");
    if (rs != ROM_OK) return rs;
    int st_word = 0;
    if (cudaMemcpy(&st_word, h->status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && st_word != 0)
        return (rom_status)st_word;
    {
        std::lock_guard<std::mutex> lk(h->mu);
        if (tc) h->tuned_tc[std::make_pair(prec, M)] = tcp[bi];
        else h->tuned[std::make_pair(f64 ? 0 : 1, M)] = simt[bi];
    }
    if (best_us) *best_us = best;
    return ROM_OK;
}

rom_status rom_set_tc_columns(rom_t h, int cols) {
    if (!h || cols < 0 || cols > 256 || cols % 16 != 0) return ROM_E_INVAL;
    std::lock_guard<std::mutex> lk(h->mu);
    h->tc_cols = cols;
    return ROM_OK;
}

rom_status rom_set_companion(rom_t h, int cluster_size, int columns) {
    if (!h || !(cluster_size == -1 || cluster_size == 0 || cluster_size == 2 || cluster_size == 4))
        return ROM_E_INVAL;
    if ((cluster_size == 2 || cluster_size == 4) && columns < 1) return ROM_E_INVAL;
    std::lock_guard<std::mutex> lk(h->mu);
    h->comp_cs = cluster_size;
    h->comp_cols = cluster_size > 0 ? columns : 0;
    h->plans.clear();
    h->tuned.clear();
    return ROM_OK;
}

rom_status rom_set_kernel(rom_t h, int kernel) {
    if (!h || kernel < ROM_KERNEL_AUTO || kernel > ROM_KERNEL_DATAFLOW) return ROM_E_INVAL;
    std::lock_guard<std::mutex> lk(h->mu);
    h->kernel_choice = kernel;
    return ROM_OK;
}

rom_status rom_get_plan(rom_t h, int prec, int M, int* variant, int* cluster_size,
                        int* cols_per_block, int* nclusters) {
    if (!h || M < 1 || !valid_prec(prec)) return ROM_E_INVAL;
    if (prec != ROM_FP64 && prec != ROM_FP32) return ROM_E_UNSUPPORTED;
    Rank2Plan p;
    rom_status s = get_plan(h, prec, M, false, &p);
    if (s != ROM_OK) return s;
    if (variant) *variant = p.comp_cols > 0 ? 4 : p.variant;
    if (cluster_size) *cluster_size = p.cs;
    if (cols_per_block) *cols_per_block = p.Wv;
    if (nclusters) *nclusters = p.nclusters;
    return ROM_OK;
}

rom_status rom_get_companion(rom_t h, int M, int* cluster_size, int* nclusters, int* columns) {
    if (!h || M < 1) return ROM_E_INVAL;
    Rank2Plan p;
    rom_status s = get_plan(h, ROM_FP32, M, false, &p);
    if (s != ROM_OK) return s;
    const bool on = p.variant == 2 && p.comp_cols > 0;
    if (cluster_size) *cluster_size = on ? p.comp_cs : 0;
    if (nclusters) *nclusters = on ? p.comp_n : 0;
    if (columns) *columns = on ? p.comp_cols : 0;
    return ROM_OK;
}

rom_status rom_run_rank2(rom_t h, void* V, void* S, const void* T, int M, int nsteps, long n0,
                         int r, void* traces, int prec, void* stream) {
    return run_common(h, V, S, T, nullptr, nullptr, nullptr, M, nsteps, n0, r, traces, prec,
                      stream, false);
}

rom_status rom_run_rank2_ex(rom_t h, void* V, void* S, const void* T, const void* ftab,
                            void* compV, void* compS, int M, int nsteps, long n0, int r,
                            void* traces, int prec, void* stream) {
    if ((compV == nullptr) != (compS == nullptr)) return ROM_E_INVAL;
    return run_common(h, V, S, T, ftab, compV, compS, M, nsteps, n0, r, traces, prec, stream,
                      false);
}

rom_status rom_run_rank1_ensemble(rom_t h, void* V, void* S, const void* T, int M, int nsteps,
                                  long n0, int r, void* traces, int prec, void* stream) {
    return run_common(h, V, S, T, nullptr, nullptr, nullptr, M, nsteps, n0, r, traces, prec,
                      stream, true);
}

rom_status rom_run_rank1(rom_t h, void* v, void* s, double T, int nsteps, long n0, int r,
                         void* trace, int prec, void* stream) {
    if (!h || !v || !s || nsteps < 0 || r < 0 || !valid_prec(prec) || !(T > 0.0)) return ROM_E_INVAL;
    if (trace && (r < 1 || h->R < 1)) return ROM_E_INVAL;
    if (nsteps == 0) return ROM_OK;
    if (prec != ROM_FP64 && prec != ROM_FP32) return ROM_E_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t es = prec == ROM_FP64 ? 8 : 4;
    // the period goes to a small device scratch in the state's element type
    if (prec == ROM_FP64) {
        ROM_CUDA(cudaMemcpyAsync(h->scalar, &T, 8, cudaMemcpyHostToDevice, st));
    } else {
        const float Tf = (float)T;
        ROM_CUDA(cudaMemcpyAsync(h->scalar, &Tf, 4, cudaMemcpyHostToDevice, st));
    }
    const bool host = !is_device_ptr(v);
    const int nrec = trace ? nsteps / r : 0;
    if (!host) {
        RunBufs b = {v, s, h->scalar, nullptr, nullptr, nullptr, nrec > 0 ? trace : nullptr};
        return run_rank2_device(h, b, 1, nsteps, n0, r, prec, true, st);
    }
    const size_t nV = h->Kv, nS = h->Ks, nTr = (size_t)nrec * h->R;
    ROM_CUDA(h->stage.ensure((nV + nS + nTr) * es + 512));
    char* base = static_cast<char*>(h->stage.p);
    RunBufs b = {base, base + ((nV * es + 255) & ~size_t(255)), h->scalar, nullptr, nullptr,
                 nullptr, nullptr};
    b.traces = nTr ? static_cast<char*>(b.S) + ((nS * es + 255) & ~size_t(255)) : nullptr;
    ROM_CUDA(cudaMemcpyAsync(b.V, v, nV * es, cudaMemcpyHostToDevice, st));
    ROM_CUDA(cudaMemcpyAsync(b.S, s, nS * es, cudaMemcpyHostToDevice, st));
    rom_status rs = run_rank2_device(h, b, 1, nsteps, n0, r, prec, true, st);
    if (rs != ROM_OK) return rs;
    ROM_CUDA(cudaMemcpyAsync(v, b.V, nV * es, cudaMemcpyDeviceToHost, st));
    ROM_CUDA(cudaMemcpyAsync(s, b.S, nS * es, cudaMemcpyDeviceToHost, st));
    if (nTr) ROM_CUDA(cudaMemcpyAsync(trace, b.traces, nTr * es, cudaMemcpyDeviceToHost, st));
    ROM_CUDA(cudaStreamSynchronize(st));
    return ROM_OK;
}

// ---------------------------------------------------------------- batched
//
// Many ROMs with uneven K and M in one CUDA-graph launch.  Each job keeps its
// own persistent cluster kernel; the scheduler gives job i a share of the
// GPU's SMs proportional to its work 4 K_i^2 M_i (its cluster budget, which
// fixes the columns per cluster block), orders the launches longest-first and
// captures them, forked over a pool of streams, into one graph that is
// instantiated once per job list and replayed.
}  // extern "C"

namespace {

struct BatchKey {
    std::vector<uintptr_t> words;
    bool operator<(const BatchKey& o) const { return words < o.words; }
};
std::mutex g_batch_mu;
// A captured batch: the graph, and the device tables of its work-list
// launches (operator/job tables, items, counters), freed with it.
struct BatchGraph {
    cudaGraphExec_t exec = nullptr;
    void* tables = nullptr;
};
void free_batch_graph(BatchGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.tables) cudaFree(g.tables);
    g = BatchGraph{};
}
std::map<BatchKey, BatchGraph> g_batch_graphs;
std::vector<cudaStream_t> g_batch_streams;
std::vector<cudaEvent_t> g_batch_events;
cudaStream_t g_capture_stream = nullptr;  // private: the caller's stream may be the legacy one

// Cluster-budget scale (and, for ROM_AUTO, the size threshold; for
// ROM_FP32 the choice between the work-list form, 1, and one launch per job,
// 0) chosen by rom_autotune_batched, per job list (handles and widths;
// buffers and step counts do not change the choice).  Keys: (njobs, prec,
// device), then (handle, M) per job.
std::map<std::vector<uintptr_t>, double> g_batch_scale;
std::map<std::vector<uintptr_t>, int> g_batch_kthr;
std::map<std::vector<uintptr_t>, int> g_batch_tcw;
std::map<std::vector<uintptr_t>, int> g_batch_wl;

void drop_batch_graphs(rom_s* h) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto tuned_for_h = [h](const std::vector<uintptr_t>& k) {
        for (size_t i = 3; i < k.size(); i += 2)
            if (k[i] == (uintptr_t)h) return true;
        return false;
    };
    for (auto it = g_batch_scale.begin(); it != g_batch_scale.end();)
        it = tuned_for_h(it->first) ? g_batch_scale.erase(it) : std::next(it);
    for (auto it = g_batch_kthr.begin(); it != g_batch_kthr.end();)
        it = tuned_for_h(it->first) ? g_batch_kthr.erase(it) : std::next(it);
    for (auto it = g_batch_tcw.begin(); it != g_batch_tcw.end();)
        it = tuned_for_h(it->first) ? g_batch_tcw.erase(it) : std::next(it);
    for (auto it = g_batch_wl.begin(); it != g_batch_wl.end();)
        it = tuned_for_h(it->first) ? g_batch_wl.erase(it) : std::next(it);
    for (auto it = g_batch_graphs.begin(); it != g_batch_graphs.end();) {
        bool uses = false;
        const auto& w = it->first.words;
        for (size_t k = 6; k < w.size(); k += 6) uses |= (w[k] == (uintptr_t)h);
        if (uses) {
            free_batch_graph(it->second);
            it = g_batch_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

rom_status batch_streams(size_t n) {
    if (!g_capture_stream) ROM_CUDA(cudaStreamCreateWithFlags(&g_capture_stream, cudaStreamNonBlocking));
    while (g_batch_streams.size() < n) {
        cudaStream_t s;
        ROM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        g_batch_streams.push_back(s);
    }
    while (g_batch_events.size() < n + 1) {
        cudaEvent_t e;
        ROM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        g_batch_events.push_back(e);
    }
    return ROM_OK;
}

}  // namespace

extern "C" {

// Default size threshold of ROM_AUTO: jobs with max(Kv, Ks) at or above it
// run the exact-slice BF16 tensor-core path, the others FP32 SIMT.
constexpr int kAutoKthr = 256;

static bool batch_prec(int prec) { return valid_prec(prec) || prec == ROM_AUTO; }

// Block width of a tensor-core job in a batch: the narrowest width that
// holds all M columns in one block, else the widest.  A tcgen05 MMA costs the
// same for every block width up to 128 columns, so when jobs share the SMs
// the widest block yields the most columns per SM and step (the planner's
// own choice, tuned for one job alone, spreads it over more SMs instead).
static int batch_tc_width(int prec, int M) {
    if (prec == ROM_BF16S) {
        const int w[4] = {32, 48, 64, 80};
        for (int c : w)
            if (M <= c) return c;
        return 80;
    }
    return M <= 64 ? 64 : 128;
}

// ---- work-list batched launch (FP32): ONE persistent launch of the
// work-list kernel for every job of the batch.  All clusters have the same
// size cs (2: 76 co-resident clusters cover all 152 SMs of a GB300; 4: 36
// clusters, 144 SMs); a job's Kp / 32 row tiles are dealt out to the CTAs of
// whichever cluster takes one of its items, so jobs of every size share one
// kernel and one device work list.  Job j is cut into column blocks of width
// W_j: the widest that fits the shared memory (and the cap `wcap`), then
// narrowed to spread M_j evenly over that many blocks.  The items are
// ordered longest first (a step of an item costs about its busiest CTA's
// rows x Kp x W_j multiply-adds plus a fixed part), so the clusters, which
// take the next item whenever they finish one, end within about one short
// item of each other (list scheduling, longest processing time first).
// Receiver rows are staged in shared memory when a CTA's share is at most
// 16 KB, else read from global memory.
//
// `wl` encodes the form: cs * 1000 + wcap.
constexpr int kWlDefault = 2 * 1000 + 32;

static bool wl_decode(int wl, int* cs, int* wcap) {
    *cs = wl / 1000;
    *wcap = wl % 1000;
    return (*cs == 2 || *cs == 4 || *cs == 8) && *wcap >= 8 && *wcap % 8 == 0 && *wcap <= 256;
}

// A job's layout in the work-list form with clusters of cs CTAs: tiles per
// CTA, whether its receiver rows are read from global memory, the widest
// multiple of 8 (<= wcap) that fits `budget` bytes of shared memory narrowed
// to spread M evenly over that many blocks, and that width's shared memory.
struct WlJob {
    int nrt = 0, cglob = 0, W = 0, nblocks = 0;
    size_t smem = 0;
};
static bool wl_job_layout(const rom_s* h, int M, int cs, int wcap, size_t budget, WlJob* L) {
    const int Kp = h->Kp;
    L->nrt = (Kp / 32 + cs - 1) / cs;
    const int rpc = (h->R + cs - 1) / cs;
    L->cglob = (size_t)rpc * Kp * sizeof(float) > 16384 ? 1 : 0;
    const int rst = L->cglob ? 0 : rpc;
    int wmax = 0;
    for (int w = 8; w <= wcap; w += 8) {
        if (worklist_smem(w, Kp, rst, L->nrt) > budget) break;
        wmax = w;
    }
    if (wmax == 0) return false;
    L->nblocks = (M + wmax - 1) / wmax;
    L->W = (((M + L->nblocks - 1) / L->nblocks) + 7) / 8 * 8;
    L->smem = worklist_smem(L->W, Kp, rst, L->nrt);
    return true;
}

// The form an FP32 job list runs in when nothing pinned or tuned one: the
// work-list launch (kWlDefault) or one launch per job (0), whichever the
// step-time models predict faster.  Work list: its items run longest first
// on the co-resident clusters, so a step lasts about max(longest item,
// sum of item times / clusters).  Per job: each job on its own plan, the
// jobs side by side, so about max(slowest job, sum of job time x SMs / SMs
// of the GPU).  Few items (small M, say 16 operators of 16 columns) leave
// the work list's clusters idle while the split kernel keeps its operators
// in registers; many uneven jobs favour the list.
static int batched_default_form(const rom_job* jobs, int njobs, int dev, int nsm) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return kWlDefault;
    }
    const size_t budget = (size_t)optin - 1024;
    int cs = 0, wcap = 0;
    wl_decode(kWlDefault, &cs, &wcap);
    double sum = 0.0, cmax = 0.0;
    long nitems = 0;
    size_t smem = 0;
    for (int i = 0; i < njobs; ++i) {
        WlJob L;
        if (!wl_job_layout(jobs[i].h, jobs[i].M, cs, wcap, budget, &L)) return 0;
        const double c = model_streamed_us(jobs[i].h->Kp, L.nrt, L.W);
        sum += c * L.nblocks;
        cmax = c > cmax ? c : cmax;
        nitems += L.nblocks;
        smem = L.smem > smem ? L.smem : smem;
    }
    int P = worklist_max_clusters(cs, smem);
    if (P <= 0) return 0;
    if (P > nitems) P = (int)nitems;
    const double t_wl = fmax(cmax, sum / P);
    double tmax = 0.0, sm_us = 0.0;
    for (int i = 0; i < njobs; ++i) {
        const rom_s* h = jobs[i].h;
        Rank2Plan p;
        double t = 0.0;
        if (plan_rank2_split_f32(h->Kp, jobs[i].M, h->R, &p)) {
            t = model_split_us(h->Kp, p.Wa);
        } else if (plan_rank2_simt_f32(h->Kp, jobs[i].M, h->R, false, &p)) {
            const int act = p.max_active_clusters > 0 ? p.max_active_clusters : 1;
            t = ((p.nclusters + act - 1) / act) * model_streamed_us(h->Kp, p.nrt, p.Wa);
        } else {
            return kWlDefault;
        }
        const int busy = p.nclusters < p.max_active_clusters ? p.nclusters : p.max_active_clusters;
        tmax = t > tmax ? t : tmax;
        sm_us += t * busy * p.cs;
    }
    const double t_pj = fmax(tmax, sm_us / nsm);
    return t_pj < t_wl ? 0 : kWlDefault;
}

static rom_status run_batched_worklist(const rom_job* jobs, int njobs, int nsteps, int r,
                                       cudaStream_t st, int dev, int wl) {
    int cs = 0, wcap = 0;
    if (!wl_decode(wl, &cs, &wcap)) return ROM_E_INVAL;
    BatchKey key;
    key.words = {(uintptr_t)njobs, (uintptr_t)nsteps, (uintptr_t)r, (uintptr_t)ROM_FP32, (uintptr_t)st,
                 (uintptr_t)dev};
    for (int i = 0; i < njobs; ++i) {
        const rom_job& j = jobs[i];
        key.words.insert(key.words.end(), {(uintptr_t)j.h, (uintptr_t)j.V, (uintptr_t)j.S,
                                           (uintptr_t)j.T, (uintptr_t)j.M, (uintptr_t)j.traces});
    }
    key.words.push_back((uintptr_t)0x574c0000 + (uintptr_t)wl);  // work-list form
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto it = g_batch_graphs.find(key);
    if (it == g_batch_graphs.end()) {
        int optin = 0;
        ROM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        const size_t budget = (size_t)optin - 1024;
        // ---- per job: tiles per CTA, receiver rows, width
        std::vector<GroupOp> ops(njobs);
        std::vector<double> cost(njobs);
        size_t smem = 0;
        int nitems = 0;
        for (int i = 0; i < njobs; ++i) {
            const rom_s* h = jobs[i].h;
            const int Kp = h->Kp, M = jobs[i].M;
            WlJob L;
            if (!wl_job_layout(h, M, cs, wcap, budget, &L)) {
                snprintf(g_last_error, sizeof(g_last_error), "no work-list width for Kp=%d", Kp);
                return ROM_E_UNSUPPORTED;
            }
            const int nrt = L.nrt, cglob = L.cglob, W = L.W, nb = L.nblocks;
            smem = L.smem > smem ? L.smem : smem;
            GroupOp& g = ops[i];
            g.Avs_rm = h->Avs_rm[1];
            g.Asv_rm = h->Asv_rm[1];
            g.g_p = h->g_p[1];
            g.C_p = h->C_rm[1];
            g.V = jobs[i].V;
            g.S = jobs[i].S;
            g.Tper = jobs[i].T;
            g.traces = jobs[i].traces;
            g.status = h->status;
            g.dt = h->dt;
            g.Kv = h->Kv;
            g.Ks = h->Ks;
            g.R = h->R;
            g.M = M;
            g.wavelet = h->wavelet;
            g.Kp = Kp;
            g.Wa = W;
            g.c_global = cglob;
            cost[i] = model_streamed_us(Kp, nrt, W);
            nitems += nb;
        }
        // ---- the item list, longest first (ties: job order, then columns)
        std::vector<WorkItem> items;
        items.reserve(nitems);
        for (int i = 0; i < njobs; ++i)
            for (int col = 0; col < jobs[i].M; col += ops[i].Wa)
                items.push_back({i, col, jobs[i].M - col < ops[i].Wa ? jobs[i].M - col : ops[i].Wa, 0});
        std::stable_sort(items.begin(), items.end(),
                         [&](const WorkItem& x, const WorkItem& y) { return cost[x.job] > cost[y.job]; });
        nitems = (int)items.size();  // the list as built (equal to the blocks counted above)
        int ncl = worklist_max_clusters(cs, smem);
        if (ncl <= 0) {
            snprintf(g_last_error, sizeof(g_last_error), "work-list kernel does not fit (cs=%d, %zu B)", cs, smem);
            return ROM_E_UNSUPPORTED;
        }
        if (ncl > nitems) ncl = nitems;
        // ---- device tables: counter, job table, items
        const size_t off_ops = 256;
        const size_t off_items = off_ops + ((sizeof(GroupOp) * njobs + 255) / 256) * 256;
        const size_t bytes = off_items + sizeof(WorkItem) * items.size();
        std::vector<unsigned char> host(bytes, 0);
        memcpy(host.data() + off_ops, ops.data(), sizeof(GroupOp) * njobs);
        memcpy(host.data() + off_items, items.data(), sizeof(WorkItem) * items.size());
        void* tables = nullptr;
        ROM_CUDA(cudaMalloc(&tables, bytes));
        cudaError_t e = cudaMemcpy(tables, host.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(tables);
            return cuda_fail(e, "rom_run_batched work list");
        }
        const rom_s* h0 = jobs[0].h;
        Rank2Args a = {};
        a.nsteps = nsteps;
        a.r = r > 0 ? r : 1;
        a.spin_limit = h0->wait_limit;
        a.group = reinterpret_cast<const GroupOp*>(static_cast<unsigned char*>(tables) + off_ops);
        a.items = reinterpret_cast<const WorkItem*>(static_cast<unsigned char*>(tables) + off_items);
        a.nitems = nitems;
        a.item_counter = static_cast<int*>(tables);
        // ---- capture: reset the counter, then the one launch
        rom_status s = batch_streams(1);
        if (s != ROM_OK) {
            cudaFree(tables);
            return s;
        }
        cudaGraph_t graph = nullptr;
        cudaStream_t cap = g_capture_stream;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) e = cudaMemsetAsync(tables, 0, sizeof(int), cap);
        if (e == cudaSuccess) e = launch_rank2_worklist_f32(a, cs, ncl, smem, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaFree(tables);
            return cuda_fail(e, "rom_run_batched work-list capture");
        }
        it = g_batch_graphs.emplace(key, BatchGraph{exec, tables}).first;
    }
    ROM_CUDA(cudaGraphLaunch(it->second.exec, st));
    return ROM_OK;
}

// tcw: tensor-core block widths, 1 = batch_tc_width, 0 = the planner's.
// wl: FP32 batches run as one work-list launch of that form (cs * 1000 +
// wcap), 0 = one launch per job.
static rom_status run_batched_impl(const rom_job* jobs, int njobs, int nsteps, int r, int prec,
                                   void* stream, double scale, int kthr = kAutoKthr, int tcw = 1,
                                   int wl = kWlDefault) {
    if (!jobs || njobs < 1 || nsteps < 0 || r < 0 || !batch_prec(prec)) return ROM_E_INVAL;
    for (int i = 0; i < njobs; ++i) {
        const rom_job& j = jobs[i];
        if (!j.h || !j.V || !j.S || j.M < 1) return ROM_E_INVAL;
        if (!is_device_ptr(j.V) || !is_device_ptr(j.S)) return ROM_E_INVAL;  // device buffers only
        if (j.traces && (r < 1 || j.h->R < 1)) return ROM_E_INVAL;
        for (int k = 0; k < i; ++k)
            if (jobs[k].h == j.h) return ROM_E_INVAL;  // one job per handle (handles own workspaces)
    }
    if (nsteps == 0) return ROM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the precision of every job (ROM_AUTO: by size)
    std::vector<int> jp(njobs);
    bool any_tc = false;
    for (int i = 0; i < njobs; ++i) {
        const int K = jobs[i].h->Kv > jobs[i].h->Ks ? jobs[i].h->Kv : jobs[i].h->Ks;
        jp[i] = prec != ROM_AUTO ? prec : (K >= kthr ? ROM_BF16S : ROM_FP32);
        any_tc = any_tc || tc_prec(jp[i]);
    }
    int dev = 0, nsm = 0;
    ROM_CUDA(cudaGetDevice(&dev));
    ROM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (wl && prec == ROM_FP32) {
        bool ok = true;
        for (int i = 0; i < njobs; ++i) ok = ok && jobs[i].h->xref_M == 0 && jobs[i].h->Kp <= 1024;
        if (ok) return run_batched_worklist(jobs, njobs, nsteps, r, st, dev, wl);
    }
    // share of the SMs per job, proportional to its work per step
    std::vector<double> cost(njobs);
    double total = 0.0;
    for (int i = 0; i < njobs; ++i) {
        const double K = (double)(jobs[i].h->Kv > jobs[i].h->Ks ? jobs[i].h->Kv : jobs[i].h->Ks);
        cost[i] = 4.0 * K * K * jobs[i].M;
        total += cost[i];
    }
    std::vector<Rank2Plan> plans(njobs);
    std::vector<double> est(njobs);
    std::vector<TcPlan> tcplans(njobs);
    std::vector<char> tcwide(njobs, 0);
    for (int i = 0; i < njobs; ++i) {
        rom_s* h = jobs[i].h;
        const int pj = jp[i];
        if (tc_prec(pj)) {
            rom_status s = tc_prepare(h, pj, st);
            if (s != ROM_OK) return s;
            est[i] = cost[i];
            // a width pinned with rom_set_tc_columns wins over the batch rule
            if (tcw == 1 && h->tc_cols == 0 &&
                plan_rank2_tc(pj, h->Kp_tc, jobs[i].M, h->R, batch_tc_width(pj, jobs[i].M), &tcplans[i]))
                tcwide[i] = 1;
            continue;
        }
        const int Kp = h->Kp;
        const int cs_guess = Kp > 512 ? Kp / 64 : Kp / 32;
        const int budget = (int)(scale * (double)nsm * cost[i] / total / cs_guess);
        bool ok = false;
        if (pj == ROM_FP32) ok = plan_rank2_split_f32(Kp, jobs[i].M, h->R, &plans[i], budget > 0 ? budget : 1);
        if (ok) plans[i].variant = 2;
        if (!ok) {
            ok = pj == ROM_FP64 ? plan_rank2_simt_f64(Kp, jobs[i].M, h->R, false, &plans[i])
                                  : plan_rank2_simt_f32(Kp, jobs[i].M, h->R, false, &plans[i],
                                                        budget > 0 ? budget : 1);
            if (ok) plans[i].variant = 1;
        }
        if (!ok) return ROM_E_UNSUPPORTED;
        est[i] = cost[i] / (double)(plans[i].nclusters * plans[i].cs);
    }
    std::vector<int> order(njobs);
    for (int i = 0; i < njobs; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return est[x] > est[y]; });

    BatchKey key;
    key.words = {(uintptr_t)njobs, (uintptr_t)nsteps, (uintptr_t)r, (uintptr_t)prec, (uintptr_t)st,
                 (uintptr_t)dev};
    for (int i = 0; i < njobs; ++i) {
        const rom_job& j = jobs[i];
        key.words.insert(key.words.end(), {(uintptr_t)j.h, (uintptr_t)j.V, (uintptr_t)j.S,
                                           (uintptr_t)j.T, (uintptr_t)j.M, (uintptr_t)j.traces});
    }
    key.words.push_back((uintptr_t)(scale * 1024.0));
    key.words.push_back((uintptr_t)(prec == ROM_AUTO ? kthr : -1));
    key.words.push_back((uintptr_t)tcw);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    auto it = g_batch_graphs.find(key);
    if (it == g_batch_graphs.end()) {
        const size_t npool = (size_t)(njobs < 32 ? njobs : 32);
        rom_status s = batch_streams(npool);
        if (s != ROM_OK) return s;
        cudaGraph_t graph = nullptr;
        cudaStream_t cap = g_capture_stream;
        ROM_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
        cudaEvent_t fork = g_batch_events[npool];
        cudaError_t e = cudaEventRecord(fork, cap);
        rom_status rs = ROM_OK;
        for (size_t k = 0; k < npool && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(g_batch_streams[k], fork, 0);
        for (int oi = 0; oi < njobs && e == cudaSuccess && rs == ROM_OK; ++oi) {
            const int i = order[oi];
            const rom_job& j = jobs[i];
            cudaStream_t ss = g_batch_streams[oi % npool];
            RunBufs b = {j.V, j.S, const_cast<void*>(j.T), nullptr, nullptr, nullptr, j.traces};
            if (!tc_prec(jp[i]))
                rs = launch_simt_with_plan(j.h, b, j.M, nsteps, 0, r, jp[i], plans[i], ss);
            else if (tcwide[i])
                rs = run_rank2_tc_plan(j.h, b, j.M, nsteps, 0, r, jp[i], tcplans[i], ss);
            else
                rs = run_rank2_tc(j.h, b, j.M, nsteps, 0, r, jp[i], ss);
        }
        for (size_t k = 0; k < npool && e == cudaSuccess; ++k) {
            e = cudaEventRecord(g_batch_events[k], g_batch_streams[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, g_batch_events[k], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
        if (rs != ROM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rs;
        }
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e, "rom_run_batched capture");
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "rom_run_batched instantiate");
        it = g_batch_graphs.emplace(key, BatchGraph{exec, nullptr}).first;
    }
    ROM_CUDA(cudaGraphLaunch(it->second.exec, st));
    if (any_tc) {
        // tensor-core jobs use per-handle workspaces that a later call may
        // reallocate: their graphs are not kept
        BatchGraph g = it->second;
        g_batch_graphs.erase(it);
        ROM_CUDA(cudaStreamSynchronize(st));
        free_batch_graph(g);
    }
    return ROM_OK;
}

static std::vector<uintptr_t> batch_tune_key(const rom_job* jobs, int njobs, int prec) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<uintptr_t> k = {(uintptr_t)njobs, (uintptr_t)prec, (uintptr_t)dev};
    for (int i = 0; i < njobs; ++i) {
        k.push_back((uintptr_t)jobs[i].h);
        k.push_back((uintptr_t)jobs[i].M);
    }
    return k;
}

rom_status rom_run_batched(const rom_job* jobs, int njobs, int nsteps, int r, int prec, void* stream) {
    double scale = 1.0;
    int kthr = kAutoKthr, tcw = 1, wl = kWlDefault;
    bool model_form = false;
    if (jobs && njobs > 0) {
        bool valid = true;
        for (int i = 0; i < njobs; ++i) {
            if (!jobs[i].h) return ROM_E_INVAL;
            valid = valid && jobs[i].M >= 1;
        }
        std::lock_guard<std::mutex> lk(g_batch_mu);
        const auto key = batch_tune_key(jobs, njobs, prec);
        auto it = g_batch_scale.find(key);
        if (it != g_batch_scale.end()) scale = it->second;
        auto kt = g_batch_kthr.find(key);
        if (kt != g_batch_kthr.end()) kthr = kt->second;
        auto tw = g_batch_tcw.find(key);
        if (tw != g_batch_tcw.end()) tcw = tw->second;
        auto wt = g_batch_wl.find(key);
        if (wt != g_batch_wl.end()) wl = wt->second;
        else model_form = prec == ROM_FP32 && valid;
    }
    if (model_form) {
        // neither pinned nor tuned: the models' choice, kept for this list
        int dev = 0, nsm = 0;
        ROM_CUDA(cudaGetDevice(&dev));
        ROM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        wl = batched_default_form(jobs, njobs, dev, nsm);
        std::lock_guard<std::mutex> lk(g_batch_mu);
        g_batch_wl.emplace(batch_tune_key(jobs, njobs, prec), wl);
    }
    return run_batched_impl(jobs, njobs, nsteps, r, prec, stream, scale, kthr, tcw, wl);
}

rom_status rom_set_batched_form(const rom_job* jobs, int njobs, int prec, int cluster_size, int width_cap) {
    if (!jobs || njobs < 1 || prec != ROM_FP32) return ROM_E_INVAL;
    for (int i = 0; i < njobs; ++i)
        if (!jobs[i].h || jobs[i].M < 1) return ROM_E_INVAL;
    int wl = 0;
    if (cluster_size != 0) {
        int cs = 0, wcap = 0;
        wl = cluster_size * 1000 + width_cap;
        if (width_cap < 0 || width_cap >= 1000 || !wl_decode(wl, &cs, &wcap)) return ROM_E_INVAL;
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_batch_wl[batch_tune_key(jobs, njobs, prec)] = wl;
    return ROM_OK;
}

rom_status rom_autotune_batched(const rom_job* jobs, int njobs, int prec, int probe_steps,
                                double* best_us, void* stream) {
    if (!jobs || njobs < 1 || probe_steps < 1 || !batch_prec(prec)) return ROM_E_INVAL;
    for (int i = 0; i < njobs; ++i)
        if (!jobs[i].h || jobs[i].M < 1) return ROM_E_INVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t es = prec == ROM_FP64 ? 8 : 4;
    // scratch state of every job (zero state, every period 45 dt)
    std::vector<rom_job> sj(jobs, jobs + njobs);
    std::vector<void*> bufs;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < njobs && e == cudaSuccess; ++i) {
        void *V = nullptr, *S = nullptr, *T = nullptr;
        e = cudaMalloc(&V, es * (size_t)jobs[i].h->Kv * jobs[i].M);
        if (e == cudaSuccess) bufs.push_back(V);
        if (e == cudaSuccess) e = cudaMalloc(&S, es * (size_t)jobs[i].h->Ks * jobs[i].M);
        if (e == cudaSuccess) bufs.push_back(S);
        if (e == cudaSuccess) e = cudaMalloc(&T, es * (size_t)jobs[i].M);
        if (e == cudaSuccess) bufs.push_back(T);
        if (e == cudaSuccess) {
            std::vector<char> hT(es * (size_t)jobs[i].M);
            for (int m = 0; m < jobs[i].M; ++m) {
                if (es == 8) reinterpret_cast<double*>(hT.data())[m] = 45.0 * jobs[i].h->dt;
                else reinterpret_cast<float*>(hT.data())[m] = (float)(45.0 * jobs[i].h->dt);
            }
            e = cudaMemcpy(T, hT.data(), hT.size(), cudaMemcpyHostToDevice);
        }
        sj[i].V = V;
        sj[i].S = S;
        sj[i].T = T;
        sj[i].traces = nullptr;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const double scales[4] = {0.5, 1.0, 2.0, 4.0};
    // ROM_AUTO: size thresholds from every job on BF16S to every job on FP32
    const int kthrs[4] = {0, 256, 512, 1 << 20};
    const int nk = prec == ROM_AUTO ? 4 : 1;
    // tensor-core block widths: the batch rule (1) and the planner's (0)
    const int ntw = (prec == ROM_AUTO || tc_prec(prec)) ? 2 : 1;
    double best = -1.0, best_scale = 1.0;
    int best_kthr = kAutoKthr, best_tcw = 1, best_wl = 0;
    rom_status rs = ROM_OK;
    // FP32: work-list forms (clusters of 2 or 4 CTAs, width caps 16 / 32 /
    // 64) besides one launch per job (0)
    const int wls[7] = {kWlDefault, 2016, 2064, 4016, 4032, 4064, 0};
    const int nwl = prec == ROM_FP32 ? 7 : 1;
    for (int iw = 0; iw < nwl && e == cudaSuccess && rs == ROM_OK; ++iw)
    for (int t = 0; t < nk && e == cudaSuccess && rs == ROM_OK; ++t) {
        const int wl = prec == ROM_FP32 ? wls[iw] : 0;
        for (int tw = 0; tw < ntw && e == cudaSuccess && rs == ROM_OK; ++tw) {
            const int tcw = 1 - tw;
            for (int c = 0; c < (wl ? 1 : 4) && e == cudaSuccess && rs == ROM_OK; ++c) {
                float ms = 0.f;
                for (int pass = 0; pass < 2 && e == cudaSuccess && rs == ROM_OK; ++pass) {  // warm-up, timed
                    const int n = pass == 0 ? (probe_steps < 20 ? probe_steps : 20) : probe_steps;
                    e = cudaEventRecord(e0, st);
                    if (e == cudaSuccess)
                        rs = run_batched_impl(sj.data(), njobs, n, 0, prec, stream, scales[c],
                                              prec == ROM_AUTO ? kthrs[t] : kAutoKthr, tcw, wl);
                    if (e == cudaSuccess && rs == ROM_OK) e = cudaEventRecord(e1, st);
                    if (e == cudaSuccess && rs == ROM_OK) e = cudaEventSynchronize(e1);
                    if (e == cudaSuccess && rs == ROM_OK) e = cudaEventElapsedTime(&ms, e0, e1);
                }
                if (wl && rs == ROM_E_UNSUPPORTED) {  // a form that does not fit: next candidate
                    rs = ROM_OK;
                    continue;
                }
                if (e == cudaSuccess && rs == ROM_OK) {
                    const double us = 1e3 * ms / probe_steps;
                    if (best < 0.0 || us < best) {
                        best = us;
                        best_scale = scales[c];
                        best_kthr = prec == ROM_AUTO ? kthrs[t] : kAutoKthr;
                        best_tcw = tcw;
                        best_wl = wl;
                    }
                }
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    {
        // graphs captured on the scratch buffers are dropped with them
        std::lock_guard<std::mutex> lk(g_batch_mu);
        for (auto it = g_batch_graphs.begin(); it != g_batch_graphs.end();) {
            bool uses = false;
            for (uintptr_t w : it->first.words)
                for (void* b : bufs) uses |= (w == (uintptr_t)b);
            if (uses) {
                free_batch_graph(it->second);
                it = g_batch_graphs.erase(it);
            } else {
                ++it;
            }
        }
    }
    for (void* b : bufs) cudaFree(b);
    if (e != cudaSuccess) return cuda_fail(e, "rom_autotune_batched");
    if (rs != ROM_OK) return rs;
    {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        g_batch_scale[batch_tune_key(jobs, njobs, prec)] = best_scale;
        if (prec == ROM_AUTO) g_batch_kthr[batch_tune_key(jobs, njobs, prec)] = best_kthr;
        g_batch_tcw[batch_tune_key(jobs, njobs, prec)] = best_tcw;
        g_batch_wl[batch_tune_key(jobs, njobs, prec)] = best_wl;
    }
    if (best_us) *best_us = best;
    return ROM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- rank-3
//
// Many operators (realizations of the system parameters) times many
// forcings in ONE launch (the rank-3 outlook of Sec. 5).  The operators share
// K, R and dt; the state is the rank-3 tensor of nops slabs of M columns,
// stored as one Kv x (M nops) matrix.  A device table holds each operator's
// pointers; cluster c of the persistent kernel advances operator c / cpj on
// its own column block, so every cluster keeps one operator resident.

namespace {

std::mutex g_group_mu;
std::map<std::vector<uintptr_t>, GroupOp*> g_group_tables;  // key: t, then the handles

void drop_group_tables(rom_s* h) {
    std::lock_guard<std::mutex> lk(g_group_mu);
    for (auto it = g_group_tables.begin(); it != g_group_tables.end();) {
        bool uses = false;
        for (size_t k = 1; k < it->first.size(); ++k) uses |= (it->first[k] == (uintptr_t)h);
        if (uses) {
            cudaFree(it->second);
            it = g_group_tables.erase(it);
        } else {
            ++it;
        }
    }
}

// The device operator table of this handle list and precision copy t
// (built once, then reused).
rom_status group_table(const rom_t* hs, int nops, int t, const GroupOp** out) {
    std::vector<uintptr_t> key;
    key.push_back((uintptr_t)t);
    for (int i = 0; i < nops; ++i) key.push_back((uintptr_t)hs[i]);
    std::lock_guard<std::mutex> lk(g_group_mu);
    auto it = g_group_tables.find(key);
    if (it == g_group_tables.end()) {
        std::vector<GroupOp> host(nops);
        for (int i = 0; i < nops; ++i)
            host[i] = {hs[i]->Avs_rm[t], hs[i]->Asv_rm[t], hs[i]->g_p[t], hs[i]->C_rm[t]};
        GroupOp* dev = nullptr;
        ROM_CUDA(cudaMalloc(&dev, sizeof(GroupOp) * nops));
        const cudaError_t e = cudaMemcpy(dev, host.data(), sizeof(GroupOp) * nops, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(dev);
            return cuda_fail(e, "rank-3 operator table");
        }
        it = g_group_tables.emplace(key, dev).first;
    }
    *out = it->second;
    return ROM_OK;
}

}  // namespace

extern "C" {

rom_status rom_run_rank3(const rom_t* hs, int nops, void* V, void* S, const void* T, int M,
                         int nsteps, int r, void* traces, int prec, void* stream) {
    if (!hs || nops < 1 || !V || !S || M < 1 || nsteps < 0 || r < 0 || !valid_prec(prec))
        return ROM_E_INVAL;
    const rom_s* h0 = hs[0];
    if (!h0) return ROM_E_INVAL;
    for (int i = 0; i < nops; ++i) {
        const rom_s* h = hs[i];
        if (!h || h->Kv != h0->Kv || h->Ks != h0->Ks || h->R != h0->R || h->dt != h0->dt ||
            h->wavelet != h0->wavelet)
            return ROM_E_INVAL;
        if (h->xref_M != 0) {
            snprintf(g_last_error, sizeof(g_last_error), "rom_run_rank3 takes no reference state");
            return ROM_E_UNSUPPORTED;
        }
    }
    if (prec != ROM_FP32 && prec != ROM_FP64) return ROM_E_UNSUPPORTED;
    if (traces && (r < 1 || h0->R < 1)) return ROM_E_INVAL;
    if (!is_device_ptr(V) || !is_device_ptr(S) || (T && !is_device_ptr(T)) ||
        (traces && !is_device_ptr(traces)))
        return ROM_E_INVAL;
    if (nsteps == 0) return ROM_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int t = prec == ROM_FP64 ? 0 : 1;
    const int Kp = h0->Kp, R = h0->R;
    // each operator gets an equal share of the co-resident clusters
    Rank2Plan p;
    bool ok = false;
    if (prec == ROM_FP32) {
        Rank2Plan p0;
        if (plan_rank2_split_f32(Kp, M, R, &p0)) {
            const int budget = p0.max_active_clusters / nops > 0 ? p0.max_active_clusters / nops : 1;
            ok = plan_rank2_split_f32(Kp, M, R, &p, budget);
            if (ok) p.variant = 2;
        }
    }
    if (!ok) {
        Rank2Plan p0;
        const bool ok0 = prec == ROM_FP64 ? plan_rank2_simt_f64(Kp, M, R, false, &p0)
                                          : plan_rank2_simt_f32(Kp, M, R, false, &p0);
        if (ok0) {
            const int budget = p0.max_active_clusters / nops > 0 ? p0.max_active_clusters / nops : 1;
            ok = prec == ROM_FP64 ? plan_rank2_simt_f64(Kp, M, R, false, &p, budget)
                                  : plan_rank2_simt_f32(Kp, M, R, false, &p, budget);
            if (ok) p.variant = 1;
        }
    }
    if (!ok) {
        snprintf(g_last_error, sizeof(g_last_error), "no rank-3 plan for Kp=%d M=%d", Kp, M);
        return ROM_E_UNSUPPORTED;
    }
    const int cpj = p.nclusters;  // clusters (column-block pairs or blocks) per operator
    p.nclusters = cpj * nops;
    const GroupOp* table = nullptr;
    rom_status gs = group_table(hs, nops, t, &table);
    if (gs != ROM_OK) return gs;
    Rank2Args a = {};
    a.Avs_rm = h0->Avs_rm[t];
    a.Asv_rm = h0->Asv_rm[t];
    a.g_p = h0->g_p[t];
    a.C_p = h0->C_rm[t];
    a.group = table;
    a.group_cpj = cpj;
    a.V = V;
    a.S = S;
    a.Tper = T;
    a.traces = traces;
    a.status = h0->status;
    a.dt = h0->dt;
    a.wavelet = h0->wavelet;
    a.n0 = 0;
    a.Kv = h0->Kv;
    a.Ks = h0->Ks;
    a.Kp = Kp;
    a.R = R;
    a.M = M;
    a.Mtot = M * nops;
    a.col_base = 0;
    a.nsteps = nsteps;
    a.r = traces ? r : 1;
    a.spin_limit = h0->wait_limit;
    cudaError_t e = prec == ROM_FP64   ? launch_rank2_simt_f64(a, p, st)
                    : p.variant >= 2 ? launch_rank2_split_f32(a, p, st)
                                     : launch_rank2_simt_f32(a, p, st);
    if (e != cudaSuccess) return cuda_fail(e, "rank-3 launch");
    return ROM_OK;
}

// ---------------------------------------------------------------- adjoint

}  // extern "C"

namespace {

struct AdjLayout {
    size_t traces, ckpt, work, acomp, gtp, acc, src, total;
    int seg, nseg;
};

// es: bytes of an element (4 FP32, 8 FP64).  The FP32 path also checkpoints
// and reverses Kahan carries; the FP64 path keeps the same slots, unused.
AdjLayout adjoint_layout(const rom_s* h, int M, int nsteps, int ckpt_every, size_t es) {
    AdjLayout L{};
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    L.seg = ckpt_every > 0 && ckpt_every < nsteps ? ckpt_every : nsteps;
    L.nseg = (nsteps + L.seg - 1) / L.seg;
    const size_t kvm = (size_t)(h->Kv + h->Ks) * M;  // one (V, S) pair
    size_t o = 0;
    L.traces = o; o += al(es * (size_t)L.seg * h->R * M);
    L.ckpt = o;   o += al(es * 2 * kvm * (size_t)L.nseg);   // state + Kahan carries
    L.work = o;   o += al(es * 2 * kvm);
    L.acomp = o;  o += al(sizeof(float) * kvm);
    L.gtp = o;    o += al(es * 16 * (size_t)M);
    L.acc = o;    o += al(sizeof(double) * 2);
    // the source term of one launch range of reverse steps
    L.src = o;  o += al(es * (size_t)adj_src_steps(M, h->Kp, L.seg, (int)es) * M * h->Kp);
    L.total = o;
    return L;
}

// The forward sweep with checkpoints, then the reverse sweep segment by
// segment, in element type T (float: ROM_FP32, double: ROM_FP64).
template <typename T>
rom_status adjoint_run(rom_s* h, const void* V0, const void* S0, const void* Tp, int M, int nsteps,
                       const void* ystar, int ckpt_every, void* gV0, void* gS0, void* gT, double* loss,
                       void* workspace, size_t ws_bytes, const AdjPlan& ap, cudaStream_t st) {
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int prec = F32 ? ROM_FP32 : ROM_FP64;
    constexpr int t = F32 ? 1 : 0;  // index of the handle's operator copies
    const AdjLayout L = adjoint_layout(h, M, nsteps, ckpt_every, sizeof(T));
    void* own_ws = nullptr;
    if (!workspace) {
        ROM_CUDA(cudaMalloc(&own_ws, L.total));
        workspace = own_ws;
    } else if (ws_bytes < L.total) {
        return ROM_E_INVAL;
    }
    char* ws = static_cast<char*>(workspace);
    T* traces = reinterpret_cast<T*>(ws + L.traces);
    T* ckpt = reinterpret_cast<T*>(ws + L.ckpt);
    T* work = reinterpret_cast<T*>(ws + L.work);
    float* acomp = reinterpret_cast<float*>(ws + L.acomp);
    T* gtp = reinterpret_cast<T*>(ws + L.gtp);
    double* acc = reinterpret_cast<double*>(ws + L.acc);
    T* asrc = reinterpret_cast<T*>(ws + L.src);
    const size_t nv = (size_t)h->Kv * M, ns = (size_t)h->Ks * M, kvm = nv + ns;
    T* wV = work;
    T* wS = work + nv;
    T* wcV = work + kvm;  // FP32 carries (FP32 path only)
    T* wcS = work + kvm + nv;
    const size_t rec = (size_t)h->R * M;
    const T* ys = static_cast<const T*>(ystar);
    rom_status s = ROM_OK;
    cudaError_t e = cudaSuccess;
    auto forward = [&](int n_start, int len) -> rom_status {
        RunBufs b = {wV, wS, const_cast<void*>(Tp), nullptr, F32 ? (void*)wcV : nullptr,
                     F32 ? (void*)wcS : nullptr, traces};
        return run_rank2_device(h, b, M, len, n_start, 1, prec, false, st);
    };
    // ---- forward sweep: checkpoints, traces, misfit
    e = cudaMemcpyAsync(wV, V0, sizeof(T) * nv, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(wS, S0, sizeof(T) * ns, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(wcV, 0, sizeof(T) * kvm, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(double) * 2, st);
    const int dt_code = F32 ? 1 : 0;  // element type codes of launch_rel_l2
    for (int k = 0; k < L.nseg && e == cudaSuccess && s == ROM_OK; ++k) {
        const int n_start = k * L.seg, len = nsteps - n_start < L.seg ? nsteps - n_start : L.seg;
        e = cudaMemcpyAsync(ckpt + (size_t)k * 2 * kvm, work, sizeof(T) * 2 * kvm,
                            cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) break;
        s = forward(n_start, len);
        if (s == ROM_OK)
            e = launch_rel_l2(traces, dt_code, ys + (size_t)n_start * rec, dt_code, (size_t)len * rec, acc, st);
    }
    // ---- reverse sweep, segment by segment (recomputing each one's traces)
    if (e == cudaSuccess && s == ROM_OK) {
        e = cudaMemsetAsync(gV0, 0, sizeof(T) * nv, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(gS0, 0, sizeof(T) * ns, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(acomp, 0, sizeof(float) * kvm, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(gtp, 0, sizeof(T) * 16 * (size_t)M, st);
    }
    for (int k = L.nseg - 1; k >= 0 && e == cudaSuccess && s == ROM_OK; --k) {
        const int n_start = k * L.seg, len = nsteps - n_start < L.seg ? nsteps - n_start : L.seg;
        if (k != L.nseg - 1) {  // the last segment's traces are still in place
            e = cudaMemcpyAsync(work, ckpt + (size_t)k * 2 * kvm, sizeof(T) * 2 * kvm,
                                cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) break;
            s = forward(n_start, len);
            if (s != ROM_OK) break;
        }
        AdjArgsT<T> aa = {};
        aa.opA_rm = static_cast<const T*>(h->Asv_cm[t]);
        aa.opB_rm = static_cast<const T*>(h->Avs_cm[t]);
        aa.g_p = static_cast<const T*>(h->g_p[t]);
        aa.C_rm = static_cast<const T*>(h->C_rm[t]);
        aa.lamV = static_cast<T*>(gV0);
        aa.lamS = static_cast<T*>(gS0);
        aa.compV = F32 ? acomp : nullptr;
        aa.compS = F32 ? acomp + nv : nullptr;
        aa.Tper = static_cast<const T*>(Tp);
        aa.traces = traces;
        aa.ystar = ys;
        aa.gTpart = gtp;
        aa.status = h->status;
        aa.dt = h->dt;
        aa.wavelet = h->wavelet;
        aa.n0 = 0;
        aa.n_lo = n_start;
        aa.n_hi = n_start + len;
        aa.rec_base = n_start + 1;
        aa.Kv = h->Kv;
        aa.Ks = h->Ks;
        aa.Kp = h->Kp;
        aa.R = h->R;
        aa.M = M;
        {
            // the reverse kernels read the source term precomputed for a range
            // of steps: the segment's latest steps first
            const int nsrc = adj_src_steps(M, h->Kp, L.seg, (int)sizeof(T));
            for (int hi = n_start + len; hi > n_start && e == cudaSuccess;) {
                const int lo = hi - nsrc > n_start ? hi - nsrc : n_start;
                e = launch_adj_source(static_cast<const T*>(h->C_rm[t]), traces, ys, lo, hi - lo, aa.rec_base, M,
                                      h->R, h->Kp, asrc, st);
                aa.src = asrc;
                aa.n_lo = lo;
                aa.n_hi = hi;
                if (e == cudaSuccess) e = launch_adjoint(aa, ap, st);
                hi = lo;
            }
        }
    }
    if (e == cudaSuccess && s == ROM_OK) e = launch_sum_partials(gtp, ap.cs, M, static_cast<T*>(gT), st);
    double hacc[2] = {0.0, 0.0};
    if (e == cudaSuccess && s == ROM_OK) e = cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && s == ROM_OK) e = cudaStreamSynchronize(st);
    if (own_ws) cudaFree(own_ws);
    if (s != ROM_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "rom_adjoint");
    if (loss) *loss = hacc[0];
    return ROM_OK;
}

}  // namespace

extern "C" {

size_t rom_adjoint_workspace_size(rom_t h, int M, int nsteps, int ckpt_every, int prec) {
    if (!h || M < 1 || nsteps < 1 || ckpt_every < 0 || (prec != ROM_FP32 && prec != ROM_FP64)) return 0;
    return adjoint_layout(h, M, nsteps, ckpt_every, prec == ROM_FP64 ? 8 : 4).total;
}

rom_status rom_adjoint(rom_t h, const void* V0, const void* S0, const void* T, int M, int nsteps,
                       const void* ystar, int ckpt_every, void* gV0, void* gS0, void* gT,
                       double* loss, void* workspace, size_t ws_bytes, int prec, void* stream) {
    if (!h || !V0 || !S0 || !T || !ystar || !gV0 || !gS0 || !gT || M < 1 || nsteps < 1 ||
        ckpt_every < 0 || h->R < 1)
        return ROM_E_INVAL;
    if (prec != ROM_FP32 && prec != ROM_FP64) return ROM_E_UNSUPPORTED;
    if (h->xref_M != 0 && h->xref_M != M) return ROM_E_INVAL;  // reference state of another ensemble
    const void* ptrs[] = {V0, S0, T, ystar, gV0, gS0, gT};
    for (const void* p : ptrs)
        if (!is_device_ptr(p)) return ROM_E_INVAL;
    AdjPlan ap;
    if (!plan_adjoint(h->Kp, M, h->R, &ap, prec == ROM_FP64)) {
        snprintf(g_last_error, sizeof(g_last_error), "no adjoint plan for Kp=%d M=%d (prec %d)", h->Kp, M, prec);
        return ROM_E_UNSUPPORTED;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return prec == ROM_FP64
               ? adjoint_run<double>(h, V0, S0, T, M, nsteps, ystar, ckpt_every, gV0, gS0, gT, loss,
                                     workspace, ws_bytes, ap, st)
               : adjoint_run<float>(h, V0, S0, T, M, nsteps, ystar, ckpt_every, gV0, gS0, gT, loss,
                                    workspace, ws_bytes, ap, st);
}

rom_status rom_rel_l2(const void* x, int x_dtype, const void* ref, int ref_dtype, size_t n,
                      double* out, void* stream) {
    if (!x || !ref || !out || n == 0 || (x_dtype != 0 && x_dtype != 1) ||
        (ref_dtype != 0 && ref_dtype != 1))
        return ROM_E_INVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* acc = nullptr;
    ROM_CUDA(cudaMalloc(&acc, 2 * sizeof(double)));
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), st);
    if (e == cudaSuccess) e = launch_rel_l2(x, x_dtype, ref, ref_dtype, n, acc, st);
    double hacc[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(acc);
    if (e != cudaSuccess) return cuda_fail(e, "rom_rel_l2");
    *out = hacc[1] > 0.0 ? sqrt(hacc[0] / hacc[1]) : sqrt(hacc[0]);
    return ROM_OK;
}

}  // extern "C"
