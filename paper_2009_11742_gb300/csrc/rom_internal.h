// Internal declarations of librom (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/rom.h"

namespace romk {

// Record a message for rom_last_error() (this thread).
void set_last_error(const char* msg);
// Record "where: <CUDA error text>" for rom_last_error() and map the error to
// a status: ROM_E_NOMEM for an allocation failure, ROM_E_CUDA otherwise.
rom_status cuda_fail(cudaError_t e, const char* where);

// Arguments of one rank-2 launch (all device pointers).  Element type T of
// the state-like buffers is double for ROM_FP64 and float otherwise.
// One operator of a grouped (rank-3) launch: its handle's device copies.
struct GroupOp {
    const void* Avs_rm;
    const void* Asv_rm;
    const void* g_p;
    const void* C_p;
    // work-list launches only (the batched scheduler): the job's own state,
    // periods, traces, status word and constants, its padded size Kp, the
    // columns of one item (Wa, a multiple of 8), and whether its receiver
    // rows are read from C_p rather than staged in shared memory
    void* V;
    void* S;
    const void* Tper;
    void* traces;
    int* status;
    double dt;
    int Kv, Ks, R, M, wavelet, Kp, Wa, c_global;
};

// One item of a work-list launch: columns [col0, col0 + ncol) of job `job` of
// the operator table.
struct WorkItem {
    int job, col0, ncol, pad;
};

struct Rank2Args {
    const void* Avs_rm;  // Kp x Kp row-major, zero padded (T)
    const void* Asv_rm;  // Kp x Kp row-major, zero padded (T)
    const void* g_p;     // Kp (T)
    const void* C_p;     // R x Kp row-major (T); may be null when R == 0
    void* V;             // Kv x Mtot column-major (T)
    void* S;             // Ks x Mtot column-major (T)
    void* compV;         // optional Kahan carry, Kv x Mtot float
    void* compS;         // optional Kahan carry, Ks x Mtot float
    const void* Tper;    // Mtot Ricker periods (T) or null
    const void* ftab;    // nsteps x Mtot forcing table (T) or null
    void* traces;        // nrec x Mtot x R (T) or null
    int* status;         // device status word
    double dt;
    long long n0;
    int Kv, Ks, Kp, R;
    int M;         // columns covered by this launch
    int Mtot;      // columns of the caller's arrays (leading extent of ftab rows)
    int col_base;  // first caller column covered by this launch
    int Wv;        // valid columns per cluster
    int Wa;        // allocated columns per cluster (multiple of the column group)
    int nsteps;
    int r;         // trace interval (> 0 when traces != null)
    int rpc;       // trace rows of C per CTA
    int nrt;               // 32-row tiles owned per CTA by the one-block kernel (1 or 2)
    long long spin_limit;  // clock cycles a device-side wait may last before ROM_E_TIMEOUT
    int debug_skip_push;   // fault injection: CTA 0 never publishes (forces the timeout path)
    int wavelet;           // source signal of the periods: 0 Ricker, 1 first derivative of a Gaussian
    const void* Xv;        // reduced reference state, velocity part, Kv x Mtot (T), or null
    const void* Xs;        // stress part, Ks x Mtot (T), or null
    // rank-3 grouped launch: operator table (device) and clusters (one-block
    // kernel: column blocks) per operator; cluster c advances operator
    // c / group_cpj on that operator's M columns, global columns
    // job * M + local.  Null: one operator (the fields above).
    const GroupOp* group;
    int group_cpj;
    int c_global;          // one-block kernel: read receiver rows from C_p instead of shared memory
    // work-list launch: clusters take items from `items` (nitems of them) in
    // the order a global counter hands them out; the operator table `group`
    // then also carries each job's state and constants.  Null: off.
    const WorkItem* items;
    int nitems;
    int* item_counter;
};

// Step-time models, microseconds per leapfrog step of one cluster, fitted on
// GB300: the two-block split kernel with W columns per block (operators in
// registers), and a kernel that streams its operators from L2 with nrt
// 32-row tiles per CTA and W columns (one-block kernel above Kp = 512, the
// work-list kernel).
inline double model_split_us(int Kp, int W) { return 2.24 + 0.466 * W * (Kp / 512.0); }
inline double model_streamed_us(int Kp, int nrt, int W) { return 3.5 + 0.71 * nrt * W * (Kp / 1024.0); }

// Launch plan chosen by the host for a rank-2 call.
struct Rank2Plan {
    int cs;        // cluster size (CTAs)
    int KI;        // 64-wide k groups per thread
    int cb;        // columns per register group
    int Wv, Wa;    // valid / allocated columns per cluster
    int nclusters; // clusters launched
    int max_active_clusters;
    size_t smem;
    bool resident; // operators kept in registers for the whole run
    int variant;   // 1: one-block, 2: two-block split-role, 3: two-block dataflow
    bool c_global; // one-block: the CTA's receiver rows are read from global memory (too many to stage)
    int nrt;       // one-block kernel: 32-row tiles per CTA (2 when Kp > 512)
    // streaming companion (two-block variant only): the last comp_cols
    // columns run on comp_n clusters of comp_cs CTAs, comp_W columns each,
    // beside the split kernel; comp_cols = 0: none
    int comp_cs = 0, comp_n = 0, comp_W = 0, comp_cols = 0;
};

// Host launchers (defined in the kernel translation units).  Return a CUDA
// error code; `plan` must come from plan_rank2_simt.
cudaError_t launch_rank2_simt_f32(const Rank2Args& a, const Rank2Plan& plan, cudaStream_t st);
cudaError_t launch_rank2_simt_f64(const Rank2Args& a, const Rank2Plan& plan, cudaStream_t st);
// Fill `plan` for M columns; returns false if the shape is not supported.
bool plan_rank2_simt_f32(int Kp, int M, int R, bool rank1, Rank2Plan* plan, int cluster_budget = 0);
bool plan_rank2_simt_f64(int Kp, int M, int R, bool rank1, Rank2Plan* plan, int cluster_budget = 0);

// Two-block split-role FP32 kernels (velocity and stress rows on different
// CTAs): variant 2 synchronises with a cluster barrier per phase, variant 3
// with per-block mbarriers fed by asynchronous stores (bounded waits).
bool plan_rank2_split_f32(int Kp, int M, int R, Rank2Plan* plan, int cluster_budget = 0);
bool plan_rank2_dataflow_f32(int Kp, int M, int R, Rank2Plan* plan);
cudaError_t launch_rank2_split_f32(const Rank2Args& a, const Rank2Plan& plan, cudaStream_t st);
// The work-list kernel (FP32, any Kp <= 1024, clusters of cs CTAs): the
// co-resident clusters at `smem` bytes of dynamic shared memory (0: the
// size does not fit), and the launch of ncl clusters (a.group / items /
// nitems / item_counter set).
int worklist_max_clusters(int cs, size_t smem);
size_t worklist_smem(int W, int Kp, int rpc, int nrt);
cudaError_t launch_rank2_worklist_f32(const Rank2Args& a, int cs, int ncl, size_t smem, cudaStream_t st);

// Streaming companion of the split kernel (FP32, Kp <= 512, clusters of 2
// or 4 CTAs, at most 4 columns per cluster; operators streamed from L2).
bool stream_supported(int Kp, int csz);
int stream_max_columns_per_cluster();
cudaError_t launch_rank2_stream_f32(const Rank2Args& a, int csz, int cols_per_cluster, int nclusters,
                                    cudaStream_t st);
// Model-based split at saturation (false: no gain predicted) and the split
// for a caller-pinned number of companion columns.
bool plan_rank2_companion(int Kp, int M, int R, Rank2Plan* plan);
bool plan_rank2_companion_pinned(int Kp, int M, int R, int csz, int cols, Rank2Plan* plan);

// Tensor-core (tcgen05) rank-2 path for ROM_TF32X3 / ROM_BF16X3 / ROM_BF16 / ROM_BF16S.
struct TcArgs {
    const void* Aop[2];   // split operator tiles: [0] Avs (V half), [1] Asv (S half)
    const float* Ascale[2];  // ROM_BF16S: per-row scales 2^(e_r - 7) of the operator digits
    void* X[2];           // exchange tiles: [0] S (operand of the V half), [1] V
    const float* g_p;     // Kp (tensor-core padding)
    const float* C_p;     // R x Kp row-major (or null)
    float* V;             // Kv x Mtot
    float* S;             // Ks x Mtot
    float* compV;         // Kv x Mtot Kahan carries (workspace or caller's)
    float* compS;
    const float* Tper;    // Mtot or null
    const float* ftab;    // nsteps x Mtot or null
    float* traces;        // nrec x Mtot x R or null
    int* status;
    double dt;
    long long n0;
    long long spin_limit;
    int Kv, Ks, Kp, R, M, Mtot, W, nsteps, r, rpc, stages;
    int wavelet;          // source signal of the periods (see Rank2Args)
    const float* Xv;      // reduced reference state (see Rank2Args), or null
    const float* Xs;
};
struct TcPlan {
    int prec, cs, W, stages, nclusters, rpc, max_active_clusters;
    size_t smem;
};
size_t tc_operator_bytes_for(int prec, int Kp);
// Offset of the per-row scales inside a prepared ROM_BF16S operator (after the tiles).
size_t tc_scale_offset(int prec, int Kp);
int tc_exchange_terms(int prec);
int tc_element_bytes(int prec);
cudaError_t tc_prepare_operator(int prec, const float* A_rm, int Ksrc, int Kp, void* out,
                                cudaStream_t st);
cudaError_t tc_pad_rows(const float* src, int rows, int src_cols, int dst_cols, float* dst,
                        cudaStream_t st);
// Wforce > 0 pins the columns per block (64 or 128; for ROM_BF16S 32, 48, 64 or 80).
bool plan_rank2_tc(int prec, int Kp, int M, int R, int Wforce, TcPlan* plan);
cudaError_t launch_rank2_tc(const TcArgs& a, const TcPlan& plan, cudaStream_t st);

// Reverse-time adjoint kernel (FP32, K <= 512).
// Arguments of the reverse sweep, element type T (float: the FP32 path with
// Kahan-compensated adjoint state; double: the FP64 path, plain sums, the
// carries unused and may be null).
template <typename T>
struct AdjArgsT {
    const T* opA_rm;  // Asv^T as Kp x Kp row-major (the column-major copy of Asv)
    const T* opB_rm;  // Avs^T as Kp x Kp row-major
    const T* g_p;     // Kp
    const T* C_rm;    // R x Kp row-major
    T* lamV;          // Kv x M adjoint of V (in: running value, out: after the range)
    T* lamS;          // Ks x M
    float* compV;     // Kahan carries of lamV / lamS (FP32 path)
    float* compS;
    const T* Tper;    // M periods
    const T* traces;  // forward records: record k = C V^{rec_base + k}, [k][m][j]
    const T* ystar;   // targets: record n = ystar^{n+1}, [n][m][j]
    T* gTpart;        // cs x M per-CTA partial dL/dT (in/out)
    const T* src;     // C^T r of the range's steps, [n - n_lo][m][Kp] (adj_source_kernel)
    int* status;
    double dt;
    long long n0;
    int n_lo, n_hi;       // reverse steps n_hi-1 .. n_lo
    int rec_base;
    int Kv, Ks, Kp, R, M, Wv, Wa;
    int nrt;              // 32-row tiles the layout holds per CTA (FP32 above Kp = 512)
    int wavelet;          // source signal of the periods (see Rank2Args)
};
using AdjArgs = AdjArgsT<float>;
struct AdjPlan {
    int cs, KI, cb, Wv, Wa, nclusters, nrt;
    size_t smem;
    bool f64;         // the FP64 instance (Kp <= 512)
    double model_us;  // modelled µs per reverse step (cluster-size choice)
    bool split;       // the split-role kernel (FP32, Kp <= 512): Wv columns per block, two blocks per cluster
};
bool plan_adjoint(int Kp, int M, int R, AdjPlan* p, bool f64 = false);
cudaError_t launch_adjoint(const AdjArgsT<float>& a, const AdjPlan& p, cudaStream_t st);
cudaError_t launch_adjoint(const AdjArgsT<double>& a, const AdjPlan& p, cudaStream_t st);
// The reverse step's source term, hoisted out of the recurrence of the
// reverse kernels: src[s][m][k] = sum_jr C[jr][k] r[jr] with r = traces of
// record n + 1 - rec_base minus ystar of step n, n = n_lo + s, s < ns.
constexpr int kAdjSrcSteps = 64;  // most reverse steps per launch of the reverse kernels
// Reverse steps per launch range for M columns of Kp rows within a segment of
// seg steps: at most kAdjSrcSteps, and the source buffer (steps x M x Kp
// elements of es bytes) within about 64 MB.
inline int adj_src_steps(int M, int Kp, int seg, int es) {
    const long long per = (long long)M * Kp * es;
    long long s = per > 0 ? (64ll << 20) / per : kAdjSrcSteps;
    if (s > kAdjSrcSteps) s = kAdjSrcSteps;
    if (s > seg) s = seg;
    return s < 1 ? 1 : (int)s;
}
cudaError_t launch_adj_source(const float* C_rm, const float* traces, const float* ystar, int n_lo, int ns,
                              int rec_base, int M, int R, int Kp, float* src, cudaStream_t st);
cudaError_t launch_adj_source(const double* C_rm, const double* traces, const double* ystar, int n_lo, int ns,
                              int rec_base, int M, int R, int Kp, double* src, cudaStream_t st);
cudaError_t launch_sum_partials(const float* part, int cs, int M, float* out, cudaStream_t st);
cudaError_t launch_sum_partials(const double* part, int cs, int M, double* out, cudaStream_t st);

// Rank-1 ensemble (one realization per CTA, operators streamed every step).
struct Rank1EnsArgs {
    const void* Avs_cm;  // Kp x Kp column-major, zero padded (T)
    const void* Asv_cm;
    const void* g_p;
    const void* C_cm;    // Kp x R: column j is row j of C (T), may be null
    void* V;
    void* S;
    const void* Tper;
    void* traces;
    int* status;
    double dt;
    long long n0;
    int Kv, Ks, Kp, R, M, nsteps, r;
    int wavelet;          // source signal of the periods (see Rank2Args)
    const void* Xv;       // reduced reference state (see Rank2Args), or null
    const void* Xs;
};
cudaError_t launch_rank1_ensemble_f32(const Rank1EnsArgs& a, cudaStream_t st);
cudaError_t launch_rank1_ensemble_f64(const Rank1EnsArgs& a, cudaStream_t st);

// FP64 utilities.
cudaError_t launch_matvec_f64(const double* A_rm, int rows, int cols, int ld, const double* x,
                              double* y, cudaStream_t st);
cudaError_t launch_power_step(const double* y, double* x, int n, double* lam_out, int it,
                              cudaStream_t st);
cudaError_t launch_rel_l2(const void* x, int xd, const void* ref, int rd, size_t n,
                          double* acc2, cudaStream_t st);
// Padded / transposed copies: dst (Kp x Kp, row-major when rm) from a column-major
// rows x cols source of element type src_dtype (0 = f64, 1 = f32).
cudaError_t launch_pad_copy(const void* src, int src_dtype, int rows, int cols, int Kp_rows,
                            int Kp_cols, bool row_major_out, void* dst, int dst_dtype,
                            cudaStream_t st);

}  // namespace romk
