/*
 * rom.h -- C ABI of librom.so, a GB300 (sm_103a) library that integrates
 * rank-2 Galerkin reduced-order models of linear time-invariant systems.
 *
 * The model (Eq. (shwave_rom_ode_tensor), Sec. 3.1) is the velocity/stress
 * pair of reduced ODEs
 *
 *     dV/dt = Avs S + g f(t; T_m)^T,      dS/dt = Asv V,
 *
 * with M realizations stacked as the columns of V (Kv x M) and S (Ks x M)
 * (the rank-2 formulation, Eq. (rom_ode_tensor), Sec. 2.4).  Time stepping is
 * the leapfrog of Sec. 3.1, velocity first, then stress with the new velocity:
 *
 *     V^{n+1} = V^n + dt (Avs S^n + g f_n^T),   S^{n+1} = S^n + dt Asv V^{n+1},
 *
 * with f_n[m] = f(t_n; T_m), t_n = (n0 + n) dt, and the point-source Ricker
 * wavelet of Sec. 3.2 (sparse reduced forcing, Sec. 2.2)
 *
 *     f(t; T) = (1 - 2u) exp(-u),  u = pi^2 (t - 1.5 T)^2 / T^2,
 *
 * or the paper's second signal, the first derivative of a Gaussian
 * (rom_set_wavelet).
 *
 * Receiver traces (seismograms from basis rows, Sec. 4.5.2) are y = C V^{n+1}
 * after every step with (n + 1) mod r == 0.
 *
 * Conventions shared by every entry point
 *  - Every call returns a rom_status.  Nothing aborts, traps or throws across
 *    the ABI.
 *  - Matrices are column-major.  Avs is Kv x Ks, Asv is Ks x Kv, C is R x Kv,
 *    V is Kv x M (ld Kv), S is Ks x M (ld Ks).  A trace buffer holds
 *    floor(nsteps / r) records; record k is R x M column-major at offset
 *    k * R * M (element (j, m) at k*R*M + m*R + j).
 *  - Element type of states, periods, forcing tables and traces: double for
 *    ROM_FP64, float for every other precision.
 *  - Pointers may be device pointers or host pointers (pageable or pinned);
 *    the library tells them apart with cudaPointerGetAttributes.  Device
 *    buffers are used in place and the call is asynchronous on `stream`.
 *    Host buffers are staged through library-owned device memory and the
 *    call returns after the results are copied back (synchronous).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *  - A handle is not re-entrant: do not run two calls on one handle
 *    concurrently on different streams.
 *  - Device-side failures (a non-finite final state, a bounded wait that
 *    ran out) are recorded in a per-handle status word read by
 *    rom_sync_status().
 */
#ifndef ROM_H
#define ROM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rom_s* rom_t;

typedef enum {
    ROM_OK = 0,
    ROM_E_INVAL = 1,       /* bad argument: NULL pointer, size <= 0, misaligned buffer */
    ROM_E_NOMEM = 2,       /* a device or host allocation failed */
    ROM_E_CUDA = 3,        /* a CUDA runtime call failed (see rom_last_error) */
    ROM_E_UNSTABLE = 4,    /* dt * rho >= 2 at rom_create: leapfrog would blow up */
    ROM_E_TIMEOUT = 5,     /* a bounded device wait ran out */
    ROM_E_NONFINITE = 6,   /* the final state holds NaN or Inf */
    ROM_E_UNSUPPORTED = 7, /* shape/precision combination not provided */
    ROM_E_NOCONV = 8       /* the FP64 power iteration of the dt-stability check did not
                              settle within its iteration limit */
} rom_status;

typedef enum {
    ROM_FP64 = 0,   /* FP64 check path: FP64 state, FP64 arithmetic */
    ROM_FP32 = 1,   /* FP32 SIMT products, Kahan-compensated state update */
    ROM_TF32X3 = 2, /* tensor cores, tf32 hi/lo split, 3 products, Kahan update */
    ROM_BF16X3 = 3, /* tensor cores, bf16 3-term operator / 2-term state split */
    ROM_BF16 = 4,   /* tensor cores, plain bf16 products (reported, not accepted) */
    ROM_BF16S = 5,  /* tensor cores, exact sliced-integer bf16: operator rows and state
                       columns as three 8-bit digits with power-of-two scales, six digit
                       products accumulated without rounding, Kahan update */
    ROM_AUTO = 6    /* rom_run_batched / rom_autotune_batched only: each job runs ROM_FP32
                       or ROM_BF16S (both meet the FP32 accuracy bar), BF16S for jobs with
                       max(Kv, Ks) at or above a threshold (256 unless tuned) */
} rom_prec;

typedef enum { ROM_IN_F64 = 0, ROM_IN_F32 = 1 } rom_dtype;

/* ------------------------------------------------------------------ handle */

/*
 * rom_create -- copy a reduced model into library-owned device memory.
 *
 * The reduced operators of Eq. (shwave_rom_ode_tensor) (Sec. 3.1): Avs
 * (Kv x Ks, the paper's velocity operator), Asv (Ks x Kv, the stress
 * operator), the source row g (Kv) of the velocity basis (Sec. 2.2, 3.2) and
 * the receiver rows C (R x Kv; R may be 0 and C NULL) of Sec. 4.5.2.  Inputs
 * are column-major, element type `in_dtype`, host or device; the caller may
 * free them on return.  The library keeps FP64 and FP32 copies (row- and
 * column-major, zero-padded) and the split copies the tensor-core paths use.
 *
 * dt-stability check (stable step, Sec. 4.4 and App. A): rho, the spectral
 * radius of the coupled operator [[0, Avs], [Asv, 0]], equals
 * sqrt(rho(Avs Asv)) and is computed by FP64 power iteration on the GPU.  If
 * dt * rho >= 2 the handle is not created and ROM_E_UNSTABLE is returned.
 * The iteration stops once two successive estimates agree to 1e-14
 * relative; if that has not happened after 20000 iterations the estimate is
 * only a lower bound on rho, so the check cannot be certified: the handle is
 * not created and ROM_E_NOCONV is returned.  *rho_out (may be NULL) receives
 * rho (or, for ROM_E_NOCONV, the last estimate) in every one of these cases.
 * Limits: 1 <= Kv, Ks <= 1024, 0 <= R <= 1024.  Runs on the current device.
 */
rom_status rom_create(const void* Avs, const void* Asv, const void* g, const void* C,
                      int Kv, int Ks, int R, double dt, int in_dtype, rom_t* out,
                      double* rho_out);

/* Free a handle and everything it owns (synchronizes its work first). */
rom_status rom_destroy(rom_t h);

/* The spectral radius computed by rom_create (FP64 power iteration). */
rom_status rom_spectral_radius(rom_t h, double* rho);

/* Read and clear the handle's device status word (synchronizes the device). */
rom_status rom_sync_status(rom_t h, rom_status* device_status);

/* Model dimensions of a handle (any output may be NULL). */
rom_status rom_get_dims(rom_t h, int* Kv, int* Ks, int* R, double* dt);

/* Kernel selection for the rank-2 FP32 path (the FP64 path always uses the
 * one-block kernel):
 *  ROM_KERNEL_AUTO      planner's choice (default: two-block);
 *  ROM_KERNEL_ONE_BLOCK one column block per cluster, every CTA owns 32 rows
 *                       of both V and S;
 *  ROM_KERNEL_TWO_BLOCK two column blocks per cluster half a step apart,
 *                       velocity rows and stress rows on different CTAs, one
 *                       cluster barrier per half-step phase;
 *  ROM_KERNEL_DATAFLOW  the two-block schedule synchronised by per-block
 *                       mbarriers fed with asynchronous remote stores; its
 *                       waits are bounded (rom_set_wait_limit).
 * All compute the same leapfrog (Sec. 3.1); their results agree to FP32
 * rounding. */
enum { ROM_KERNEL_AUTO = 0, ROM_KERNEL_ONE_BLOCK = 1, ROM_KERNEL_TWO_BLOCK = 2,
       ROM_KERNEL_DATAFLOW = 3 };
rom_status rom_set_kernel(rom_t h, int kernel);

/* The launch plan the handle would use for M realizations at precision prec
 * (ROM_FP32 or ROM_FP64): kernel variant (1 one-block, 2 two-block, 3
 * dataflow, 4 two-block with the streaming companion of rom_set_companion on
 * the last columns), cluster size, columns per column block and number of
 * clusters of the main kernel (outputs may be NULL).  ROM_E_UNSUPPORTED for
 * another precision or if no kernel fits. */
rom_status rom_get_plan(rom_t h, int prec, int M, int* variant, int* cluster_size,
                        int* cols_per_block, int* nclusters);

/*
 * rom_set_companion -- the streaming companion of the FP32 two-block kernel.
 * The two-block kernel keeps both operators in the registers of clusters of
 * Kp/32 CTAs (16 at K = 512); clusters that large only fit where a GPU
 * processing cluster has that many free SMs, and the rest of the SMs stay
 * idle.  The companion runs beside it on those SMs as a second kernel on a
 * private stream (forked from and joined back to the caller's stream) and
 * integrates the LAST columns of the run with the same leapfrog: clusters of
 * 2 or 4 CTAs, each owning Kp/size rows of V and S for up to 4 columns,
 * stream their operator rows from L2 every half-step.  Kp <= 512; the run
 * must carry no reduced reference state (otherwise the two-block kernel
 * runs alone).  Results agree with the two-block kernel's to FP32 rounding.
 *   cluster_size 0  (default) the planner decides from a step-time model:
 *                   when the two-block kernel already uses every cluster
 *                   that fits, it narrows the column blocks and hands the
 *                   freed columns to the companion if that is predicted to
 *                   be at least 5 % faster;
 *   cluster_size -1 never;
 *   cluster_size 2 or 4: always, with `columns` (>= 1) columns on the
 *                   companion (all of them when columns >= M).
 * Applies while the kernel choice is ROM_KERNEL_AUTO.  Clears the plans
 * rom_autotune kept.  If the run is captured in a CUDA graph, the two
 * kernels become parallel nodes whose launch order the graph does not fix,
 * so the large clusters may no longer be placed first.  ROM_E_INVAL for
 * another cluster size or columns < 1 with a pinned size.
 */
rom_status rom_set_companion(rom_t h, int cluster_size, int columns);

/* The companion part of the FP32 plan for M realizations: its cluster size,
 * number of clusters and columns (all 0 when the plan has none). */
rom_status rom_get_companion(rom_t h, int M, int* cluster_size, int* nclusters, int* columns);

/*
 * rom_autotune -- measure instead of model: time every candidate launch plan
 * for M realizations at precision `prec` on a probe run of `probe_steps`
 * steps (zero state, every period 45 dt, no traces, library-allocated
 * scratch) and keep the fastest for this handle.  Later rom_run_rank2 /
 * rom_run_rank2_ex calls with the same precision and M use it while the
 * kernel choice (rom_set_kernel) and the tensor-core width
 * (rom_set_tc_columns) are automatic.  Candidates:
 *   ROM_FP32  the two-block and the one-block kernels, each with the cluster
 *             count capped at the co-resident maximum, half and a quarter of
 *             it (wider column blocks on fewer clusters); and, when the
 *             two-block kernel fills every cluster that fits, the same with
 *             4, 8 or 12 fewer columns per block and the freed columns on the
 *             streaming companion (rom_set_companion) in clusters of 2 or 4;
 *   ROM_FP64  the one-block kernel;
 *   tensor-core precisions: every column-block width the precision provides.
 * Every candidate computes the same leapfrog; the FP32 kernels differ only in
 * the order of FP32 roundings (results agree to FP32 rounding).
 * *best_us (may be NULL) receives the chosen plan's probe time per step.
 * Synchronous on `stream`.  Errors: ROM_E_INVAL, ROM_E_UNSUPPORTED (no
 * candidate fits), ROM_E_NOMEM, ROM_E_CUDA, or a device status the probe set.
 */
rom_status rom_autotune(rom_t h, int prec, int M, int probe_steps, double* best_us, void* stream);

/*
 * rom_set_wavelet -- source signal evaluated from the periods T by every run
 * and by the adjoint (Sec. 3.2 supports two): ROM_WAVELET_RICKER (default),
 *   f = (1 - 2u) exp(-u),  u = pi^2 (t - t0)^2 / T^2,
 * or ROM_WAVELET_GAUSS1, the first derivative of a Gaussian, read as the
 * derivative of the same Gaussian envelope scaled to unit peak magnitude,
 *   f = -sqrt(2e) a exp(-a^2),  a = pi (t - t0) / T,
 * both with delay t0 = 1.5 T.  Tabulated forcing (rom_run_rank2_ex) is not
 * affected.  ROM_E_INVAL for another value.
 */
enum { ROM_WAVELET_RICKER = 0, ROM_WAVELET_GAUSS1 = 1 };
rom_status rom_set_wavelet(rom_t h, int wavelet);

/*
 * rom_set_reference -- the reduced reference state of Eq. (rom_ode) and
 * Eq. (rom_ode_tensor), Xhat_ref = Phi^T A X_ref: a time-independent term, one
 * column per realization, split like the state into Xv (Kv x M) and Xs
 * (Ks x M), column-major, FP64 or FP32 (in_dtype), host or device.  Later
 * runs on this handle add it to both halves of every leapfrog step,
 *     V += dt (Avs S + g f + Xv),   S += dt (Asv V + Xs),
 * on every path (rank-2 in every precision, the rank-1 runs with M = 1, the
 * ensemble, the batched launch, and the forward and recomputed sweeps of the
 * adjoint, whose reverse sweep the constant does not change).  Either part
 * may be NULL (zero); both NULL clears it (the default, and the paper's
 * seismic runs, Sec. 3.1).  The data is copied; the caller may free it on
 * return.  A run over a number of columns other than M returns
 * ROM_E_INVAL.  Synchronous.  Errors: ROM_E_INVAL, ROM_E_NOMEM, ROM_E_CUDA.
 */
rom_status rom_set_reference(rom_t h, const void* Xv, const void* Xs, int M, int in_dtype);

/*
 * rom_set_tc_columns -- columns per cluster block of the tensor-core path:
 * 64 or 128 for ROM_TF32X3 / ROM_BF16X3 / ROM_BF16, 32, 48, 64 or 80 for
 * ROM_BF16S, or 0 to let the planner choose (default).  Wider blocks re-read
 * each operator slab fewer times per step; narrower blocks spread the run
 * over more SMs.  A width the precision does not provide makes the next run
 * return ROM_E_UNSUPPORTED.
 */
rom_status rom_set_tc_columns(rom_t h, int cols);

/*
 * rom_set_wait_limit -- bound, in SM clock cycles, on every device-side wait
 * of the dataflow kernel (a consumer waiting for a producer's rows) and of
 * the tensor-core kernels (stage and accumulator handshakes).  A wait that
 * runs out makes the kernel stop, leave cleanly, and record ROM_E_TIMEOUT in
 * the handle's status word (rom_sync_status).  Default
 * 4e9 cycles (about 2 s), far above any legitimate wait.
 */
rom_status rom_set_wait_limit(rom_t h, long long cycles);

/*
 * rom_debug_inject_stall -- failure injection for tests of the timeout path:
 * when on, one CTA of every cluster of ROM_KERNEL_DATAFLOW never publishes
 * its rows, so its peers' waits run out (set a small wait limit first).  The
 * kernel then ends with ROM_E_TIMEOUT instead of hanging.  Off by default.
 */
rom_status rom_debug_inject_stall(rom_t h, int on);

/* ------------------------------------------------------------- integrate */

/*
 * rom_run_rank2 -- the rank-2 Galerkin leapfrog (Eq. (rom_ode_tensor) with the
 * split of Eq. (shwave_rom_ode_tensor), leapfrog of Sec. 3.1): advance all M
 * realizations sharing the handle's operators by nsteps steps, IN PLACE on V
 * (Kv x M) and S (Ks x M).  T (M) holds each realization's source period in
 * time units (signal chosen by rom_set_wavelet).  Steps n = 0 .. nsteps-1 use t_n = (n0 + n) dt.  traces (may be
 * NULL; r must then be 0) receives floor(nsteps / r) records of C V.
 * nsteps == 0 is a no-op.  Errors: ROM_E_INVAL (bad pointer/size, r < 0, or
 * traces without receiver rows), ROM_E_UNSUPPORTED (precision not provided
 * for this shape), ROM_E_CUDA.
 */
rom_status rom_run_rank2(rom_t h, void* V, void* S, const void* T, int M, int nsteps,
                         long n0, int r, void* traces, int prec, void* stream);

/*
 * rom_run_rank2_ex -- rom_run_rank2 with the optional inputs spelled out.
 *  ftab : if non-NULL, an nsteps x M forcing table (element [n * M + m]) used
 *         in place of the wavelet; T is then ignored (may be NULL).
 *         This is the dense reduced-forcing mode of Sec. 2.2 (precomputed
 *         Phi^T f(t) at every target time).
 *  compV, compS : optional FP32 Kahan compensation carries (Kv x M, Ks x M,
 *         float, device).  When given they are read at the start and written
 *         at the end, so that a run split into chunks (n0 advanced by each
 *         chunk's nsteps) is bit-identical to one long run.  Ignored by
 *         ROM_FP64.
 */
rom_status rom_run_rank2_ex(rom_t h, void* V, void* S, const void* T, const void* ftab,
                            void* compV, void* compS, int M, int nsteps, long n0, int r,
                            void* traces, int prec, void* stream);

/*
 * rom_run_rank1 -- the rank-1 Galerkin ROM (Eq. (rom_ode), Sec. 2.2): one
 * realization (v: Kv, s: Ks, period T) advanced by the same leapfrog, two
 * matrix-vector products per step (the memory-bound GEMV of Sec. 2.3).  It is
 * the in-house baseline the rank-2 path is compared against.
 */
rom_status rom_run_rank1(rom_t h, void* v, void* s, double T, int nsteps, long n0, int r,
                         void* trace, int prec, void* stream);

/*
 * rom_run_rank1_ensemble -- M independent rank-1 runs in one launch, one
 * realization per thread block, with no reuse of operator reads across
 * realizations: every realization streams both operators from memory every
 * step.  This is the GPU counterpart of running many single-threaded rank-1
 * ROMs side by side (Sec. 4.3, 4.5.2).  Arguments as rom_run_rank2.
 */
rom_status rom_run_rank1_ensemble(rom_t h, void* V, void* S, const void* T, int M,
                                  int nsteps, long n0, int r, void* traces, int prec,
                                  void* stream);

/*
 * rom_run_batched -- many ensembles at once: job i advances its handle's
 * model (any Kv, Ks <= 1024) for its M columns exactly as rom_run_rank2 would
 * with n0 = 0, and all jobs run in ONE launch of a CUDA graph on `stream`.
 * With prec = ROM_FP32 (and no job carrying a reduced reference state) the
 * graph can hold ONE persistent launch for all jobs: co-resident clusters of
 * 2 CTAs (by default) take (job, column block) items from a device work
 * list, longest first, in the order a counter hands them out, until none
 * are left; a job's rows are dealt out to the CTAs of whichever cluster
 * takes one of its items, and its operators are read from L2.  The
 * summation order differs from rom_run_rank2's (the results agree to FP32
 * rounding, column by column).  The alternative is one launch per job:
 * every job gets a share of the GPU proportional to its work per step,
 * 4 K^2 M (the rank-2 GEMM cost of Sec. 2.5), which sets its columns per
 * cluster block, and the longest jobs are issued first; each column's
 * arithmetic is then rom_run_rank2's (bitwise equal results).  FP32 lists
 * take the form pinned with rom_set_batched_form or measured by
 * rom_autotune_batched, else the one the step-time models predict faster
 * (see rom_set_batched_form); other precisions run one launch per job.  The graph is built
 * (captured and instantiated) on the first call for a given job list and
 * replayed afterwards.  Requirements: device buffers only, one job per
 * handle, traces (per job, optional) need r > 0 and receiver rows.
 * With prec = ROM_AUTO every job takes ROM_FP32 or ROM_BF16S by its size
 * (the threshold that rom_autotune_batched measured for this job list, else
 * 256).  A tensor-core job runs blocks as wide as its columns allow (the
 * narrowest width that holds all M columns, else the widest; a width pinned
 * with rom_set_tc_columns wins): an MMA costs the same at every width, so
 * among jobs that share the SMs wide blocks give the most columns per SM.
 * Asynchronous on `stream`.  This is the first step of the rank-3
 * outlook of Sec. 5 (many operators and many forcings in one launch).
 */
typedef struct {
    rom_t h;         /* the job's model */
    void* V;         /* Kv x M, column-major, device, updated in place */
    void* S;         /* Ks x M */
    const void* T;   /* M periods, or NULL for no forcing */
    int M;           /* realizations of this job */
    void* traces;    /* floor(nsteps / r) records of R x M, or NULL */
} rom_job;
rom_status rom_run_batched(const rom_job* jobs, int njobs, int nsteps, int r, int prec,
                           void* stream);

/*
 * rom_run_rank3 -- the rank-3 outlook of Sec. 5: many realizations of the
 * system operator (nops handles) times many forcings (M columns each) in ONE
 * launch of the persistent kernel.  The handles must share Kv, Ks, R, dt and
 * the wavelet, and carry no reference state.  The state is the rank-3
 * tensor of nops slabs of M columns stored as one column-major matrix:
 * V is Kv x (M nops) (operator i owns columns [i M, (i+1) M)), S is
 * Ks x (M nops), T (or NULL) holds M nops periods in the same order, and
 * traces (optional, r > 0) holds floor(nsteps / r) records of
 * R x (M nops).  Each operator gets an equal share of the GPU's co-resident
 * clusters, each of which keeps one operator in registers; the result for
 * operator i equals rom_run_rank2 on handle i over its slab.  Device
 * buffers only, n0 = 0, ROM_FP32 or ROM_FP64 (other precisions:
 * ROM_E_UNSUPPORTED).  Asynchronous on `stream`; device-side status goes to
 * the first handle.  The first call for a handle list copies a small
 * operator table to the device (synchronous); it is kept until one of the
 * handles is destroyed.
 */
rom_status rom_run_rank3(const rom_t* handles, int nops, void* V, void* S, const void* T, int M,
                         int nsteps, int r, void* traces, int prec, void* stream);

/*
 * rom_autotune_batched -- the batching schedule by measurement: replay the
 * job list's captured graph on scratch copies of its state (zero state,
 * every period 45 dt, no traces) for `probe_steps` steps with the SMs shared
 * in proportion to each job's work times a scale of 0.5, 1, 2 and 4 (fewer
 * or more clusters per job than its share), and keep the fastest scale for
 * this list of (handle, M) pairs: later rom_run_batched calls with the same
 * handles and widths use it.  The scale affects the SIMT jobs (the
 * tensor-core jobs plan their own widths).  With prec = ROM_AUTO it also
 * tries the size thresholds 0 (every job BF16S), 256, 512 and none (every
 * job FP32), and with tensor-core jobs both the batch widths and the ones
 * the planner picks for a job alone; with ROM_FP32 it also times the
 * work-list form; it keeps the fastest combination.  *best_us (may be
 * NULL) receives the chosen schedule's probe time per step.  Synchronous on
 * `stream`.  Errors as for rom_run_batched, plus ROM_E_NOMEM.
 */
rom_status rom_autotune_batched(const rom_job* jobs, int njobs, int prec, int probe_steps,
                                double* best_us, void* stream);

/*
 * rom_set_batched_form -- pin how rom_run_batched runs this FP32 job list
 * (the same handles and widths; buffers and step counts may change), as
 * rom_autotune_batched would: cluster_size 2, 4 or 8 with width_cap a
 * multiple of 8 in [8, 256] selects the work-list launch with clusters of
 * that many CTAs and at most width_cap columns per item; cluster_size 0
 * selects one launch per job (width_cap ignored).  Without a pinned or
 * tuned form, an FP32 list runs the form that the library's step-time
 * models predict faster for it: the work-list launch with clusters of 2
 * and a cap of 32, or one launch per job (chosen at the list's first call
 * and kept).  prec must be ROM_FP32.  Errors: ROM_E_INVAL (null or empty
 * list, a null handle, M < 1, another precision, a form outside the above).
 */
rom_status rom_set_batched_form(const rom_job* jobs, int njobs, int prec, int cluster_size, int width_cap);

/*
 * rom_adjoint -- gradients of the receiver-trace misfit
 *     L = sum_{n=1..N} sum_m || C V_m^n - ystar_m^n ||^2
 * with respect to the initial state (V0, S0) and the Ricker periods T, by a
 * reverse-time leapfrog (the paper has no adjoint; the reverse step is the
 * exact transpose of the forward step of Sec. 3.1):
 *     lamV += 2 C^T r^{n+1} + dt Asv^T lamS ,  dL/dT_m += dt g^T lamV df/dT ,
 *     lamS += dt Avs^T lamV ,                  n = N-1 .. 0,
 * r^n = C V^n - ystar^n.  ystar holds N records, record n-1 = ystar^n as
 * R x M column-major ([n-1][m][j]).  The forward states come from a forward
 * sweep that keeps a checkpoint (V, S and their Kahan carries) every
 * ckpt_every steps (0: keep every trace, one segment) and recomputes each
 * segment's traces, bit for bit, before reversing it.
 * Outputs: gV0 (Kv x M), gS0 (Ks x M), gT (M) on the device; *loss (host).
 * prec: ROM_FP32 (V0, S0, T, ystar and the outputs float; the adjoint state
 * Kahan-compensated; Kv, Ks <= 1024, and above 512 the reverse kernel reads
 * the transposed operators from L2 every half-step instead of keeping them
 * in registers) or ROM_FP64 (the check path: all of them double, plain
 * FP64 sums; Kv, Ks <= 512); other precisions: ROM_E_UNSUPPORTED.
 * workspace: device, rom_adjoint_workspace_size bytes for the same prec, or
 * NULL to let the library allocate it for the call.  Device buffers only.
 * Synchronous on `stream`.
 */
rom_status rom_adjoint(rom_t h, const void* V0, const void* S0, const void* T, int M, int nsteps,
                       const void* ystar, int ckpt_every, void* gV0, void* gS0, void* gT,
                       double* loss, void* workspace, size_t ws_bytes, int prec, void* stream);
/* Workspace bytes rom_adjoint needs (0 for unsupported arguments). */
size_t rom_adjoint_workspace_size(rom_t h, int M, int nsteps, int ckpt_every, int prec);

/* ------------------------------------------------------ ensemble statistics */

/*
 * rom_trace_stats -- per-receiver statistics of an ensemble of receiver
 * traces: the mean and percentile bands of the seismograms over the
 * realizations, as in the Monte Carlo study of Sec. 4.5.2 (there over 512
 * samples of the source period).
 *   traces   device float, nrec x M x R in the layout rom_run_rank2 writes
 *            (record k, realization m, receiver j at traces[(k M + m) R + j]);
 *            every value finite.
 *   probs    host array of nprobs probabilities in [0, 1] (nprobs <= 16).
 *   mean_out device double, nrec x R (may be NULL): mean over the M
 *            realizations, summed in FP64 by a fixed pairwise tree.
 *   q_out    device double, nprobs x nrec x R (may be NULL): for each p the
 *            quantile by linear interpolation between order statistics
 *            (Hyndman-Fan type 7): h = (M - 1) p, i = floor(h), t = h - i,
 *            q = x(i) + t (x(i+1) - x(i)) with x(.) the values sorted
 *            ascending on the device, evaluated as b - (1 - t)(b - a) when
 *            t >= 1/2 (a = x(i), b = x(i+1)).
 * 1 <= M <= 4096.  Asynchronous on `stream`.  Errors: ROM_E_INVAL (sizes,
 * host pointers, a probability outside [0, 1]), ROM_E_CUDA.
 */
rom_status rom_trace_stats(const float* traces, int nrec, int R, int M, const double* probs,
                           int nprobs, double* mean_out, double* q_out, void* stream);

/* ------------------------------------------------------------- utilities */

/*
 * rom_rel_l2 -- FP64 relative L2 error ||x - ref||_2 / ||ref||_2 (the error
 * measure of Eq. (errors), Sec. 4.4) of two device vectors of n elements,
 * element types x_dtype / ref_dtype (rom_dtype).  Synchronous; *out gets the
 * ratio (or ||x - ref|| when ||ref|| == 0).
 */
rom_status rom_rel_l2(const void* x, int x_dtype, const void* ref, int ref_dtype, size_t n,
                      double* out, void* stream);

/*
 * rom_spectral_radius_noalloc -- the dt-stability check of rom_create (the
 * spectral radius of [[0, Avs], [Asv, 0]] by FP64 power iteration) for
 * callers that cannot allocate device memory: code that runs where
 * cudaMalloc is unavailable or forbidden, such as a host that hands the
 * library a fixed memory budget, or a section that must not grow the device
 * footprint.  It allocates nothing.  The paper has no counterpart; it exists
 * for those callers only.
 *
 * Avs (Kv x Ks) and Asv (Ks x Kv) are the caller's column-major FP64 DEVICE
 * buffers (host pointers are refused with ROM_E_INVAL).  *rho receives the
 * same quantity rom_create computes.  The iteration's work vectors live in a
 * fixed file-scope device array of 3 * 4096 + 65 doubles (about 99 KB) that
 * every GPU which loads the library holds until the process exits; Kv or Ks
 * above 4096 is refused with ROM_E_INVAL.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls on a device share the array and it
 * keeps the last call's contents (each call re-initialises what it reads), so
 * calls that overlap on the GPU -- on two streams, or from two host threads --
 * race and must be serialised by the caller.  The address is looked up once
 * per device and kept: after cudaDeviceReset (or any other teardown of the
 * device's primary context) the cached address is stale, so do not call this
 * entry point again in that process after such a reset.  Synchronous on
 * `stream`.  Errors: ROM_E_INVAL (sizes, host buffers, or buffers that live
 * on a device other than the current one), ROM_E_NOCONV (no convergence
 * within 20000 iterations; *rho then holds the last estimate), ROM_E_CUDA or
 * ROM_E_NOMEM (a CUDA call failed; rom_last_error gives the text).
 */
rom_status rom_spectral_radius_noalloc(const double* Avs, const double* Asv, int Kv, int Ks,
                                       double* rho, void* stream);

/*
 * rom_measure_peak -- measure, on the current device, a denominator of the
 * roofline fractions this library reports (the paper has no counterpart: it
 * measures CPU runs only).  Each kind is one throughput microbenchmark over
 * every SM, run once untimed and once timed with CUDA events on `stream`:
 *   ROM_PEAK_FP32  FP32 FMA pipe: 8 independent FMA chains per thread, 4
 *                  blocks of 512 threads per SM; *value in TFLOP/s (2 per FMA);
 *   ROM_PEAK_FP64  the same in FP64; TFLOP/s;
 *   ROM_PEAK_TF32  tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, 100000
 *                  back-to-back MMAs per SM from resident shared-memory tiles
 *                  into one tensor-memory accumulator; TFLOP/s;
 *   ROM_PEAK_BF16  the same with kind::f16 BF16 operands, K = 16; TFLOP/s;
 *   ROM_PEAK_L2    512 passes of 16-byte L2-cached loads over a 32 MB
 *                  (L2-resident) buffer; GB/s.
 * *ms (may be NULL) receives the timed launch's duration.  Synchronous.
 * Allocates a few MB of scratch (32 MB for ROM_PEAK_L2) for the call.
 * Errors: ROM_E_INVAL (kind), ROM_E_TIMEOUT (an MMA completion wait ran past
 * about 2 s), ROM_E_CUDA / ROM_E_NOMEM.
 */
enum { ROM_PEAK_FP32 = 0, ROM_PEAK_FP64 = 1, ROM_PEAK_TF32 = 2, ROM_PEAK_BF16 = 3, ROM_PEAK_L2 = 4 };
rom_status rom_measure_peak(int kind, double* value, double* ms, void* stream);

/* Human-readable name of a status code (static storage). */
const char* rom_status_string(rom_status s);

/* Text of the last CUDA error seen by this thread (static per thread). */
const char* rom_last_error(void);

/* Library version as major * 10000 + minor * 100 + patch. */
int rom_version(void);

/*
 * ---- Rank-2 full-order model (FOM) of the test case (Sec. 3) ----
 *
 * The axisymmetric elastic shear-wave system of Eq. (fom_asym) in
 * velocity-stress form on the shell r_cmb <= r <= r_earth, 0 <= theta <= pi,
 * a homogeneous material (density rho, shear speed vs, mu = rho vs^2; the
 * single layer of App. A), discretized on a second-order staggered grid of
 * Nr x Ntheta intervals in flux form:
 *     v        at (r_{i+1/2}, theta_j),       i in [0, Nr), j in [1, Ntheta)
 *     sigma_rp at (r_i, theta_j),             i in [1, Nr), j in [1, Ntheta)
 *     sigma_tp at (r_{i+1/2}, theta_{j+1/2}), i in [0, Nr), j in [1, Ntheta - 1)
 * with v = 0 on the axis and sigma_rp = 0 on the axis and the free surfaces
 * (Sec. 3), and sigma_tp = 0 next to the axis.  At most four non-zeros per
 * velocity row and two per stress row.  Advanced by the velocity-first
 * leapfrog for M forcing realizations at once (the rank-2 FOM,
 * Eq. (shwave_ode_tensor)); each run is one point source on one velocity
 * unknown whose signal has period T_m (ROM_WAVELET_*, delay 1.5 T).
 */
typedef struct rom_fom_s* rom_fom_t;

/* rom_fom_create -- grid, material and time step; lengths in m, rho in
 * kg/m^3, vs in m/s, dt in s.  The caller chooses a stable dt (the leapfrog
 * needs dt rho(L) < 2).  Synchronous.  Errors: ROM_E_INVAL (Nr < 2 or
 * > 65535, Ntheta < 3, non-positive or non-finite values, more than 2^31 unknowns
 * per field), ROM_E_NOMEM, ROM_E_CUDA. */
rom_status rom_fom_create(int Nr, int Ntheta, double r_cmb, double r_earth, double rho, double vs,
                          double dt, rom_fom_t* out);
rom_status rom_fom_destroy(rom_fom_t f);

/* rom_fom_set_passes -- 1 (default): one fused pass per step that reads
 * and writes every state value once (8 bytes per unknown and realization
 * in FP32), ping-ponging between the caller's buffers and a library-owned
 * second set (allocated on the first run that needs it, sized by M); 2: a
 * velocity pass then a stress pass in place (12 bytes).  Both compute the
 * same arithmetic.  ROM_E_INVAL for another value. */
rom_status rom_fom_set_passes(rom_fom_t f, int passes);

/* Unknowns per realization: velocity Nr (Ntheta - 1), sigma_rp
 * (Nr - 1)(Ntheta - 1), sigma_tp Nr (Ntheta - 2). */
rom_status rom_fom_dims(rom_fom_t f, int* nv, int* n1, int* n2);

/*
 * rom_fom_run -- nsteps leapfrog steps (t_n = (n0 + n) dt) of M realizations,
 * in place.  States are unknown-major with the M realizations contiguous
 * per unknown (device, FP64 or FP32 per prec):
 *     V[k M + m], k = i (Ntheta - 1) + (j - 1);
 *     S1[k M + m], k = (i - 1)(Ntheta - 1) + (j - 1);
 *     S2[k M + m], k = i (Ntheta - 2) + (j - 1).
 * T (M periods, or NULL for no forcing) drives velocity unknown src.
 * recv (device int[nrecv], velocity unknowns) are recorded after every step
 * with (n + 1) mod r == 0 into traces[(rec nrecv + k) M + m] (NULL: none).
 * The run is a CUDA graph of 64 steps, captured on the first call for a
 * given set of buffers and arguments and replayed; it is asynchronous on
 * `stream` (the first fused run allocates the second buffer set).  A handle is not re-entrant across concurrent streams.  Errors:
 * ROM_E_INVAL (host buffers, bad indices), ROM_E_UNSUPPORTED (prec other than
 * ROM_FP32 / ROM_FP64), ROM_E_CUDA.
 */
rom_status rom_fom_run(rom_fom_t f, void* V, void* S1, void* S2, int M, int nsteps, long n0,
                       int src, const void* T, int wavelet, const int* recv, int nrecv, int r,
                       void* traces, int prec, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ROM_H */
