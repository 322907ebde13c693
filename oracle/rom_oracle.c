/*
 * FP64 reference ("oracle") for the rank-2 Galerkin ROM leapfrog.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or constant with the CUDA library and must never serve as a
 * fallback for it.
 *
 * What it computes (all in double precision, plain loops, natural index
 * order, one realization at a time):
 *
 *   Reduced model, Eq. (shwave_rom_ode_tensor), Sec. 3.1:
 *       dV/dt = Avs S + g f(t),     dS/dt = Asv V
 *   with V (Kv x M), S (Ks x M) stacked realizations (Eq. (rom_ode_tensor),
 *   Sec. 2.4).  The rank-2 system is M independent rank-1 systems
 *   (Eq. (rom_ode)) sharing the operators, so the oracle simply loops over
 *   columns: rank-2 column m *is* the rank-1 run m by construction.
 *
 *   Leapfrog, velocity first then stress (Sec. 3.1), read as
 *       V^{n+1} = V^n + dt (Avs S^n + g f(t_n))
 *       S^{n+1} = S^n + dt  Asv V^{n+1}
 *   with t_n = (n0 + n) dt, forcing sampled at the start of the step.
 *
 *   Reduced reference state (Eq. (rom_ode), Eq. (rom_ode_tensor)): the
 *   time-independent term Xhat_ref = Phi^T A X_ref, one column per
 *   realization, split like the state into Xv (Kv x M) and Xs (Ks x M),
 *   enters both halves of the step as one more constant forcing:
 *       V^{n+1} = V^n + dt (Avs S^n + g f(t_n) + Xv)
 *       S^{n+1} = S^n + dt (Asv V^{n+1} + Xs)
 *   NULL (the default, and the paper's seismic runs, Sec. 3.1) drops it.
 *
 *   Point-source forcing (Sec. 2.2, sparse case; Sec. 3.2 signal): the
 *   reduced forcing of realization m is g * f(t; T_m) with the Ricker wavelet
 *       f(t; T) = (1 - 2 u) exp(-u),  u = pi^2 (t - t0)^2 / T^2,  t0 = 1.5 T,
 *   or (wavelet = 1) the first derivative of a Gaussian defined below.
 *
 *   Receiver traces (seismograms from basis rows, Sec. 4.5.2):
 *       y = C V^{n+1}  after every step with (n + 1) mod r == 0.
 *
 * Parallelism: OpenMP over realizations only, so the arithmetic of each
 * column is independent of the thread count.
 *
 * Layout: every matrix is column-major.  Avs is Kv x Ks, Asv is Ks x Kv,
 * C is R x Kv, V is Kv x M, S is Ks x M.  Forcing tables are [n * M + m].
 * Trace records are [rec][m][j]: rec * R * M + m * R + j.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

static int orc_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Ricker wavelet, Sec. 3.2 (signal), with delay t0 = 1.5 T. */
static double ricker(double t, double T) {
    double tau = t - 1.5 * T;
    double u = ORC_PI * ORC_PI * tau * tau / (T * T);
    return (1.0 - 2.0 * u) * exp(-u);
}

/* d f / d T at fixed t (t0 = 1.5 T moves with T):
 *   df/du = (2u - 3) e^{-u},   du/dT = -pi^2 tau (3T + 2 tau) / T^3. */
static double ricker_dT(double t, double T) {
    double tau = t - 1.5 * T;
    double u = ORC_PI * ORC_PI * tau * tau / (T * T);
    double dfdu = (2.0 * u - 3.0) * exp(-u);
    double dudT = -ORC_PI * ORC_PI * tau * (3.0 * T + 2.0 * tau) / (T * T * T);
    return dfdu * dudT;
}

/* First derivative of a Gaussian, the paper's second source signal
 * (Sec. 3.2), read as the tau-derivative of the Ricker's Gaussian envelope
 * exp(-pi^2 tau^2 / T^2), delay t0 = 1.5 T, scaled to unit peak magnitude:
 *   f = -sqrt(2e) a exp(-a^2),   a = pi tau / T,   tau = t - 1.5 T
 * (extrema -1 at tau = +T / (pi sqrt 2) and +1 at tau = -T / (pi sqrt 2)). */
#define ORC_SQRT2E 2.33164398159712420
static double gauss1(double t, double T) {
    double a = ORC_PI * (t - 1.5 * T) / T;
    return -ORC_SQRT2E * a * exp(-a * a);
}

/* d f / d T at fixed t: df/da = -sqrt(2e) (1 - 2a^2) e^{-a^2},
 * da/dT = -pi t / T^2 (a = pi t / T - 1.5 pi). */
static double gauss1_dT(double t, double T) {
    double a = ORC_PI * (t - 1.5 * T) / T;
    double dfda = -ORC_SQRT2E * (1.0 - 2.0 * a * a) * exp(-a * a);
    double dadT = -ORC_PI * t / (T * T);
    return dfda * dadT;
}

/* Source signal of kind `wavelet`: 0 Ricker, 1 first derivative of a Gaussian. */
static double wavelet_f(int wavelet, double t, double T) {
    return wavelet == 1 ? gauss1(t, T) : ricker(t, T);
}
static double wavelet_dT(int wavelet, double t, double T) {
    return wavelet == 1 ? gauss1_dT(t, T) : ricker_dT(t, T);
}

void orc_wavelet(int wavelet, const double* t, const double* T, int n, double* f, double* dfdT) {
    for (int i = 0; i < n; ++i) {
        if (f) f[i] = wavelet_f(wavelet, t[i], T[i]);
        if (dfdT) dfdT[i] = wavelet_dT(wavelet, t[i], T[i]);
    }
}

void orc_ricker(const double* t, const double* T, int n, double* f, double* dfdT) {
    for (int i = 0; i < n; ++i) {
        if (f) f[i] = ricker(t[i], T[i]);
        if (dfdT) dfdT[i] = ricker_dT(t[i], T[i]);
    }
}

/* y = A x for a column-major rows x cols matrix A; y[i] accumulates over
 * k = 0 .. cols-1 in order (the k-outer loop keeps that order per i). */
static void matvec(const double* A, int rows, int cols, const double* x, double* y) {
    for (int i = 0; i < rows; ++i) y[i] = 0.0;
    for (int k = 0; k < cols; ++k) {
        const double xk = x[k];
        const double* a = A + (size_t)k * rows;
        for (int i = 0; i < rows; ++i) y[i] += a[i] * xk;
    }
}

/* y = A^T x for a column-major rows x cols matrix A (y has cols entries). */
static void matvec_t(const double* A, int rows, int cols, const double* x, double* y) {
    for (int k = 0; k < cols; ++k) {
        const double* a = A + (size_t)k * rows;
        double acc = 0.0;
        for (int i = 0; i < rows; ++i) acc += a[i] * x[i];
        y[k] = acc;
    }
}

static double forcing_value(const double* T, const double* ftab, int M, int m,
                            int n, long n0, double dt, int wavelet) {
    if (ftab) return ftab[(size_t)n * M + m];
    return wavelet_f(wavelet, (double)(n0 + n) * dt, T[m]);
}

/*
 * Forward leapfrog over nsteps steps, in place on V and S.
 * Exactly one of T (M periods) and ftab (nsteps x M forcing values) is used
 * (ftab wins when both are given; both NULL means zero forcing).
 * traces may be NULL; otherwise it receives floor(nsteps / r) records.
 * Returns 0, or -1 on a bad argument, -2 on allocation failure.
 */
int orc_forward(const double* Avs, const double* Asv, const double* g, const double* C,
                int Kv, int Ks, int R, double dt,
                double* V, double* S, const double* T, const double* ftab, int M,
                int nsteps, long n0, int r, double* traces, int nthreads, int wavelet,
                const double* Xv, const double* Xs) {
    if (Kv <= 0 || Ks <= 0 || M < 0 || nsteps < 0 || R < 0) return -1;
    if (traces && (r <= 0 || R <= 0 || !C)) return -1;
    orc_set_threads(nthreads);
    int err = 0;
#pragma omp parallel
    {
        double* tv = (double*)malloc(sizeof(double) * (size_t)Kv);
        double* ts = (double*)malloc(sizeof(double) * (size_t)Ks);
        double* ty = (double*)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1));
        if (!tv || !ts || !ty) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (int m = 0; m < M; ++m) {
                double* v = V + (size_t)m * Kv;
                double* s = S + (size_t)m * Ks;
                const double* xv = Xv ? Xv + (size_t)m * Kv : NULL;
                const double* xs = Xs ? Xs + (size_t)m * Ks : NULL;
                for (int n = 0; n < nsteps; ++n) {
                    const double f = (T || ftab) ? forcing_value(T, ftab, M, m, n, n0, dt, wavelet) : 0.0;
                    /* velocity first: v <- v + dt (Avs s + g f + xv) */
                    matvec(Avs, Kv, Ks, s, tv);
                    for (int i = 0; i < Kv; ++i) v[i] = v[i] + dt * (tv[i] + g[i] * f + (xv ? xv[i] : 0.0));
                    /* then stress with the new velocity: s <- s + dt (Asv v + xs) */
                    matvec(Asv, Ks, Kv, v, ts);
                    for (int i = 0; i < Ks; ++i) s[i] = s[i] + dt * (ts[i] + (xs ? xs[i] : 0.0));
                    if (traces && ((n + 1) % r) == 0) {
                        const int rec = (n + 1) / r - 1;
                        matvec(C, R, Kv, v, ty);
                        double* y = traces + ((size_t)rec * M + m) * R;
                        for (int j = 0; j < R; ++j) y[j] = ty[j];
                    }
                }
            }
        }
        free(tv);
        free(ts);
        free(ty);
    }
    return err;
}

/*
 * Inverse leapfrog: undoes orc_forward step by step (time reversibility,
 * Sec. 3.1).  Step n (taken from n = nsteps-1 down to 0) applies
 *   S^n = S^{n+1} - dt (Asv V^{n+1} + Xs),   V^n = V^{n+1} - dt (Avs S^n + g f(t_n) + Xv).
 */
int orc_inverse(const double* Avs, const double* Asv, const double* g,
                int Kv, int Ks, double dt, double* V, double* S,
                const double* T, const double* ftab, int M, int nsteps, long n0,
                int nthreads, int wavelet, const double* Xv, const double* Xs) {
    if (Kv <= 0 || Ks <= 0 || M < 0 || nsteps < 0) return -1;
    orc_set_threads(nthreads);
    int err = 0;
#pragma omp parallel
    {
        double* tv = (double*)malloc(sizeof(double) * (size_t)Kv);
        double* ts = (double*)malloc(sizeof(double) * (size_t)Ks);
        if (!tv || !ts) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (int m = 0; m < M; ++m) {
                double* v = V + (size_t)m * Kv;
                double* s = S + (size_t)m * Ks;
                const double* xv = Xv ? Xv + (size_t)m * Kv : NULL;
                const double* xs = Xs ? Xs + (size_t)m * Ks : NULL;
                for (int n = nsteps - 1; n >= 0; --n) {
                    const double f = (T || ftab) ? forcing_value(T, ftab, M, m, n, n0, dt, wavelet) : 0.0;
                    matvec(Asv, Ks, Kv, v, ts);
                    for (int i = 0; i < Ks; ++i) s[i] = s[i] - dt * (ts[i] + (xs ? xs[i] : 0.0));
                    matvec(Avs, Kv, Ks, s, tv);
                    for (int i = 0; i < Kv; ++i) v[i] = v[i] - dt * (tv[i] + g[i] * f + (xv ? xv[i] : 0.0));
                }
            }
        }
        free(tv);
        free(ts);
    }
    return err;
}

/*
 * Discrete leapfrog energy of the skew-coupled system (Avs = -Asv^T):
 *   E(V, S) = ||V||_F^2 + ||S||_F^2 - dt <S, Asv V>_F.
 * It is exactly invariant under the unforced step (derivation: with
 * V' = V - dt A^T S and S' = S + dt A V', <S', S' - dt A V'> = <S', S> and
 * the cross terms cancel).  Used only as a pin on orc_forward.
 */
double orc_energy(const double* Asv, int Kv, int Ks, double dt,
                  const double* V, const double* S, int M) {
    double e = 0.0;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)Ks);
    if (!tmp) return NAN;
    for (int m = 0; m < M; ++m) {
        const double* v = V + (size_t)m * Kv;
        const double* s = S + (size_t)m * Ks;
        double vv = 0.0, ss = 0.0, sav = 0.0;
        for (int i = 0; i < Kv; ++i) vv += v[i] * v[i];
        for (int i = 0; i < Ks; ++i) ss += s[i] * s[i];
        matvec(Asv, Ks, Kv, v, tmp);
        for (int i = 0; i < Ks; ++i) sav += s[i] * tmp[i];
        e += vv + ss - dt * sav;
    }
    free(tmp);
    return e;
}

/*
 * Spectral radius of the coupled operator L = [[0, Avs], [Asv, 0]].
 * L^2 = diag(Avs Asv, Asv Avs), so rho(L) = sqrt(rho(Avs Asv)).  Power
 * iteration runs on B = Avs Asv (Kv x Kv) from the start vector 1/sqrt(Kv)
 * (iterating on L itself would not converge: its dominant eigenvalues come
 * in pairs +-i sigma of equal modulus).  The estimate after each iteration
 * is the Rayleigh quotient |x^T B x| / x^T x.  Stops when two successive
 * estimates differ by less than tol (relative) or after max_iter iterations.
 * Returns the iterations used (negative on error); *rho gets rho(L).
 */
int orc_spectral_radius(const double* Avs, const double* Asv, int Kv, int Ks,
                        int max_iter, double tol, double* rho) {
    if (Kv <= 0 || Ks <= 0 || !rho) return -1;
    double* x = (double*)malloc(sizeof(double) * (size_t)Kv);
    double* y = (double*)malloc(sizeof(double) * (size_t)Kv);
    double* z = (double*)malloc(sizeof(double) * (size_t)Ks);
    if (!x || !y || !z) {
        free(x); free(y); free(z);
        return -2;
    }
    for (int i = 0; i < Kv; ++i) x[i] = 1.0 / sqrt((double)Kv);
    double lam = 0.0, prev = -1.0;
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
        matvec(Asv, Ks, Kv, x, z);   /* z = Asv x   */
        matvec(Avs, Kv, Ks, z, y);   /* y = Avs z   */
        double xy = 0.0, xx = 0.0, yy = 0.0;
        for (int i = 0; i < Kv; ++i) { xy += x[i] * y[i]; xx += x[i] * x[i]; yy += y[i] * y[i]; }
        lam = fabs(xy) / xx;
        if (yy == 0.0) { lam = 0.0; break; }
        const double ny = sqrt(yy);
        for (int i = 0; i < Kv; ++i) x[i] = y[i] / ny;
        if (prev >= 0.0 && fabs(lam - prev) <= tol * lam) break;
        prev = lam;
    }
    *rho = sqrt(lam);
    free(x); free(y); free(z);
    return it > max_iter ? max_iter : it;
}

/*
 * Adjoint of the receiver-trace misfit
 *     L = sum_{n=1..N} sum_m || C V_m^n - ystar_m^n ||^2
 * (ystar records are [n-1][m][j], one per step) with respect to the initial
 * state (V0, S0) and the Ricker periods T_m.  The paper gives no adjoint; this
 * is the reverse of the leapfrog above, derived step by step:
 *
 *   lamV = 2 C^T (C V^N - y^N),  lamS = 0
 *   for n = N-1 .. 0:
 *       aS   = lamS                          (adjoint of S^{n+1})
 *       aV   = lamV + dt Asv^T aS            (total adjoint of V^{n+1})
 *       dL/df_n = dt g^T aV
 *       lamS = aS + dt Avs^T aV              (adjoint of S^n)
 *       lamV = aV + [n >= 1] 2 C^T (C V^n - y^n)   (adjoint of V^n)
 *   dL/dV0 = lamV, dL/dS0 = lamS,  dL/dT_m = sum_n dL/df_n df/dT(t_n; T_m).
 *
 * Per column it stores the N residuals C V^n - y^n (N x R doubles).
 * The reference-state term Xv, Xs (may be NULL) shifts the forward sweep
 * only: it depends on neither the state nor T, so the reverse recurrence
 * above is unchanged.
 * gV0, gS0, gT may be NULL.  *loss receives L.  Returns 0 or negative.
 */
int orc_adjoint(const double* Avs, const double* Asv, const double* g, const double* C,
                int Kv, int Ks, int R, double dt,
                const double* V0, const double* S0, const double* T, int M,
                int nsteps, long n0, const double* ystar,
                double* gV0, double* gS0, double* gT, double* loss, int nthreads,
                int wavelet, const double* Xv, const double* Xs) {
    if (Kv <= 0 || Ks <= 0 || R <= 0 || M < 0 || nsteps < 0 || !C || !ystar || !T) return -1;
    orc_set_threads(nthreads);
    int err = 0;
    double total = 0.0;
#pragma omp parallel reduction(+ : total)
    {
        double* v = (double*)malloc(sizeof(double) * (size_t)Kv);
        double* s = (double*)malloc(sizeof(double) * (size_t)Ks);
        double* tv = (double*)malloc(sizeof(double) * (size_t)Kv);
        double* ts = (double*)malloc(sizeof(double) * (size_t)Ks);
        double* ty = (double*)malloc(sizeof(double) * (size_t)R);
        double* res = (double*)malloc(sizeof(double) * (size_t)R * (size_t)(nsteps > 0 ? nsteps : 1));
        double* lv = (double*)malloc(sizeof(double) * (size_t)Kv);
        double* ls = (double*)malloc(sizeof(double) * (size_t)Ks);
        double* av = (double*)malloc(sizeof(double) * (size_t)Kv);
        double* ctr = (double*)malloc(sizeof(double) * (size_t)Kv);
        if (!v || !s || !tv || !ts || !ty || !res || !lv || !ls || !av || !ctr) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (int m = 0; m < M; ++m) {
                /* forward sweep, keeping the residuals r^n = C V^n - y^n */
                memcpy(v, V0 + (size_t)m * Kv, sizeof(double) * (size_t)Kv);
                memcpy(s, S0 + (size_t)m * Ks, sizeof(double) * (size_t)Ks);
                double lm = 0.0;
                const double* xv = Xv ? Xv + (size_t)m * Kv : NULL;
                const double* xs = Xs ? Xs + (size_t)m * Ks : NULL;
                for (int n = 0; n < nsteps; ++n) {
                    const double f = wavelet_f(wavelet, (double)(n0 + n) * dt, T[m]);
                    matvec(Avs, Kv, Ks, s, tv);
                    for (int i = 0; i < Kv; ++i) v[i] = v[i] + dt * (tv[i] + g[i] * f + (xv ? xv[i] : 0.0));
                    matvec(Asv, Ks, Kv, v, ts);
                    for (int i = 0; i < Ks; ++i) s[i] = s[i] + dt * (ts[i] + (xs ? xs[i] : 0.0));
                    matvec(C, R, Kv, v, ty);
                    const double* yst = ystar + ((size_t)n * M + m) * R;
                    double* rn = res + (size_t)n * R;
                    for (int j = 0; j < R; ++j) {
                        rn[j] = ty[j] - yst[j];
                        lm += rn[j] * rn[j];
                    }
                }
                total += lm;
                /* reverse sweep */
                for (int i = 0; i < Ks; ++i) ls[i] = 0.0;
                if (nsteps > 0) {
                    matvec_t(C, R, Kv, res + (size_t)(nsteps - 1) * R, ctr);
                    for (int i = 0; i < Kv; ++i) lv[i] = 2.0 * ctr[i];
                } else {
                    for (int i = 0; i < Kv; ++i) lv[i] = 0.0;
                }
                double gt = 0.0;
                for (int n = nsteps - 1; n >= 0; --n) {
                    /* aS = lamS (kept in ls); aV = lamV + dt Asv^T aS */
                    matvec_t(Asv, Ks, Kv, ls, tv);
                    for (int i = 0; i < Kv; ++i) av[i] = lv[i] + dt * tv[i];
                    double gav = 0.0;
                    for (int i = 0; i < Kv; ++i) gav += g[i] * av[i];
                    gt += dt * gav * wavelet_dT(wavelet, (double)(n0 + n) * dt, T[m]);
                    /* lamS = aS + dt Avs^T aV */
                    matvec_t(Avs, Kv, Ks, av, ts);
                    for (int i = 0; i < Ks; ++i) ls[i] = ls[i] + dt * ts[i];
                    /* lamV = aV + [n >= 1] 2 C^T r^n */
                    if (n >= 1) {
                        matvec_t(C, R, Kv, res + (size_t)(n - 1) * R, ctr);
                        for (int i = 0; i < Kv; ++i) lv[i] = av[i] + 2.0 * ctr[i];
                    } else {
                        for (int i = 0; i < Kv; ++i) lv[i] = av[i];
                    }
                }
                if (gV0) memcpy(gV0 + (size_t)m * Kv, lv, sizeof(double) * (size_t)Kv);
                if (gS0) memcpy(gS0 + (size_t)m * Ks, ls, sizeof(double) * (size_t)Ks);
                if (gT) gT[m] = gt;
            }
        }
        free(v); free(s); free(tv); free(ts); free(ty); free(res);
        free(lv); free(ls); free(av); free(ctr);
    }
    if (loss) *loss = total;
    return err;
}
