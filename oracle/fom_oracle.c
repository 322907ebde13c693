/*
 * FP64 reference ("oracle") for the rank-2 full-order model (FOM) of the
 * paper's test case: axisymmetric elastic shear waves in velocity-stress
 * form, Eq. (fom_asym), Sec. 3, on the circular sector r_cmb <= r <= r_earth,
 * 0 <= theta <= pi:
 *     rho v_t      = (sigma_rp)_r + (1/r)(sigma_tp)_theta
 *                    + (1/r)(3 sigma_rp + 2 cot(theta) sigma_tp) + f
 *     (sigma_rp)_t = mu (v_r - v / r)
 *     (sigma_tp)_t = mu ((1/r) v_theta - (cot(theta) / r) v),   mu = rho vs^2.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or constant with the CUDA library.
 *
 * Discretization (the paper gives a second-order staggered grid and refers
 * to the stencil only by citation; this is the reading taken).  The
 * right-hand sides are written in flux form,
 *     (sigma_rp)_r + 3 sigma_rp / r = r^-3 (r^3 sigma_rp)_r
 *     (1/r)(sigma_tp)_theta + 2 cot sigma_tp / r = (r sin^2)^-1 (sin^2 sigma_tp)_theta
 *     v_r - v / r = r (v / r)_r,     (1/r)(v_theta - cot v) = (sin / r)(v / sin)_theta,
 * with Nr radial and Nt polar intervals, dr = (r_earth - r_cmb) / Nr,
 * dth = pi / Nt, r_a = r_cmb + a dr, theta_b = b dth (a, b may be halves):
 *     v        at (r_{i+1/2}, theta_j),       i in [0, Nr),  j in [1, Nt)
 *     sigma_rp at (r_i, theta_j),             i in [1, Nr),  j in [1, Nt)
 *     sigma_tp at (r_{i+1/2}, theta_{j+1/2}), i in [0, Nr),  j in [1, Nt - 1)
 * Boundary conditions (Sec. 3): v = 0 on the axis (j = 0, Nt), sigma_rp = 0
 * there and on the free surfaces r_cmb, r_earth (i = 0, Nr).  At the two
 * sigma_tp points next to the axis (j + 1/2 = 1/2, Nt - 1/2) the stencil
 * needs v / sin(theta) ON the axis, a 0/0 whose limit is finite for a smooth
 * axisymmetric field; it is extrapolated with zero slope from the first
 * interior point, which makes sigma_tp there identically zero (the field's
 * sigma_tp vanishes towards the axis).  Points that are identically zero
 * carry no unknowns and enter the stencils as zeros.  Every row has at most
 * four (velocity) or two (stress) non-zeros, as the paper states.  Flux
 * form makes the semi-discrete operator skew-adjoint under the weights
 * rho r^2 sin(theta) (velocity) and r^2 sin(theta) / mu (stresses), each
 * at its own grid point, so the leapfrog conserves a discrete energy.
 *
 * Unknown numbering (one realization):
 *     v[i (Nt - 1) + (j - 1)],  s1[(i - 1) (Nt - 1) + (j - 1)],  s2[i (Nt - 2) + (j - 1)].
 * Leapfrog, velocity first (Sec. 3.1):
 *     v^{n+1}  = v^n + (dt / rho) (A s^n) + (dt / rho) f(t_n) e_src
 *     s^{n+1}  = s^n + dt mu (B v^{n+1})
 * Forcing: a point source on velocity unknown `src`, the signal of the
 * period T_m (0 Ricker, 1 first derivative of a Gaussian, delay 1.5 T) or
 * a table ftab[n * M + m].  Receivers: velocity unknowns recv[k], recorded
 * after every step with (n + 1) mod r == 0 into traces[(rec * M + m) * nrecv + k].
 * States are column-major per realization: V (nv x M), S1 (n1 x M),
 * S2 (n2 x M).  OpenMP over realizations only.
 */
#include <math.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* The source signals, as in rom_oracle.c (kept private to this file). */
static double fom_signal(int wavelet, double t, double T) {
    const double pi = 3.14159265358979323846;
    const double tau = t - 1.5 * T;
    if (wavelet == 1) {
        const double a = pi * tau / T;
        return -sqrt(2.0 * exp(1.0)) * a * exp(-a * a);
    }
    const double u = pi * pi * tau * tau / (T * T);
    return (1.0 - 2.0 * u) * exp(-u);
}

void orc_fom_dims(int Nr, int Nt, int* nv, int* n1, int* n2) {
    *nv = Nr * (Nt - 1);
    *n1 = (Nr - 1) * (Nt - 1);
    *n2 = Nr * (Nt - 2);
}

/* One realization, one step; v, s1, s2 updated in place. */
static void fom_step(int Nr, int Nt, double rc, double dr, double dth, double rho, double mu,
                     double dt, double* v, double* s1, double* s2, int src, double f) {
    /* velocity first, with the old stresses */
    for (int i = 0; i < Nr; ++i) {
        const double rm = rc + i * dr, rp = rc + (i + 1) * dr, rh = rc + (i + 0.5) * dr;
        for (int j = 1; j < Nt; ++j) {
            const double th = j * dth, thp = (j + 0.5) * dth, thm = (j - 0.5) * dth;
            const double s1p = (i + 1 < Nr) ? s1[i * (Nt - 1) + (j - 1)] : 0.0;       /* (i+1, j) */
            const double s1m = (i >= 1) ? s1[(i - 1) * (Nt - 1) + (j - 1)] : 0.0;      /* (i, j)   */
            const double s2p = (j <= Nt - 2) ? s2[i * (Nt - 2) + (j - 1)] : 0.0;        /* j + 1/2  */
            const double s2m = (j >= 2) ? s2[i * (Nt - 2) + (j - 2)] : 0.0;             /* j - 1/2  */
            const double radial = (rp * rp * rp * s1p - rm * rm * rm * s1m) / (rh * rh * rh * dr);
            const double polar = (sin(thp) * sin(thp) * s2p - sin(thm) * sin(thm) * s2m) /
                                 (rh * sin(th) * sin(th) * dth);
            double* vp = &v[i * (Nt - 1) + (j - 1)];
            *vp = *vp + (dt / rho) * (radial + polar);
        }
    }
    if (src >= 0) v[src] = v[src] + (dt / rho) * f;
    /* then the stresses, with the new velocity */
    for (int i = 1; i < Nr; ++i) {
        const double ri = rc + i * dr, rh = rc + (i + 0.5) * dr, rl = rc + (i - 0.5) * dr;
        for (int j = 1; j < Nt; ++j) {
            const double vu = v[i * (Nt - 1) + (j - 1)];        /* (i + 1/2, j) */
            const double vd = v[(i - 1) * (Nt - 1) + (j - 1)];  /* (i - 1/2, j) */
            double* sp = &s1[(i - 1) * (Nt - 1) + (j - 1)];
            *sp = *sp + dt * mu * ri * (vu / rh - vd / rl) / dr;
        }
    }
    for (int i = 0; i < Nr; ++i) {
        const double rh = rc + (i + 0.5) * dr;
        for (int j = 1; j < Nt - 1; ++j) {
            const double thh = (j + 0.5) * dth;
            const double vr = v[i * (Nt - 1) + j] / sin((j + 1) * dth);        /* (i + 1/2, j + 1) */
            const double vl = v[i * (Nt - 1) + (j - 1)] / sin(j * dth);        /* (i + 1/2, j)     */
            double* sp = &s2[i * (Nt - 2) + (j - 1)];
            *sp = *sp + dt * mu * (sin(thh) / rh) * (vr - vl) / dth;
        }
    }
}

int orc_fom_forward(int Nr, int Nt, double r_cmb, double r_earth, double rho, double vs,
                    double dt, double* V, double* S1, double* S2, int M, int nsteps, long n0,
                    int src, const double* T, const double* ftab, int wavelet, int nrecv,
                    const int* recv, int r, double* traces, int nthreads) {
    if (Nr < 2 || Nt < 3 || M < 0 || nsteps < 0 || !(r_earth > r_cmb) || !(r_cmb > 0.0)) return -1;
    if (traces && (r <= 0 || nrecv <= 0 || !recv)) return -1;
    int nv, n1, n2;
    orc_fom_dims(Nr, Nt, &nv, &n1, &n2);
    if (src >= nv) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const double dr = (r_earth - r_cmb) / Nr, dth = 3.14159265358979323846 / Nt;
    const double mu = rho * vs * vs;
#pragma omp parallel for schedule(static)
    for (int m = 0; m < M; ++m) {
        double* v = V + (size_t)m * nv;
        double* s1 = S1 + (size_t)m * n1;
        double* s2 = S2 + (size_t)m * n2;
        for (int n = 0; n < nsteps; ++n) {
            double f = 0.0;
            if (ftab) f = ftab[(size_t)n * M + m];
            else if (T) f = fom_signal(wavelet, (double)(n0 + n) * dt, T[m]);
            fom_step(Nr, Nt, r_cmb, dr, dth, rho, mu, dt, v, s1, s2, (T || ftab) ? src : -1, f);
            if (traces && ((n + 1) % r) == 0) {
                const int rec = (n + 1) / r - 1;
                for (int k = 0; k < nrecv; ++k)
                    traces[((size_t)rec * M + m) * nrecv + k] = v[recv[k]];
            }
        }
    }
    return 0;
}
