"""A plain C program drives the library on the GPU through the C ABI alone
(no Python, no PyTorch): it builds a small skew-coupled ROM with its own
generator, reads the spectral radius from rom_create, integrates M
realizations with host buffers (the library stages them) for both FP32 and
FP64, and compares states and traces with the FP64 oracle's C library
(oracle/rom_oracle.c, linked as test infrastructure)."""
import os
import shutil
import subprocess

import pytest

import oracle

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include "rom.h"

int orc_forward(const double* Avs, const double* Asv, const double* g, const double* C,
                int Kv, int Ks, int R, double dt, double* V, double* S, const double* T,
                const double* ftab, int M, int nsteps, long n0, int r, double* traces,
                int nthreads, int wavelet, const double* Xv, const double* Xs);

static unsigned long long state = 88172645463325252ULL;
static double unif(void) {  /* xorshift64, uniform in [-1, 1) */
    state ^= state << 13; state ^= state >> 7; state ^= state << 17;
    return (double)(state >> 11) / 9007199254740992.0 * 2.0 - 1.0;
}
static double rel(const double* a, const double* b, size_t n) {
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < n; ++i) { num += (a[i] - b[i]) * (a[i] - b[i]); den += b[i] * b[i]; }
    return sqrt(num / (den > 0.0 ? den : 1e-300));
}

int main(void) {
    const int K = 96, M = 12, R = 5, N = 300, r = 10;
    const size_t KK = (size_t)K * K;
    double *Avs = malloc(KK * 8), *Asv = malloc(KK * 8), *g = malloc(K * 8), *C = malloc((size_t)R * K * 8);
    double *T = malloc(M * 8);
    for (int i = 0; i < K; ++i)          /* Asv column-major, Avs = -Asv^T */
        for (int j = 0; j < K; ++j) Asv[i + (size_t)j * K] = unif() / sqrt((double)K);
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) Avs[i + (size_t)j * K] = -Asv[j + (size_t)i * K];
    double gn = 0.0;
    for (int i = 0; i < K; ++i) { g[i] = unif(); gn += g[i] * g[i]; }
    for (int i = 0; i < K; ++i) g[i] /= sqrt(gn);
    for (size_t i = 0; i < (size_t)R * K; ++i) C[i] = unif() / sqrt((double)K);
    /* the spectral radius comes back even when dt is refused */
    rom_t h = NULL;
    double rho = 0.0;
    rom_status st = rom_create(Avs, Asv, g, C, K, K, R, 10.0, ROM_IN_F64, &h, &rho);
    if (st != ROM_E_UNSTABLE || h != NULL || !(rho > 0.0)) { printf("create(dt=10): %s\n", rom_status_string(st)); return 2; }
    const double dt = (double)(float)(0.5 / rho);
    for (int m = 0; m < M; ++m) T[m] = (double)(float)((40.0 + 2.0 * m) * dt);
    /* the oracle: FP64, one realization at a time */
    double *Vo = calloc((size_t)K * M, 8), *So = calloc((size_t)K * M, 8);
    double *tro = calloc((size_t)(N / r) * M * R, 8);
    if (orc_forward(Avs, Asv, g, C, K, K, R, dt, Vo, So, T, NULL, M, N, 0, r, tro, 0, 0, NULL, NULL) != 0) return 3;
    int fails = 0;
    for (int pass = 0; pass < 2; ++pass) {
        const int in = pass == 0 ? ROM_IN_F32 : ROM_IN_F64;
        const int prec = pass == 0 ? ROM_FP32 : ROM_FP64;
        const size_t es = pass == 0 ? 4 : 8;
        /* operators handed over in the run's element type */
        void *A1 = malloc(KK * es), *A2 = malloc(KK * es), *gg = malloc(K * es), *CC = malloc((size_t)R * K * es);
        void *V = calloc((size_t)K * M, es), *S = calloc((size_t)K * M, es), *TT = malloc(M * es);
        void *tr = calloc((size_t)(N / r) * M * R, es);
        for (size_t i = 0; i < KK; ++i) {
            if (es == 4) { ((float*)A1)[i] = (float)Avs[i]; ((float*)A2)[i] = (float)Asv[i]; }
            else { ((double*)A1)[i] = Avs[i]; ((double*)A2)[i] = Asv[i]; }
        }
        for (int i = 0; i < K; ++i) { if (es == 4) ((float*)gg)[i] = (float)g[i]; else ((double*)gg)[i] = g[i]; }
        for (size_t i = 0; i < (size_t)R * K; ++i) { if (es == 4) ((float*)CC)[i] = (float)C[i]; else ((double*)CC)[i] = C[i]; }
        for (int m = 0; m < M; ++m) { if (es == 4) ((float*)TT)[m] = (float)T[m]; else ((double*)TT)[m] = T[m]; }
        st = rom_create(A1, A2, gg, CC, K, K, R, dt, in, &h, NULL);
        if (st != ROM_OK) { printf("create: %s %s\n", rom_status_string(st), rom_last_error()); return 4; }
        st = rom_run_rank2(h, V, S, TT, M, N, 0, r, tr, prec, NULL);
        if (st != ROM_OK) { printf("run: %s %s\n", rom_status_string(st), rom_last_error()); return 5; }
        rom_status dev = ROM_OK;
        if (rom_sync_status(h, &dev) != ROM_OK || dev != ROM_OK) return 6;
        double *Vd = malloc((size_t)K * M * 8), *Sd = malloc((size_t)K * M * 8), *trd = malloc((size_t)(N / r) * M * R * 8);
        for (size_t i = 0; i < (size_t)K * M; ++i) {
            Vd[i] = es == 4 ? ((float*)V)[i] : ((double*)V)[i];
            Sd[i] = es == 4 ? ((float*)S)[i] : ((double*)S)[i];
        }
        for (size_t i = 0; i < (size_t)(N / r) * M * R; ++i) trd[i] = es == 4 ? ((float*)tr)[i] : ((double*)tr)[i];
        /* the library's traces are R x M per record; the oracle's too (column m, receiver k) */
        const double ev = rel(Vd, Vo, (size_t)K * M), es_ = rel(Sd, So, (size_t)K * M);
        const double et = rel(trd, tro, (size_t)(N / r) * M * R);
        const double tol = pass == 0 ? 1e-4 : 1e-12;
        printf("%s rel V %.3e S %.3e traces %.3e\n", pass == 0 ? "fp32" : "fp64", ev, es_, et);
        if (!(ev <= tol && es_ <= tol && et <= tol)) fails |= 1 << pass;
        rom_destroy(h);
        free(A1); free(A2); free(gg); free(CC); free(V); free(S); free(TT); free(tr); free(Vd); free(Sd); free(trd);
    }
    printf("%d\n", fails);
    return fails;
}
"""


@pytest.fixture(scope="module")
def libpath():
    from paper_2009_11742_gb300 import build
    return build.build()


def test_c_program_runs_rank2_against_the_oracle(tmp_path, libpath):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    orc = oracle.build()
    src = tmp_path / "drive.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "drive"
    libdir, orcdir = os.path.dirname(libpath), os.path.dirname(orc)
    r = subprocess.run([cc, "-std=c99", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-lrom", "-L", orcdir, "-lorc", "-lm",
                        f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{orcdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, (r.stdout, r.stderr)
    assert r.stdout.strip().splitlines()[-1] == "0"
