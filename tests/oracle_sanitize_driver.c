/*
 * Test driver for the FP64 oracle (oracle/eik_oracle.c) under AddressSanitizer and
 * UndefinedBehaviorSanitizer (tests/test_oracle_sanitized.py builds and runs it).
 *
 * Every entry point of the oracle runs on small grids with the edge cases of the
 * method: single nodes and lines, 2D and 3D shapes that are not multiples of any
 * tile, impassable nodes (F = 0), duplicated sources, no sources, a source out of
 * range (an argument error), unequal spacings.  The grids come from a fixed linear
 * congruential generator (no arithmetic of the method here).  Beyond "no memory
 * error, no undefined behaviour", it checks that fast marching and Gauss-Seidel
 * sweeping agree, and that Algorithm 2 and the FIM agree with them.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int64_t eko_fmm(int64_t nx, int64_t ny, int64_t nz, double h, const double *F, int64_t n_src,
                const int64_t *src_idx, const double *src_val, double *phi, int64_t *order_out);
int64_t eko_fmm_aniso(int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz, const double *F,
                      int64_t n_src, const int64_t *src_idx, const double *src_val, double *phi, int64_t *order_out);
int64_t eko_gs(int64_t nx, int64_t ny, int64_t nz, double h, const double *F, int64_t n_src,
               const int64_t *src_idx, const double *src_val, double *phi, int64_t max_rounds);
int64_t eko_gs_aniso(int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz, const double *F,
                     int64_t n_src, const int64_t *src_idx, const double *src_val, double *phi, int64_t max_rounds);
int eko_ifim(int64_t nx, int64_t ny, int64_t nz, double h, const double *F, int64_t n_src, const int64_t *src_idx,
             const double *src_val, double *phi, int skip_remedy, int64_t max_iters, int64_t *stats);
int eko_fim(int64_t nx, int64_t ny, int64_t nz, double h, const double *F, int64_t n_src, const int64_t *src_idx,
            const double *src_val, double *phi, int64_t max_iters, int64_t *stats);
double eko_residual(int64_t nx, int64_t ny, int64_t nz, double h, const double *F, int64_t n_src,
                    const int64_t *src_idx, const double *phi, double *res);
double eko_residual_aniso(int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz, const double *F,
                          int64_t n_src, const int64_t *src_idx, const double *phi, double *res);
int eko_backtrace(int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz, const double *phi,
                  int64_t n_paths, const int64_t *start_idx, int64_t max_len, int64_t *path_out, int64_t *len_out);
int eko_adjoint(int64_t nx, int64_t ny, int64_t nz, double h, const double *F, int64_t n_src,
                const int64_t *src_idx, const double *phi, const double *r, double *g, double *lambda_out);
double eko_local_solve(double ax, double ay, double az, double tau);
double eko_local_solve_aniso(double ax, double ay, double az, double hx, double hy, double hz, double F);

static uint64_t lcg_state = 12345u;
static double uniform01(void) {
    lcg_state = lcg_state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(lcg_state >> 11) * (1.0 / 9007199254740992.0);
}

static int failures = 0;
#define CHECK(cond, ...)                                    \
    do {                                                    \
        if (!(cond)) {                                      \
            fprintf(stderr, __VA_ARGS__);                   \
            fprintf(stderr, "\n");                          \
            ++failures;                                     \
        }                                                   \
    } while (0)

static double max_abs_diff(const double *a, const double *b, int64_t n) {
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (isinf(a[i]) || isinf(b[i])) {
            if (isinf(a[i]) != isinf(b[i])) return INFINITY;
            continue;
        }
        const double d = fabs(a[i] - b[i]);
        if (d > m) m = d;
    }
    return m;
}

static void one_grid(int64_t nx, int64_t ny, int64_t nz, double p_barrier, int n_src) {
    const int64_t N = nx * ny * nz;
    double *F = malloc(sizeof(double) * N), *phi = malloc(sizeof(double) * N), *ref = malloc(sizeof(double) * N);
    double *res = malloc(sizeof(double) * N), *r = malloc(sizeof(double) * N), *g = malloc(sizeof(double) * N);
    double *lam = malloc(sizeof(double) * N);
    int64_t *order = malloc(sizeof(int64_t) * N);
    int64_t src[8];
    double val[8];
    for (int64_t i = 0; i < N; ++i) F[i] = uniform01() < p_barrier ? 0.0 : 0.2 + 3.0 * uniform01();
    for (int s = 0; s < n_src; ++s) {
        src[s] = (int64_t)(uniform01() * (double)N) % N;
        val[s] = 0.0;
    }
    if (n_src >= 3) src[2] = src[1];                   /* a duplicated source index */
    const double h = 0.1;
    const int64_t na = eko_fmm(nx, ny, nz, h, F, n_src, src, val, ref, order);
    CHECK(na >= 0 && na <= N, "fmm returned %lld", (long long)na);
    const int64_t rounds = eko_gs(nx, ny, nz, h, F, n_src, src, val, phi, 100000);
    CHECK(rounds >= 0, "gs returned %lld", (long long)rounds);
    CHECK(max_abs_diff(ref, phi, N) <= 1e-12, "gs differs from fmm on %lldx%lldx%lld", (long long)nx,
          (long long)ny, (long long)nz);
    int64_t st[4] = {0, 0, 0, 0};
    CHECK(eko_ifim(nx, ny, nz, h, F, n_src, src, val, phi, 0, 1000000, st) == 0, "ifim failed");
    CHECK(max_abs_diff(ref, phi, N) <= 1e-12, "Algorithm 2 differs from fmm");
    int64_t st2[2] = {0, 0};
    CHECK(eko_fim(nx, ny, nz, h, F, n_src, src, val, phi, 1000000, st2) == 0, "fim failed");
    CHECK(max_abs_diff(ref, phi, N) <= 1e-12, "FIM differs from fmm");
    const double worst = eko_residual(nx, ny, nz, h, F, n_src, src, ref, res);
    CHECK(worst < 1e-10, "residual %g on the fmm solution", worst);
    for (int64_t i = 0; i < N; ++i) r[i] = (isfinite(ref[i]) && uniform01() < 0.3) ? uniform01() - 0.5 : 0.0;
    for (int64_t i = 0; i < N; ++i) g[i] = 0.0;
    CHECK(eko_adjoint(nx, ny, nz, h, F, n_src, src, ref, r, g, lam) == 0, "adjoint failed");
    int64_t starts[4];
    for (int q = 0; q < 4; ++q) starts[q] = (int64_t)(uniform01() * (double)N) % N;
    int64_t *paths = malloc(sizeof(int64_t) * 4 * (N + 1)), lens[4];
    CHECK(eko_backtrace(nx, ny, nz, h, h, h, ref, 4, starts, N + 1, paths, lens) == 0, "backtrace failed");
    for (int q = 0; q < 4; ++q) CHECK(lens[q] >= 0 && lens[q] <= N + 1, "path length %lld", (long long)lens[q]);
    /* unequal spacings */
    const int64_t nb = eko_fmm_aniso(nx, ny, nz, h, 1.7 * h, 0.6 * h, F, n_src, src, val, ref, NULL);
    CHECK(nb >= 0, "fmm_aniso returned %lld", (long long)nb);
    CHECK(eko_gs_aniso(nx, ny, nz, h, 1.7 * h, 0.6 * h, F, n_src, src, val, phi, 100000) >= 0, "gs_aniso failed");
    CHECK(max_abs_diff(ref, phi, N) <= 1e-12, "gs_aniso differs from fmm_aniso");
    (void)eko_residual_aniso(nx, ny, nz, h, 1.7 * h, 0.6 * h, F, n_src, src, ref, res);
    free(F); free(phi); free(ref); free(res); free(r); free(g); free(lam); free(order); free(paths);
}

int main(void) {
    static const int64_t dims[][3] = {{1, 1, 1}, {1, 1, 9}, {17, 1, 1}, {1, 13, 1}, {9, 9, 1},
                                      {3, 5, 7}, {8, 8, 8}, {13, 7, 5}, {16, 16, 17}, {21, 4, 3}};
    for (size_t k = 0; k < sizeof(dims) / sizeof(dims[0]); ++k)
        for (int variant = 0; variant < 3; ++variant)
            one_grid(dims[k][0], dims[k][1], dims[k][2], variant == 2 ? 0.1 : 0.0, variant == 0 ? 1 : 4);
    /* no sources: everything unreachable */
    double F[27], phi[27];
    for (int i = 0; i < 27; ++i) F[i] = 1.0;
    CHECK(eko_fmm(3, 3, 3, 0.5, F, 0, NULL, NULL, phi, NULL) >= 0, "fmm without sources");
    for (int i = 0; i < 27; ++i) CHECK(isinf(phi[i]), "unreachable node %d is finite", i);
    /* a source out of range is an argument error, not a memory error */
    int64_t bad = 27;
    double zero = 0.0;
    CHECK(eko_fmm(3, 3, 3, 0.5, F, 1, &bad, &zero, phi, NULL) < 0, "out-of-range source accepted");
    /* local solves at the cascade's thresholds and with infinities */
    CHECK(eko_local_solve(0.0, 1.0, INFINITY, 1.0) == 1.0, "one-sided at the threshold");
    CHECK(isinf(eko_local_solve(INFINITY, INFINITY, INFINITY, 1.0)), "no finite neighbour");
    CHECK(eko_local_solve_aniso(0.0, INFINITY, INFINITY, 1.0, 2.0, 3.0, 1.0) == 1.0, "aniso one-sided");
    if (failures) {
        fprintf(stderr, "%d check(s) failed\n", failures);
        return 1;
    }
    printf("oracle sanitize driver ok\n");
    return 0;
}
