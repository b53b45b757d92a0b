/*
 * eik_oracle.c -- plain, slow FP64 CPU oracle for the first-order Godunov
 * upwind discretisation of ||grad phi|| = 1/F (eq. 4 in 2D, eq. 6 in 3D).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing here is part of the product path: only
 * the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * load this library.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * Conventions (all functions):
 *   - grid is (nz, ny, nx), row-major, x fastest; flat index = (k*ny + j)*nx + i;
 *     a 2D grid is nz = 1 (the z neighbours are then out of grid = +inf).
 *   - isotropic spacing h (Alg 1.1 / Alg 1.3 assume a square mesh).
 *   - F > 0 is a speed (eq. 3, F > 0 assumed in Sec. 1); F == 0 marks an
 *     impassable node (eq. 8: barrier), which keeps phi = +inf unless it is a
 *     source.  tau = h / F.
 *   - out-of-grid neighbours count as +inf.
 *   - sources are (flat index, value) pairs held fixed (Dirichlet, Alg 2
 *     Step 1).  A duplicated source index keeps the smaller value.
 *
 * Functions and the passages they follow:
 *   eko_local_solve  exact root of eq. (6) (cascade of one-, two-, three-sided
 *                    roots; the thresholds are the validity conditions of the
 *                    "^+" equation, not the ones printed in Alg 1.1 / 1.3)
 *   eko_fmm          fast marching (Sec. 2.1), the plain definition of the
 *                    discrete solution; heap ordered by (value, flat index)
 *   eko_gs           Gauss-Seidel with 2^d alternating sweep orders (Sec. 2.2)
 *                    to an exact fixed point; tiny grids only
 *   eko_ifim         Algorithm 2 (Steps 1-3) point by point, with the
 *                    two-phase parallel semantics of Sec. 3.2.1
 *   eko_fim          the fast iterative method of Sec. 2.3 (with the
 *                    neighbour convergence check), point by point, same
 *                    two-phase semantics
 *   eko_local_solve_aniso, eko_fmm_aniso, eko_gs_aniso, eko_residual_aniso
 *                    the same with unequal spacings dx, dy, dz (eq. 5/6 as
 *                    written with them; Alg 1.2 with the validity thresholds)
 *   eko_residual     max relative residual of eq. (6) over non-source nodes
 *   eko_backtrace    shortest-path back-trace by steepest descent on the phi
 *                    map over the 26 (8 in 2D) neighbours (Example 4)
 *   eko_adjoint      transposed upwind-linearised system solved by back
 *                    substitution in increasing-phi order (adjoint-state
 *                    traveltime method, Leung & Qian 2006); not in the paper
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EKO_INF (1.0 / 0.0)

typedef struct {
    int64_t nx, ny, nz;
} dims_t;

static inline int64_t flat(const dims_t *d, int64_t i, int64_t j, int64_t k) {
    return (k * d->ny + j) * d->nx + i;
}

static inline void unflat(const dims_t *d, int64_t p, int64_t *i, int64_t *j, int64_t *k) {
    *i = p % d->nx;
    *j = (p / d->nx) % d->ny;
    *k = p / (d->nx * d->ny);
}

/* value of a neighbour, +inf outside the grid */
static inline double nbval(const dims_t *d, const double *phi, int64_t i, int64_t j, int64_t k) {
    if (i < 0 || j < 0 || k < 0 || i >= d->nx || j >= d->ny || k >= d->nz) return EKO_INF;
    return phi[flat(d, i, j, k)];
}

static inline double dmin(double a, double b) { return a < b ? a : b; }

/*
 * Exact root u of eq. (6):  sum_d ((u - a_d)^+)^2 = tau^2,  a_d = per-axis
 * upwind minimum.  With a1 <= a2 <= a3 (sorted):
 *   one-sided   u = a1 + tau                                valid iff u <= a2
 *   two-sided   u = (a1 + a2 + sqrt(2 tau^2 - (a1-a2)^2))/2 valid iff u <= a3
 *   three-sided u = (a1 + a2 + a3 + sqrt(3 tau^2 - S))/3,
 *               S = (a1-a2)^2 + (a1-a3)^2 + (a2-a3)^2
 * (the three-sided form is the root of 3u^2 - 2u sum(a) + sum(a^2) - tau^2,
 *  the quadratic of Alg 1.3).  a1 = +inf or tau = +inf gives +inf.
 */
double eko_local_solve(double ax, double ay, double az, double tau) {
    double a1 = ax, a2 = ay, a3 = az, t;
    /* sort three values */
    if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
    if (a2 > a3) { t = a2; a2 = a3; a3 = t; }
    if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
    if (isinf(a1) || isinf(tau)) return EKO_INF;
    double u = a1 + tau;
    if (u <= a2) return u;
    double d12 = a1 - a2;
    u = 0.5 * (a1 + a2 + sqrt(2.0 * tau * tau - d12 * d12));
    if (u <= a3) return u;
    double d13 = a1 - a3, d23 = a2 - a3;
    double disc = 3.0 * tau * tau - (d12 * d12 + d13 * d13 + d23 * d23);
    if (disc < 0.0) disc = 0.0; /* >= 0 in exact arithmetic on this branch */
    return (a1 + a2 + a3 + sqrt(disc)) / 3.0;
}

static inline double tau_of(double h, double F) {
    return F > 0.0 ? h / F : EKO_INF;
}

/*
 * Exact root u of eq. (6) with unequal spacings (eq. 5 in 2D as written with
 * dx, dy; Alg 1.2):  sum_d ((u - a_d)^+ / h_d)^2 = 1 / F^2.  The axes with
 * a_d < u at the root are a prefix of the axes sorted by a_d (g(u) = the left
 * side is increasing), so with (a_d, h_d) sorted by a_d:
 *   one-sided   u = a1 + h1 / F                                   valid iff u <= a2
 *   two-sided   u = (a1 h2^2 + a2 h1^2 + h1 h2 sqrt((h1^2 + h2^2)/F^2 - (a1-a2)^2))
 *                   / (h1^2 + h2^2)                               valid iff u <= a3
 *   three-sided with w_d = 1/h_d^2, W = sum w_d:
 *               u = (sum w_d a_d + sqrt(W/F^2 - sum_{i<j} w_i w_j (a_i-a_j)^2)) / W
 * (the two-sided form is Alg 1.2's; its printed switch at |a1-a2| >
 * sqrt(dx^2+dy^2)/F is where the discriminant vanishes, not where the root
 * stops being valid).  F <= 0 or a1 = +inf gives +inf.
 */
double eko_local_solve_aniso(double ax, double ay, double az, double hx, double hy, double hz, double F) {
    double a[3] = {ax, ay, az}, h[3] = {hx, hy, hz};
    /* sort (a, h) pairs by a */
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2 - p; ++q)
            if (a[q] > a[q + 1]) {
                double t = a[q]; a[q] = a[q + 1]; a[q + 1] = t;
                t = h[q]; h[q] = h[q + 1]; h[q + 1] = t;
            }
    if (!(F > 0.0) || isinf(a[0])) return EKO_INF;
    double s = 1.0 / F;
    double u = a[0] + h[0] * s;
    if (u <= a[1]) return u;
    double h1s = h[0] * h[0], h2s = h[1] * h[1], d12 = a[0] - a[1];
    u = (a[0] * h2s + a[1] * h1s + h[0] * h[1] * sqrt((h1s + h2s) * s * s - d12 * d12)) / (h1s + h2s);
    if (u <= a[2]) return u;
    double w[3] = {1.0 / h1s, 1.0 / h2s, 1.0 / (h[2] * h[2])};
    double W = w[0] + w[1] + w[2];
    double sa = w[0] * a[0] + w[1] * a[1] + w[2] * a[2];
    double cross = 0.0;
    for (int p = 0; p < 3; ++p)
        for (int q = p + 1; q < 3; ++q) cross += w[p] * w[q] * (a[p] - a[q]) * (a[p] - a[q]);
    double disc = W * s * s - cross;
    if (disc < 0.0) disc = 0.0; /* >= 0 in exact arithmetic on this branch */
    return (sa + sqrt(disc)) / W;
}

/* grid spacings; iso = all equal (the isotropic cascade of eko_local_solve is used) */
typedef struct {
    double hx, hy, hz;
    int iso;
} spacing_t;

static spacing_t iso_spacing(double h) {
    spacing_t sp = {h, h, h, 1};
    return sp;
}

static spacing_t make_spacing(double hx, double hy, double hz) {
    spacing_t sp = {hx, hy, hz, hx == hy && hy == hz};
    return sp;
}

static int check_spacing(const spacing_t *sp) {
    return !(sp->hx > 0.0 && sp->hy > 0.0 && sp->hz > 0.0) || isinf(sp->hx) || isinf(sp->hy) || isinf(sp->hz);
}

/* local solve at node p (speed Fp) from the current values phi */
static double solve_at(const dims_t *d, const double *phi, int64_t p, const spacing_t *sp, double Fp) {
    int64_t i, j, k;
    unflat(d, p, &i, &j, &k);
    double ax = dmin(nbval(d, phi, i - 1, j, k), nbval(d, phi, i + 1, j, k));
    double ay = dmin(nbval(d, phi, i, j - 1, k), nbval(d, phi, i, j + 1, k));
    double az = dmin(nbval(d, phi, i, j, k - 1), nbval(d, phi, i, j, k + 1));
    if (sp->iso) return eko_local_solve(ax, ay, az, tau_of(sp->hx, Fp));
    return eko_local_solve_aniso(ax, ay, az, sp->hx, sp->hy, sp->hz, Fp);
}

/* neighbour list: up to 6 in-grid face neighbours */
static int neighbours(const dims_t *d, int64_t p, int64_t out[6]) {
    int64_t i, j, k;
    int n = 0;
    unflat(d, p, &i, &j, &k);
    if (i > 0) out[n++] = p - 1;
    if (i + 1 < d->nx) out[n++] = p + 1;
    if (j > 0) out[n++] = p - d->nx;
    if (j + 1 < d->ny) out[n++] = p + d->nx;
    if (k > 0) out[n++] = p - d->nx * d->ny;
    if (k + 1 < d->nz) out[n++] = p + d->nx * d->ny;
    return n;
}

static int check_args(const dims_t *d, double h, const double *F, int64_t n_src,
                      const int64_t *src_idx, const double *src_val) {
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return 1;
    if (!(h > 0.0) || isinf(h)) return 1;
    int64_t N = d->nx * d->ny * d->nz;
    for (int64_t p = 0; p < N; ++p)
        if (!(F[p] >= 0.0) || isinf(F[p])) return 1; /* NaN, negative or inf speed */
    for (int64_t s = 0; s < n_src; ++s) {
        if (src_idx[s] < 0 || src_idx[s] >= N) return 1;
        if (!isfinite(src_val[s])) return 1;
    }
    return 0;
}

/* Dirichlet set-up shared by every solver below: phi = +inf, sources fixed */
static void init_sources(int64_t N, double *phi, unsigned char *is_src, int64_t n_src,
                         const int64_t *src_idx, const double *src_val) {
    for (int64_t p = 0; p < N; ++p) { phi[p] = EKO_INF; is_src[p] = 0; }
    for (int64_t s = 0; s < n_src; ++s) {
        int64_t p = src_idx[s];
        if (!is_src[p] || src_val[s] < phi[p]) phi[p] = src_val[s];
        is_src[p] = 1;
    }
}

/* ------------------------------------------------------------------ */
/* Binary min-heap keyed by (phi[p], p) with a position map (decrease-key). */
typedef struct {
    int64_t *heap;   /* node ids */
    int64_t *pos;    /* position in heap or -1 */
    int64_t size;
    const double *key;
} heap_t;

static inline int heap_less(const heap_t *H, int64_t a, int64_t b) {
    double ka = H->key[a], kb = H->key[b];
    if (ka != kb) return ka < kb;
    return a < b;
}

static void heap_swap(heap_t *H, int64_t x, int64_t y) {
    int64_t a = H->heap[x], b = H->heap[y];
    H->heap[x] = b; H->heap[y] = a;
    H->pos[b] = x; H->pos[a] = y;
}

static void heap_up(heap_t *H, int64_t x) {
    while (x > 0) {
        int64_t par = (x - 1) / 2;
        if (!heap_less(H, H->heap[x], H->heap[par])) break;
        heap_swap(H, x, par);
        x = par;
    }
}

static void heap_down(heap_t *H, int64_t x) {
    for (;;) {
        int64_t l = 2 * x + 1, r = l + 1, m = x;
        if (l < H->size && heap_less(H, H->heap[l], H->heap[m])) m = l;
        if (r < H->size && heap_less(H, H->heap[r], H->heap[m])) m = r;
        if (m == x) break;
        heap_swap(H, x, m);
        x = m;
    }
}

static void heap_push_or_decrease(heap_t *H, int64_t p) {
    if (H->pos[p] < 0) {
        H->heap[H->size] = p;
        H->pos[p] = H->size;
        H->size++;
    }
    heap_up(H, H->pos[p]);
}

static int64_t heap_pop(heap_t *H) {
    int64_t top = H->heap[0];
    H->size--;
    if (H->size > 0) {
        H->heap[0] = H->heap[H->size];
        H->pos[H->heap[0]] = 0;
        heap_down(H, 0);
    }
    H->pos[top] = -1;
    return top;
}

/*
 * Fast marching (Sec. 2.1).  Accepted / Tentative / Distant labels; the
 * tentative set is a min-heap; each popped node is accepted and its
 * non-accepted neighbours are re-solved by eq. (6) from accepted values only.
 * Sources enter the heap at their fixed values and are never re-solved.
 * order_out (nullable) receives the acceptance order; returns the number of
 * accepted nodes (finite phi), or -1 on an argument error.
 */
static int64_t fmm_impl(int64_t nx, int64_t ny, int64_t nz, spacing_t sp, const double *F,
                        int64_t n_src, const int64_t *src_idx, const double *src_val,
                        double *phi, int64_t *order_out) {
    dims_t d = {nx, ny, nz};
    if (check_args(&d, sp.hx, F, n_src, src_idx, src_val) || check_spacing(&sp)) return -1;
    int64_t N = nx * ny * nz;
    unsigned char *is_src = malloc((size_t)N);
    unsigned char *accepted = calloc((size_t)N, 1);
    double *known = malloc(sizeof(double) * (size_t)N); /* accepted values, +inf otherwise */
    heap_t H;
    H.heap = malloc(sizeof(int64_t) * (size_t)N);
    H.pos = malloc(sizeof(int64_t) * (size_t)N);
    H.size = 0;
    H.key = phi;
    init_sources(N, phi, is_src, n_src, src_idx, src_val);
    for (int64_t p = 0; p < N; ++p) { H.pos[p] = -1; known[p] = EKO_INF; }
    for (int64_t p = 0; p < N; ++p)
        if (is_src[p]) heap_push_or_decrease(&H, p);
    int64_t n_acc = 0;
    while (H.size > 0) {
        int64_t p = heap_pop(&H);
        accepted[p] = 1;
        known[p] = phi[p];
        if (order_out) order_out[n_acc] = p;
        n_acc++;
        int64_t nb[6];
        int nn = neighbours(&d, p, nb);
        for (int q = 0; q < nn; ++q) {
            int64_t r = nb[q];
            if (accepted[r] || is_src[r]) continue;
            double u = solve_at(&d, known, r, &sp, F[r]);
            if (u < phi[r]) {
                phi[r] = u;
                heap_push_or_decrease(&H, r);
            }
        }
    }
    free(is_src); free(accepted); free(known); free(H.heap); free(H.pos);
    return n_acc;
}

int64_t eko_fmm(int64_t nx, int64_t ny, int64_t nz, double h, const double *F,
                int64_t n_src, const int64_t *src_idx, const double *src_val,
                double *phi, int64_t *order_out) {
    return fmm_impl(nx, ny, nz, iso_spacing(h), F, n_src, src_idx, src_val, phi, order_out);
}

/* fast marching with spacings hx, hy, hz (equal spacings take the isotropic cascade) */
int64_t eko_fmm_aniso(int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz, const double *F,
                      int64_t n_src, const int64_t *src_idx, const double *src_val,
                      double *phi, int64_t *order_out) {
    return fmm_impl(nx, ny, nz, make_spacing(hx, hy, hz), F, n_src, src_idx, src_val, phi, order_out);
}

/*
 * Gauss-Seidel with alternating sweep orders (Sec. 2.2): in 2D the four
 * orders (i up/down) x (j up/down); in 3D the eight analogous orders.  Each
 * non-source node takes phi = min(phi, eq.(6) root).  Rounds of all 2^d
 * sweeps repeat until a full round changes no value (exact FP64 equality).
 * Returns the number of rounds, or -1 on an argument error, or -2 when
 * max_rounds is reached.
 */
static int64_t gs_impl(int64_t nx, int64_t ny, int64_t nz, spacing_t sp, const double *F,
                       int64_t n_src, const int64_t *src_idx, const double *src_val,
                       double *phi, int64_t max_rounds) {
    dims_t d = {nx, ny, nz};
    if (check_args(&d, sp.hx, F, n_src, src_idx, src_val) || check_spacing(&sp)) return -1;
    int64_t N = nx * ny * nz;
    unsigned char *is_src = malloc((size_t)N);
    init_sources(N, phi, is_src, n_src, src_idx, src_val);
    int ndir = nz > 1 ? 8 : 4;
    int64_t rounds = 0;
    int changed = 1;
    while (changed) {
        if (rounds >= max_rounds) { free(is_src); return -2; }
        changed = 0;
        rounds++;
        for (int s = 0; s < ndir; ++s) {
            int rx = s & 1, ry = (s >> 1) & 1, rz = (s >> 2) & 1;
            for (int64_t kk = 0; kk < nz; ++kk) {
                int64_t k = rz ? nz - 1 - kk : kk;
                for (int64_t jj = 0; jj < ny; ++jj) {
                    int64_t j = ry ? ny - 1 - jj : jj;
                    for (int64_t ii = 0; ii < nx; ++ii) {
                        int64_t i = rx ? nx - 1 - ii : ii;
                        int64_t p = flat(&d, i, j, k);
                        if (is_src[p]) continue;
                        double u = solve_at(&d, phi, p, &sp, F[p]);
                        if (u < phi[p]) { phi[p] = u; changed = 1; }
                    }
                }
            }
        }
    }
    free(is_src);
    return rounds;
}

int64_t eko_gs(int64_t nx, int64_t ny, int64_t nz, double h, const double *F,
               int64_t n_src, const int64_t *src_idx, const double *src_val,
               double *phi, int64_t max_rounds) {
    return gs_impl(nx, ny, nz, iso_spacing(h), F, n_src, src_idx, src_val, phi, max_rounds);
}

int64_t eko_gs_aniso(int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz, const double *F,
                     int64_t n_src, const int64_t *src_idx, const double *src_val,
                     double *phi, int64_t max_rounds) {
    return gs_impl(nx, ny, nz, make_spacing(hx, hy, hz), F, n_src, src_idx, src_val, phi, max_rounds);
}

/*
 * Algorithm 2, point by point, with the parallel semantics of Sec. 3.2:
 * in every iteration all listed points first compute phi~ from the values at
 * the start of the iteration, then all of them update the sets.
 *   Step 1: Source = given points with their values, others +inf;
 *           Active = points adjacent to Source.
 *   Step 2: while Active is not empty: phi~ = eq.(6) root; if phi~ == phi the
 *           point leaves Active, joins Source, and each neighbour not in
 *           Active or Source joins Active; otherwise phi = phi~ (kept as
 *           min(phi, phi~), which is the same in exact arithmetic).
 *   Step 3: Remedy = non-source points whose phi~ < phi (recomputed over the
 *           whole grid); then repeat: a Remedy point with phi~ < phi takes
 *           phi~ and its neighbours not in Remedy join it; a point with
 *           phi~ >= phi leaves Remedy; until Remedy is empty.
 * Fixed (given) sources are never recomputed.  stats (nullable, 4 entries):
 * update iterations, remedy iterations, size of the initial Remedy set,
 * total remedy point-updates that lowered a value.
 * Returns 0, -1 on an argument error, -2 on reaching max_iters.
 */
int eko_ifim(int64_t nx, int64_t ny, int64_t nz, double h, const double *F,
             int64_t n_src, const int64_t *src_idx, const double *src_val,
             double *phi, int skip_remedy, int64_t max_iters, int64_t *stats) {
    dims_t d = {nx, ny, nz};
    spacing_t sp = iso_spacing(h);
    if (check_args(&d, h, F, n_src, src_idx, src_val)) return -1;
    int64_t N = nx * ny * nz;
    unsigned char *is_fixed = malloc((size_t)N);
    /* set labels: bit0 Active (current), bit1 Source, bit2 Active (next) */
    unsigned char *lab = calloc((size_t)N, 1);
    int64_t *list = malloc(sizeof(int64_t) * (size_t)N);
    int64_t *next = malloc(sizeof(int64_t) * (size_t)N);
    double *cand = malloc(sizeof(double) * (size_t)N);
    int64_t st[4] = {0, 0, 0, 0};
    int rc = 0;
    init_sources(N, phi, is_fixed, n_src, src_idx, src_val);

    /* Step 1 */
    int64_t n = 0;
    for (int64_t p = 0; p < N; ++p) if (is_fixed[p]) lab[p] |= 2;
    for (int64_t p = 0; p < N; ++p) {
        if (!is_fixed[p]) continue;
        int64_t nb[6];
        int nn = neighbours(&d, p, nb);
        for (int q = 0; q < nn; ++q)
            if (!(lab[nb[q]] & 3)) { lab[nb[q]] |= 1; list[n++] = nb[q]; }
    }

    /* Step 2 */
    while (n > 0) {
        if (st[0] >= max_iters) { rc = -2; goto done; }
        st[0]++;
        for (int64_t a = 0; a < n; ++a)
            cand[a] = solve_at(&d, phi, list[a], &sp, F[list[a]]);
        int64_t m = 0;
        for (int64_t a = 0; a < n; ++a) {
            int64_t p = list[a];
            if (cand[a] == phi[p]) {
                lab[p] = (unsigned char)((lab[p] & ~1) | 2);
                int64_t nb[6];
                int nn = neighbours(&d, p, nb);
                for (int q = 0; q < nn; ++q) {
                    int64_t r = nb[q];
                    if (!(lab[r] & 3) && !(lab[r] & 4)) { lab[r] |= 4; next[m++] = r; }
                }
            } else {
                if (cand[a] < phi[p]) phi[p] = cand[a];
                lab[p] |= 4;
                next[m++] = p;
            }
        }
        for (int64_t a = 0; a < m; ++a) lab[next[a]] = (unsigned char)((lab[next[a]] & ~4) | 1);
        int64_t *t = list; list = next; next = t;
        n = m;
    }

    if (!skip_remedy) {
        /* Step 3: seed.  lab bit4 = already in the Remedy set being formed
         * for the next iteration (the "not in Remedy" test of the loop is
         * taken against that set, so that a neighbour that was listed, did
         * not change and was dropped is listed again once a neighbour of it
         * changes). */
        n = 0;
        for (int64_t p = 0; p < N; ++p) {
            if (is_fixed[p]) continue;
            double u = solve_at(&d, phi, p, &sp, F[p]);
            if (u < phi[p]) list[n++] = p;
        }
        st[2] = n;
        while (n > 0) {
            if (st[1] >= max_iters) { rc = -2; goto done; }
            st[1]++;
            for (int64_t a = 0; a < n; ++a)
                cand[a] = solve_at(&d, phi, list[a], &sp, F[list[a]]);
            int64_t m = 0;
            for (int64_t a = 0; a < n; ++a) {
                int64_t p = list[a];
                if (cand[a] < phi[p]) {
                    phi[p] = cand[a];
                    st[3]++;
                    if (!(lab[p] & 16)) { lab[p] |= 16; next[m++] = p; }
                    int64_t nb[6];
                    int nn = neighbours(&d, p, nb);
                    for (int q = 0; q < nn; ++q) {
                        int64_t r = nb[q];
                        if (is_fixed[r]) continue;
                        if (!(lab[r] & 16)) { lab[r] |= 16; next[m++] = r; }
                    }
                }
            }
            for (int64_t a = 0; a < m; ++a) lab[next[a]] &= (unsigned char)~16;
            int64_t *t = list; list = next; next = t;
            n = m;
        }
    }
done:
    if (stats) memcpy(stats, st, sizeof(st));
    free(is_fixed); free(lab); free(list); free(next); free(cand);
    return rc;
}

/*
 * The fast iterative method of Sec. 2.3, point by point.  Active starts as
 * the points adjacent to the sources (as Step 1 of Algorithm 2).  Every
 * iteration has two phases:
 *   (a) every Active point computes phi~ from the values at the start of the
 *       iteration;
 *   (b) a point with phi~ == phi has converged: it leaves Active and each of
 *       its neighbours that is neither a fixed source nor Active (now or for
 *       the next iteration) is checked: its phi~ is computed from the current
 *       values and, if it is below its value (the neighbour is +inf or not
 *       converged), the neighbour takes phi~ and joins Active.  A point with
 *       phi~ != phi takes min(phi, phi~) and stays Active.
 * The loop ends when Active is empty.  stats (nullable, 2 entries):
 * iterations, neighbour checks that listed a point.
 * Returns 0, -1 on an argument error, -2 on reaching max_iters.
 */
int eko_fim(int64_t nx, int64_t ny, int64_t nz, double h, const double *F,
            int64_t n_src, const int64_t *src_idx, const double *src_val,
            double *phi, int64_t max_iters, int64_t *stats) {
    dims_t d = {nx, ny, nz};
    spacing_t sp = iso_spacing(h);
    if (check_args(&d, h, F, n_src, src_idx, src_val)) return -1;
    int64_t N = nx * ny * nz;
    unsigned char *is_fixed = malloc((size_t)N);
    /* bit0 Active (current iteration), bit2 Active (next iteration) */
    unsigned char *lab = calloc((size_t)N, 1);
    int64_t *list = malloc(sizeof(int64_t) * (size_t)N);
    int64_t *next = malloc(sizeof(int64_t) * (size_t)N);
    double *cand = malloc(sizeof(double) * (size_t)N);
    int64_t st[2] = {0, 0};
    int rc = 0;
    init_sources(N, phi, is_fixed, n_src, src_idx, src_val);

    int64_t n = 0;
    for (int64_t p = 0; p < N; ++p) {
        if (!is_fixed[p]) continue;
        int64_t nb[6];
        int nn = neighbours(&d, p, nb);
        for (int q = 0; q < nn; ++q)
            if (!is_fixed[nb[q]] && !(lab[nb[q]] & 1)) { lab[nb[q]] |= 1; list[n++] = nb[q]; }
    }
    while (n > 0) {
        if (st[0] >= max_iters) { rc = -2; goto done; }
        st[0]++;
        for (int64_t a = 0; a < n; ++a)
            cand[a] = solve_at(&d, phi, list[a], &sp, F[list[a]]);
        int64_t m = 0;
        for (int64_t a = 0; a < n; ++a) {
            int64_t p = list[a];
            if (cand[a] == phi[p]) {
                int64_t nb[6];
                int nn = neighbours(&d, p, nb);
                for (int q = 0; q < nn; ++q) {
                    int64_t r = nb[q];
                    if (is_fixed[r] || (lab[r] & 5)) continue;
                    double u = solve_at(&d, phi, r, &sp, F[r]);
                    if (u < phi[r]) {
                        phi[r] = u;
                        lab[r] |= 4;
                        next[m++] = r;
                        st[1]++;
                    }
                }
            } else {
                if (cand[a] < phi[p]) phi[p] = cand[a];
                lab[p] |= 4;
                next[m++] = p;
            }
        }
        for (int64_t a = 0; a < n; ++a) lab[list[a]] &= (unsigned char)~1;
        for (int64_t a = 0; a < m; ++a) lab[next[a]] = (unsigned char)((lab[next[a]] & ~4) | 1);
        int64_t *t = list; list = next; next = t;
        n = m;
    }
done:
    if (stats) memcpy(stats, st, sizeof(st));
    free(is_fixed); free(lab); free(list); free(next); free(cand);
    return rc;
}

/*
 * Residual of eq. (6) at every non-source node with finite phi:
 *   R_p = sum_d ((phi_p - a_d)^+)^2 - tau_p^2, reported relative to tau_p^2.
 * Writes |R_p| / tau_p^2 into res (nullable; 0 at sources and +inf nodes) and
 * returns the maximum.  Nodes with finite phi but tau = +inf (impassable and
 * not a source) count as an infinite residual.
 */
static double residual_impl(int64_t nx, int64_t ny, int64_t nz, spacing_t sp, const double *F,
                            int64_t n_src, const int64_t *src_idx, const double *phi, double *res) {
    dims_t d = {nx, ny, nz};
    const double hd[3] = {sp.hx, sp.hy, sp.hz};
    int64_t N = nx * ny * nz;
    unsigned char *is_src = calloc((size_t)N, 1);
    for (int64_t s = 0; s < n_src; ++s)
        if (src_idx[s] >= 0 && src_idx[s] < N) is_src[src_idx[s]] = 1;
    double worst = 0.0;
    for (int64_t p = 0; p < N; ++p) {
        double r = 0.0;
        if (!is_src[p] && isfinite(phi[p])) {
            double tau = tau_of(sp.hx, F[p]);
            if (isinf(tau)) {
                r = EKO_INF;
            } else if (!sp.iso) {
                /* sum_d ((phi - a_d)^+ / h_d)^2 against 1 / F^2 */
                int64_t i, j, k;
                unflat(&d, p, &i, &j, &k);
                double a[3];
                a[0] = dmin(nbval(&d, phi, i - 1, j, k), nbval(&d, phi, i + 1, j, k));
                a[1] = dmin(nbval(&d, phi, i, j - 1, k), nbval(&d, phi, i, j + 1, k));
                a[2] = dmin(nbval(&d, phi, i, j, k - 1), nbval(&d, phi, i, j, k + 1));
                double sum = 0.0, s2 = 1.0 / (F[p] * F[p]);
                for (int q = 0; q < 3; ++q) {
                    double t = (phi[p] - a[q]) / hd[q];
                    if (t > 0.0) sum += t * t;
                }
                r = fabs(sum - s2) / s2;
            } else {
                int64_t i, j, k;
                unflat(&d, p, &i, &j, &k);
                double a[3];
                a[0] = dmin(nbval(&d, phi, i - 1, j, k), nbval(&d, phi, i + 1, j, k));
                a[1] = dmin(nbval(&d, phi, i, j - 1, k), nbval(&d, phi, i, j + 1, k));
                a[2] = dmin(nbval(&d, phi, i, j, k - 1), nbval(&d, phi, i, j, k + 1));
                double sum = 0.0;
                for (int q = 0; q < 3; ++q) {
                    double t = phi[p] - a[q];
                    if (t > 0.0) sum += t * t;
                }
                r = fabs(sum - tau * tau) / (tau * tau);
            }
        }
        if (res) res[p] = r;
        if (r > worst) worst = r;
    }
    free(is_src);
    return worst;
}

double eko_residual(int64_t nx, int64_t ny, int64_t nz, double h, const double *F,
                    int64_t n_src, const int64_t *src_idx, const double *phi, double *res) {
    return residual_impl(nx, ny, nz, iso_spacing(h), F, n_src, src_idx, phi, res);
}

double eko_residual_aniso(int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz, const double *F,
                          int64_t n_src, const int64_t *src_idx, const double *phi, double *res) {
    return residual_impl(nx, ny, nz, make_spacing(hx, hy, hz), F, n_src, src_idx, phi, res);
}

/* ------------------------------------------------------------------ */
/*
 * Shortest-path back-trace by descent on the phi map (the application of
 * Example 4, Sec. 4.1; the paper names gradient descent without stating the
 * discrete rule, so this is the steepest descent on the grid graph):
 * from the start node, repeatedly move to the neighbour among the 26 (8 in
 * 2D) adjacent nodes with the steepest descent slope
 *     (phi[nb] - phi[cur]) / |x_nb - x_cur|      (physical distance, spacings hx, hy, hz)
 * among the neighbours with phi[nb] < phi[cur]; ties go to the lower flat
 * index.  The slope is formed in double as (phi[nb] - phi[cur]) * (1 / len),
 * with 1 / len = 1 / sqrt(dx^2 + dy^2 + dz^2) of the offset.  The path stops
 * at a node with no lower neighbour (a source or a local minimum) or after
 * max_len nodes.  phi = +inf at the start gives an empty path.
 * path_out: [n_paths][max_len] node ids (entries past len are -1);
 * len_out: [n_paths].  Returns 0, or -1 on an argument error.
 */
int eko_backtrace(int64_t nx, int64_t ny, int64_t nz, double hx, double hy, double hz, const double *phi,
                  int64_t n_paths, const int64_t *start_idx, int64_t max_len, int64_t *path_out,
                  int64_t *len_out) {
    dims_t d = {nx, ny, nz};
    spacing_t sp = make_spacing(hx, hy, hz);
    if (nx < 1 || ny < 1 || nz < 1 || check_spacing(&sp) || n_paths < 0 || max_len < 1) return -1;
    int64_t N = nx * ny * nz;
    for (int64_t q = 0; q < n_paths; ++q)
        if (start_idx[q] < 0 || start_idx[q] >= N) return -1;
    for (int64_t q = 0; q < n_paths; ++q) {
        int64_t *row = path_out + q * max_len;
        for (int64_t t = 0; t < max_len; ++t) row[t] = -1;
        int64_t cur = start_idx[q], len = 0;
        if (!isinf(phi[cur])) {
            row[len++] = cur;
            while (len < max_len) {
                int64_t i, j, k;
                unflat(&d, cur, &i, &j, &k);
                int64_t best = -1;
                double best_slope = 0.0;
                for (int dk = -1; dk <= 1; ++dk)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int di = -1; di <= 1; ++di) {
                            if (!di && !dj && !dk) continue;
                            int64_t a = i + di, b = j + dj, c = k + dk;
                            if (a < 0 || b < 0 || c < 0 || a >= nx || b >= ny || c >= nz) continue;
                            int64_t nb = flat(&d, a, b, c);
                            if (!(phi[nb] < phi[cur])) continue;
                            double ox = di * hx, oy = dj * hy, oz = dk * hz;
                            double inv_len = 1.0 / sqrt(ox * ox + oy * oy + oz * oz);
                            double slope = (phi[nb] - phi[cur]) * inv_len;
                            if (best < 0 || slope < best_slope || (slope == best_slope && nb < best)) {
                                best = nb;
                                best_slope = slope;
                            }
                        }
                if (best < 0) break;
                cur = best;
                row[len++] = cur;
            }
        }
        len_out[q] = len;
    }
    return 0;
}

/* ordering helper for the adjoint: sort node ids by (phi, id) */
static const double *g_sort_key;
static int cmp_by_phi(const void *x, const void *y) {
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    double ka = g_sort_key[a], kb = g_sort_key[b];
    if (ka < kb) return -1;
    if (ka > kb) return 1;
    return (a > b) - (a < b);
}

/*
 * Adjoint of the discrete solve with respect to slowness s = 1/F.
 * Residual form at a non-source node i:
 *   G_i(phi, s) = sum_d ((phi_i - m_{i,d})^+)^2 - h^2 s_i^2 = 0,
 * with m_{i,d} the selected upwind neighbour along axis d (argmin of the two
 * neighbours; on a tie the lower flat index).  With w_{i,d} = 2(phi_i -
 * m_{i,d})^+ the Jacobian is J_ii = sum_d w_{i,d}, J_{i,m_{i,d}} = -w_{i,d},
 * and dG_i/ds_i = -2 h^2 s_i.  For a loss L with r = dL/dphi, the adjoint
 * lambda solves J^T lambda = r:
 *   lambda_i = (r_i + sum_{j : m_{j,d} = i} w_{j,d} lambda_j) / J_ii,
 * a back substitution in decreasing-phi order (J is triangular in
 * increasing-phi order because w_{j,d} > 0 implies phi_j > m_{j,d}).  Then
 *   dL/ds_i = 2 h^2 s_i lambda_i  for non-source nodes with finite phi,
 * and 0 at sources, impassable and unreachable nodes.  This is the
 * adjoint-state traveltime method (Leung & Qian 2006) applied to eq. (6).
 * g receives the gradient (overwritten); lambda_out (nullable) the adjoint.
 * Returns 0, or -1 on an argument error.
 */
int eko_adjoint(int64_t nx, int64_t ny, int64_t nz, double h, const double *F,
                int64_t n_src, const int64_t *src_idx, const double *phi,
                const double *r, double *g, double *lambda_out) {
    dims_t d = {nx, ny, nz};
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || !(h > 0.0)) return -1;
    int64_t N = nx * ny * nz;
    unsigned char *is_src = calloc((size_t)N, 1);
    for (int64_t s = 0; s < n_src; ++s) {
        if (src_idx[s] < 0 || src_idx[s] >= N) { free(is_src); return -1; }
        is_src[src_idx[s]] = 1;
    }
    int64_t *ord = malloc(sizeof(int64_t) * (size_t)N);
    double *acc = calloc((size_t)N, sizeof(double));
    double *lam = calloc((size_t)N, sizeof(double));
    int64_t nfin = 0;
    for (int64_t p = 0; p < N; ++p)
        if (isfinite(phi[p])) ord[nfin++] = p;
    g_sort_key = phi;
    qsort(ord, (size_t)nfin, sizeof(int64_t), cmp_by_phi);
    int64_t stride[3] = {1, nx, nx * ny};
    for (int64_t q = nfin - 1; q >= 0; --q) {
        int64_t j = ord[q];
        if (is_src[j]) continue;
        int64_t c[3];
        unflat(&d, j, &c[0], &c[1], &c[2]);
        int64_t ext[3] = {nx, ny, nz};
        int64_t msel[3];
        double w[3], Jjj = 0.0;
        for (int ax = 0; ax < 3; ++ax) {
            int64_t lo = c[ax] > 0 ? j - stride[ax] : -1;
            int64_t hi = c[ax] + 1 < ext[ax] ? j + stride[ax] : -1;
            double vlo = lo >= 0 ? phi[lo] : EKO_INF;
            double vhi = hi >= 0 ? phi[hi] : EKO_INF;
            /* argmin, tie -> lower flat index (lo < hi always) */
            int64_t m = (vhi < vlo) ? hi : lo;
            double vm = (vhi < vlo) ? vhi : vlo;
            double t = (m >= 0 && isfinite(vm)) ? phi[j] - vm : 0.0;
            w[ax] = t > 0.0 ? 2.0 * t : 0.0;
            msel[ax] = m;
            Jjj += w[ax];
        }
        if (!(Jjj > 0.0)) continue;
        double lj = (r[j] + acc[j]) / Jjj;
        lam[j] = lj;
        for (int ax = 0; ax < 3; ++ax)
            if (w[ax] > 0.0) acc[msel[ax]] += w[ax] * lj;
    }
    for (int64_t p = 0; p < N; ++p) {
        double gp = 0.0;
        if (!is_src[p] && isfinite(phi[p]) && F[p] > 0.0) gp = 2.0 * h * h * (1.0 / F[p]) * lam[p];
        g[p] = gp;
        if (lambda_out) lambda_out[p] = lam[p];
    }
    free(is_src); free(ord); free(acc); free(lam);
    return 0;
}
