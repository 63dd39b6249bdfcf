/*
 * lbg_oracle.c -- plain, slow, FP64 CPU oracle of the LBG codebook design.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the independent checker of the CUDA
 * library: only the tests, the smoke check and the bench's CPU-baseline leg
 * load it.  It shares no source, header, table or constant with the CUDA
 * path, and the CUDA path never loads it.
 *
 * Method followed (Annaji & Rao, "Parallelization of the LBG Vector
 * Quantization Algorithm for Shared Memory Systems"):
 *   Sec. 2.2 "LBG Algorithm" (after Linde, Buzo & Gray): the minimum
 *     distortion partition, the distortion D_m, the relative stop test and
 *     the replacement of every codevector by the centroid of its cell.
 *   Sec. 3.2, Algorithm 1 and the prose that follows it: the initial
 *     codebook is the centroid of the whole training set (Table 1),
 *     "Codebook Splitting" turns every centroid c into c+delta and c-delta,
 *     "Cell Allocation" gives every input vector the index of its nearest
 *     codevector (the cell table) and accumulates the distortion,
 *     "Updation" replaces each codevector by the centroid of the vectors
 *     extracted from its cell.
 *
 * Arithmetic: inputs X are the float32 values the GPU sees, widened exactly
 * to double; everything else is double, round-to-nearest, summed in index
 * order.  Compile with -ffp-contract=off so that x86 and aarch64 builds give
 * identical bits.
 *
 * Readings taken where the paper is silent, garbled or inconsistent:
 *   R1 stop test: (D_prev - D) / D <= theta, the Sec. 2.2 form (Sec. 3.2
 *      divides by the previous distortion instead); "<=" so that theta = 0
 *      ends a stage whose distortion repeats exactly.
 *   R2 D == 0 ends the stage (the ratio would be 0/0).
 *   R3 D_prev = +infinity at the start of every stage, not only once.
 *   R4 a finished stage keeps the codebook that produced D (A_m, before any
 *      update), so (C, cell table, D) returned are mutually consistent.
 *   R5 split is additive on every component: c + delta, c - delta.
 *   R6 children are interleaved: child 2i = c_i + delta, 2i+1 = c_i - delta.
 *   R7 distance is the squared Euclidean distance.
 *   R8 D is the sum of per-vector minimum distances (the mean is D/M).
 *   R9 ties go to the lowest codevector index.
 *   R10 an empty cell keeps its previous codevector.
 *   R11 a stage that reaches max_passes assignments without meeting the
 *       test is ended there (status LBG oracle WARN_MAXPASS = 1) and
 *       training continues with the next split.
 * Opt-in variants (not the paper's defaults):
 *   V1 multiplicative split: child 2i = c_i (1 + delta), 2i+1 = c_i (1 - delta).
 *   V2 empty-cell re-seeding after an update: for every empty cell e in
 *      increasing index order, take the cell b with the largest count (lowest
 *      index on ties), set c_e = c_b + delta and c_b = c_b - delta (every
 *      component), and let e take half of b's count (floor) and b keep the
 *      rest, so that the next empty cell may pick another cell.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_WARN_MAXPASS 1
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_NOT_POW2 (-2)
#define ORACLE_ERR_NOMEM (-5)

/* Number of OpenMP threads a parallel region with nthreads <= 0 would use. */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Squared Euclidean distance between input vector x (float32) and
 * codevector c (double), dimension by dimension in index order
 * (Sec. 2.2 d(x_j, y_i); Sec. 3.2 "Cell Allocation": Euclidean distance). */
static double sq_dist(const float *x, const double *c, int32_t L)
{
    double s = 0.0;
    for (int32_t l = 0; l < L; ++l) {
        double d = (double)x[l] - c[l];
        s += d * d;
    }
    return s;
}

/* Initial codebook: the centroid of all M training vectors (Algorithm 1,
 * "compute centroid(input)"; Table 1).  c_out has L entries. */
int oracle_mean(const float *X, int64_t M, int32_t L, double *c_out)
{
    if (!X || !c_out || M < 1 || L < 1) return ORACLE_ERR_ARG;
    for (int32_t l = 0; l < L; ++l) c_out[l] = 0.0;
    for (int64_t m = 0; m < M; ++m)
        for (int32_t l = 0; l < L; ++l) c_out[l] += (double)X[m * L + l];
    for (int32_t l = 0; l < L; ++l) c_out[l] /= (double)M;
    return ORACLE_OK;
}

/* Codebook splitting (Algorithm 1; Sec. 3.2 "Codebook Splitting"): every
 * centroid c_i of the n-entry codebook C becomes two codevectors,
 * C2[2i] = c_i + delta and C2[2i+1] = c_i - delta (readings R5, R6). */
int oracle_split_mode(const double *C, int32_t n, int32_t L, double delta, int32_t mult, double *C2)
{
    if (!C || !C2 || n < 1 || L < 1) return ORACLE_ERR_ARG;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t l = 0; l < L; ++l) {
            const double c = C[(int64_t)i * L + l];
            C2[(2 * (int64_t)i) * L + l] = mult ? c * (1.0 + delta) : c + delta;
            C2[(2 * (int64_t)i + 1) * L + l] = mult ? c * (1.0 - delta) : c - delta;
        }
    return ORACLE_OK;
}

int oracle_split(const double *C, int32_t n, int32_t L, double delta, double *C2)
{
    return oracle_split_mode(C, n, L, delta, 0, C2);
}

/* Variant V2: re-seed the empty cells of an updated codebook C (in place)
 * from the largest cells; counts [N] are the cell sizes (updated in place). */
int oracle_reseed(double *C, int64_t *counts, int32_t N, int32_t L, double delta)
{
    if (!C || !counts || N < 1 || L < 1) return ORACLE_ERR_ARG;
    for (int32_t e = 0; e < N; ++e) {
        if (counts[e] != 0) continue;
        int32_t b = 0;
        for (int32_t n = 1; n < N; ++n)
            if (counts[n] > counts[b]) b = n;
        if (counts[b] < 2) break;   /* nothing left to split */
        for (int32_t l = 0; l < L; ++l) {
            const double c = C[(int64_t)b * L + l];
            C[(int64_t)e * L + l] = c + delta;
            C[(int64_t)b * L + l] = c - delta;
        }
        counts[e] = counts[b] / 2;
        counts[b] -= counts[e];
    }
    return ORACLE_OK;
}

/* Cell allocation (Algorithm 1 "Cell Allocation"; Sec. 2.2 minimum
 * distortion partition).  For every input vector m:
 *   a[m]   = index of the nearest codevector (lowest index on ties, R9),
 *   e[m]   = its squared distance (the MinDist added to D_rho),
 *   gap[m] = (d_2 - d_1) / d_1, the relative gap between the two smallest
 *            distances (+inf if N == 1 or d_1 == 0 < d_2; 0 if both are 0).
 * e and gap may be NULL.  The rows are split into nthreads contiguous
 * chunks, one per processor, as in the paper's data-parallel allocation;
 * every row's result is independent of that split. */
int oracle_assign(const float *X, int64_t M, int32_t L, const double *C, int32_t N,
                  int32_t *a, double *e, double *gap, int32_t nthreads)
{
    if (!X || !C || !a || M < 0 || L < 1 || N < 1) return ORACLE_ERR_ARG;
#ifdef _OPENMP
    int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nth)
#endif
    for (int64_t m = 0; m < M; ++m) {
        const float *x = X + m * L;
        double d1 = INFINITY, d2 = INFINITY;
        int32_t best = 0;
        for (int32_t n = 0; n < N; ++n) {
            double d = sq_dist(x, C + (int64_t)n * L, L);
            if (d < d1) {
                d2 = d1;
                d1 = d;
                best = n;
            } else if (d < d2) {
                d2 = d;
            }
        }
        a[m] = best;
        if (e) e[m] = d1;
        if (gap) {
            if (N == 1)
                gap[m] = INFINITY;
            else if (d1 > 0.0)
                gap[m] = (d2 - d1) / d1;
            else
                gap[m] = (d2 > 0.0) ? INFINITY : 0.0;
        }
    }
    (void)nthreads;
    return ORACLE_OK;
}

/* Integration of distortions (Algorithm 1 "IntegrateDistortions";
 * TD = sum of D_i): the total of e[0..M) in index order. */
double oracle_sum(const double *e, int64_t M)
{
    double s = 0.0;
    for (int64_t m = 0; m < M; ++m) s += e[m];
    return s;
}

/* Updation (Algorithm 1 "Updation step"; Sec. 2.2 step 3): codevector n
 * becomes the centroid of the input vectors whose cell-table entry is n
 * (ExtractVectors + centroid).  One sweep over the rows in index order adds
 * every vector into its own cell, which is the same per-cell sum in the same
 * order as extracting each cell first.  counts[n] receives the cell sizes
 * (may be NULL).  An empty cell keeps C_in[n] (reading R10). */
int oracle_update(const float *X, int64_t M, int32_t L, const int32_t *a, int32_t N,
                  const double *C_in, double *C_out, int64_t *counts)
{
    if (!X || !a || !C_in || !C_out || M < 0 || L < 1 || N < 1) return ORACLE_ERR_ARG;
    double *sum = (double *)calloc((size_t)N * L, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    if (!sum || !cnt) {
        free(sum);
        free(cnt);
        return ORACLE_ERR_NOMEM;
    }
    for (int64_t m = 0; m < M; ++m) {
        int32_t n = a[m];
        if (n < 0 || n >= N) {
            free(sum);
            free(cnt);
            return ORACLE_ERR_ARG;
        }
        cnt[n] += 1;
        for (int32_t l = 0; l < L; ++l) sum[(int64_t)n * L + l] += (double)X[m * L + l];
    }
    for (int32_t n = 0; n < N; ++n) {
        for (int32_t l = 0; l < L; ++l) {
            int64_t i = (int64_t)n * L + l;
            C_out[i] = cnt[n] > 0 ? sum[i] / (double)cnt[n] : C_in[i];
        }
        if (counts) counts[n] = cnt[n];
    }
    free(sum);
    free(cnt);
    return ORACLE_OK;
}

/* One Lloyd pass from a given codebook: cell allocation, integration of the
 * distortion, and the updation -- unconditionally, without the stop test.
 * Outputs: a, e, gap (e, gap may be NULL), D (sum), C_out, counts (NULL ok). */
int oracle_lloyd_step(const float *X, int64_t M, int32_t L, const double *C_in, int32_t N,
                      int32_t *a, double *e, double *gap, double *D, double *C_out,
                      int64_t *counts, int32_t nthreads)
{
    if (!X || !C_in || !a || !D || !C_out || M < 1 || L < 1 || N < 1) return ORACLE_ERR_ARG;
    double *ee = e ? e : (double *)malloc((size_t)M * sizeof(double));
    if (!ee) return ORACLE_ERR_NOMEM;
    int rc = oracle_assign(X, M, L, C_in, N, a, ee, gap, nthreads);
    if (rc == ORACLE_OK) {
        *D = oracle_sum(ee, M);
        rc = oracle_update(X, M, L, a, N, C_in, C_out, counts);
    }
    if (!e) free(ee);
    return rc;
}

/* Distortion at a fixed cell table: sum_m ||x_m - C[a[m]]||^2 (the D of
 * Sec. 2.2 without the minimisation), used to check gradients. */
double oracle_distortion_fixed(const float *X, int64_t M, int32_t L, const double *C,
                               const int32_t *a)
{
    double s = 0.0;
    for (int64_t m = 0; m < M; ++m) s += sq_dist(X + m * L, C + (int64_t)a[m] * L, L);
    return s;
}

/* Analytic gradient of D = sum_m ||x_m - c_{a(m)}||^2 at a fixed cell table:
 *   dD/dc_n = 2 (count_n c_n - sum_{a(m)=n} x_m),   gC is [N x L]
 *   dD/dx_m = 2 (x_m - c_{a(m)}),                   gX is [M x L]
 * Either output may be NULL.  (Not in the paper: the differentiable form of
 * its distortion.) */
int oracle_grad(const float *X, int64_t M, int32_t L, const double *C, int32_t N,
                const int32_t *a, double *gC, double *gX)
{
    if (!X || !C || !a || M < 0 || L < 1 || N < 1) return ORACLE_ERR_ARG;
    if (gC) {
        for (int64_t i = 0; i < (int64_t)N * L; ++i) gC[i] = 0.0;
        int64_t *cnt = (int64_t *)calloc((size_t)N, sizeof(int64_t));
        if (!cnt) return ORACLE_ERR_NOMEM;
        for (int64_t m = 0; m < M; ++m) {
            int32_t n = a[m];
            cnt[n] += 1;
            for (int32_t l = 0; l < L; ++l) gC[(int64_t)n * L + l] -= (double)X[m * L + l];
        }
        for (int32_t n = 0; n < N; ++n)
            for (int32_t l = 0; l < L; ++l) {
                int64_t i = (int64_t)n * L + l;
                gC[i] = 2.0 * ((double)cnt[n] * C[i] + gC[i]);
            }
        free(cnt);
    }
    if (gX) {
        for (int64_t m = 0; m < M; ++m)
            for (int32_t l = 0; l < L; ++l)
                gX[m * L + l] = 2.0 * ((double)X[m * L + l] - C[(int64_t)a[m] * L + l]);
    }
    return ORACLE_OK;
}

static int is_pow2(int32_t n) { return n > 0 && (n & (n - 1)) == 0; }

/* The whole LBG design (Algorithm 1 with the Sec. 2.2 iteration inside each
 * stage):
 *   C <- [centroid(X)]; n <- 1   (or, if n_init > 0, C <- C_init, n <- n_init:
 *                                 the initial alphabet A_0 of Sec. 2.2)
 *   stage: D_prev <- +inf (R3)
 *     pass: cell allocation -> a, e;  D <- sum e
 *           if D == 0 or (D_prev - D)/D <= theta: stage done (R1, R2, R4)
 *           else if the stage already ran max_passes passes: done, WARN (R11)
 *           else C <- centroids of the cells; D_prev <- D; next pass
 *     if n == N: stop; else C <- split(C); n <- 2n; next stage
 * Outputs: C_out [N x L] (double), a_out [M], D_out.  Optional pass trace:
 * rec_n (stage size), rec_pass (pass index within the stage), rec_D and
 * rec_near (rows of the pass whose relative gap is <= near_tol, i.e. whose
 * nearest codevector is a near-tie), up to rec_cap records; rec_count
 * receives the number of passes run (which may exceed rec_cap).  Returns 0,
 * 1 (WARN_MAXPASS) or a negative error. */
int oracle_lbg_train(const float *X, int64_t M, int32_t L, int32_t N, double delta,
                     double theta, int32_t max_passes, int32_t nthreads, int32_t split_mult,
                     int32_t reseed, const double *C_init, int32_t n_init, double *C_out,
                     int32_t *a_out, double *D_out, int32_t *rec_n, int32_t *rec_pass,
                     double *rec_D, int32_t *rec_near, double near_tol, int32_t rec_cap,
                     int32_t *rec_count)
{
    if (!X || !C_out || !a_out || !D_out || M < 1 || L < 1 || N < 1 || max_passes < 1)
        return ORACLE_ERR_ARG;
    if (!(delta >= 0.0) || !(theta >= 0.0)) return ORACLE_ERR_ARG;
    if (!is_pow2(N)) return ORACLE_ERR_NOT_POW2;
    if (n_init < 0 || n_init > N || (n_init > 0 && !C_init)) return ORACLE_ERR_ARG;
    if (n_init > 0 && !is_pow2(n_init)) return ORACLE_ERR_NOT_POW2;

    double *C = (double *)malloc((size_t)N * L * sizeof(double));
    double *Cn = (double *)malloc((size_t)N * L * sizeof(double));
    double *e = (double *)malloc((size_t)M * sizeof(double));
    double *gap = rec_near ? (double *)malloc((size_t)M * sizeof(double)) : NULL;
    int64_t *cnt = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    if (!C || !Cn || !e || !cnt || (rec_near && !gap)) {
        free(C);
        free(Cn);
        free(e);
        free(gap);
        free(cnt);
        return ORACLE_ERR_NOMEM;
    }
    int status = ORACLE_OK;
    int32_t n = 1, total = 0;
    double D = 0.0;
    if (n_init > 0) {
        n = n_init;
        memcpy(C, C_init, (size_t)n * L * sizeof(double));
    } else {
        oracle_mean(X, M, L, C);
    }
    for (;;) {
        double D_prev = INFINITY;
        for (int32_t pass = 0;; ++pass) {
            oracle_assign(X, M, L, C, n, a_out, e, gap, nthreads);
            D = oracle_sum(e, M);
            if (rec_count && total < rec_cap) {
                if (rec_n) rec_n[total] = n;
                if (rec_pass) rec_pass[total] = pass;
                if (rec_D) rec_D[total] = D;
                if (rec_near) {
                    int32_t near = 0;
                    for (int64_t m = 0; m < M; ++m) near += gap[m] <= near_tol;
                    rec_near[total] = near;
                }
            }
            ++total;
            int done = (D == 0.0) || ((D_prev - D) / D <= theta);
            if (done) break;
            if (pass + 1 >= max_passes) {
                status = ORACLE_WARN_MAXPASS;
                break;
            }
            oracle_update(X, M, L, a_out, n, C, Cn, cnt);
            if (reseed) oracle_reseed(Cn, cnt, n, L, delta);
            memcpy(C, Cn, (size_t)n * L * sizeof(double));
            D_prev = D;
        }
        if (n == N) break;
        oracle_split_mode(C, n, L, delta, split_mult, Cn);
        n *= 2;
        memcpy(C, Cn, (size_t)n * L * sizeof(double));
    }
    memcpy(C_out, C, (size_t)N * L * sizeof(double));
    *D_out = D;
    if (rec_count) *rec_count = total;
    free(C);
    free(Cn);
    free(e);
    free(gap);
    free(cnt);
    return status;
}
