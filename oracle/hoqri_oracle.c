/*
 * HOQRI oracle: a plain, slow, FP64 CPU statement of what the HOQRI hot path
 * computes (Sun, Bhat, Wang, Huang, "HOQRI", arXiv 2510.16930).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may load or call this library.  It shares no
 * code, header, table or helper with the CUDA library; the product path never
 * reaches it.
 *
 * Conventions (the paper's Sec. 2 notation):
 *   - X is an N-way sparse tensor given as COO: idx[m][z] is the 0-based mode-m
 *     index of stored entry z, vals[z] its value.  Repeated coordinates are
 *     summed (they denote one entry of X).
 *   - U[m] is I_m x K_m, row-major (U[m][i*K_m + k]).
 *   - G is K_1 x ... x K_N, row-major with the LAST index fastest, so that the
 *     columns of the unfolding G_(n) follow the Kronecker order
 *     B^(1) (x) ... (x) B^(N) of Eq. (2) (mode 1 slowest).
 *   - A_n is I_n x K_n, row-major.
 * All arithmetic is IEEE double.  OpenMP, when present, only splits
 * independent outputs (entries of G, rows of A); every output is summed in the
 * same order whatever the thread count, so results do not depend on it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXN 8

int hoqri_oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void hoqri_oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ---------------------------------------------------------------- coalescing */

static int g_cmp_N;
static const int32_t *const *g_cmp_idx;

static int cmp_coord(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    for (int m = 0; m < g_cmp_N; ++m) {
        int32_t x = g_cmp_idx[m][a], y = g_cmp_idx[m][b];
        if (x != y) return x < y ? -1 : 1;
    }
    return a < b ? -1 : (a > b ? 1 : 0); /* input position breaks ties */
}

/*
 * Sum repeated coordinates (Table 1: I(X) is a SET of nonzero positions, so a
 * coordinate listed twice is one entry whose value is the sum).  Output is in
 * lexicographic order of (i_1, ..., i_N); repeats are added in input order.
 * out_idx[m] and out_vals must hold nnz entries.  Returns the number of
 * distinct coordinates.  Not thread-safe (uses a static comparator context).
 */
int64_t hoqri_oracle_coalesce(int N, int64_t nnz, const int32_t *const *idx, const double *vals,
                              int32_t *const *out_idx, double *out_vals) {
    if (nnz <= 0) return 0;
    int64_t *perm = (int64_t *)malloc((size_t)nnz * sizeof(int64_t));
    for (int64_t z = 0; z < nnz; ++z) perm[z] = z;
    g_cmp_N = N;
    g_cmp_idx = idx;
    qsort(perm, (size_t)nnz, sizeof(int64_t), cmp_coord);
    int64_t u = -1;
    for (int64_t s = 0; s < nnz; ++s) {
        int64_t z = perm[s];
        int same = (u >= 0);
        for (int m = 0; same && m < N; ++m) same = (out_idx[m][u] == idx[m][z]);
        if (same) {
            out_vals[u] += vals[z];
        } else {
            ++u;
            for (int m = 0; m < N; ++m) out_idx[m][u] = idx[m][z];
            out_vals[u] = vals[z];
        }
    }
    free(perm);
    return u + 1;
}

/* ||X||^2 over distinct entries (pass coalesced values). */
double hoqri_oracle_norm2(int64_t n, const double *v) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += v[i] * v[i];
    return s;
}

/* -------------------------------------------------------------- index helpers */

static int64_t prod_ranks(int N, const int32_t *ranks) {
    int64_t p = 1;
    for (int m = 0; m < N; ++m) p *= ranks[m];
    return p;
}

/* row-major strides of G (last index fastest) */
static void core_strides(int N, const int32_t *ranks, int64_t *st) {
    st[N - 1] = 1;
    for (int m = N - 2; m >= 0; --m) st[m] = st[m + 1] * ranks[m + 1];
}

/* ------------------------------------------------------------------ the core */

/*
 * G = X x_1 U_1^T x_2 ... x_N U_N^T  (Sec. 2.2, optimal core; Alg. 2 last step;
 * Alg. 3 first step), written out entry by entry:
 *   G(k_1..k_N) = sum over stored entries z of  x_z * prod_m U_m(i_m(z), k_m).
 */
void hoqri_oracle_core(int N, const int32_t *ranks, int64_t nnz, const int32_t *const *idx,
                       const double *vals, const double *const *U, double *G) {
    int64_t P = prod_ranks(N, ranks);
    int64_t st[MAXN];
    core_strides(N, ranks, st);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
        int k[MAXN];
        for (int m = 0; m < N; ++m) k[m] = (int)((p / st[m]) % ranks[m]);
        double acc = 0.0;
        for (int64_t z = 0; z < nnz; ++z) {
            double t = vals[z];
            for (int m = 0; m < N; ++m) t *= U[m][(int64_t)idx[m][z] * ranks[m] + k[m]];
            acc += t;
        }
        G[p] = acc;
    }
}

/* Selected entries of G (linear row-major positions lin[s]); same sum as above. */
void hoqri_oracle_core_entries(int N, const int32_t *ranks, int64_t nnz, const int32_t *const *idx,
                               const double *vals, const double *const *U, int64_t ns,
                               const int64_t *lin, double *out) {
    int64_t st[MAXN];
    core_strides(N, ranks, st);
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < ns; ++s) {
        int k[MAXN];
        for (int m = 0; m < N; ++m) k[m] = (int)((lin[s] / st[m]) % ranks[m]);
        double acc = 0.0;
        for (int64_t z = 0; z < nnz; ++z) {
            double t = vals[z];
            for (int m = 0; m < N; ++m) t *= U[m][(int64_t)idx[m][z] * ranks[m] + k[m]];
            acc += t;
        }
        out[s] = acc;
    }
}

/* ------------------------------------------------------ TTMcTC, element-wise */

/* I^(n)_{i}: stored entries whose mode-n index is i, in input order
 * (Table 1).  Returns CSR-style start[I_n+1] and the entry list. */
static void mode_index_sets(int64_t In, int64_t nnz, const int32_t *in_idx, int64_t **start_out,
                            int64_t **list_out) {
    int64_t *start = (int64_t *)calloc((size_t)In + 1, sizeof(int64_t));
    int64_t *list = (int64_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    for (int64_t z = 0; z < nnz; ++z) start[in_idx[z] + 1]++;
    for (int64_t i = 0; i < In; ++i) start[i + 1] += start[i];
    int64_t *fill = (int64_t *)malloc((size_t)(In + 1) * sizeof(int64_t));
    memcpy(fill, start, (size_t)(In + 1) * sizeof(int64_t));
    for (int64_t z = 0; z < nnz; ++z) list[fill[in_idx[z]]++] = z;
    free(fill);
    *start_out = start;
    *list_out = list;
}

/*
 * A_n(i_n, k_n) for the rows listed in rows[0..nr) given the core G (Alg. 3
 * inner loops; Eq. (ttmctc) A_n = Y_(n) G_(n)^T with Y = X x_{-n} {U^T}):
 *   A_n(i_n,k_n) = sum_{z in I^(n)_{i_n}} sum_{k_{-n}} x_z G(k) prod_{v != n} U_v(i_v(z), k_v).
 * out is nr x K_n.
 */
static void ttmctc_rows_given_core(int N, const int32_t *ranks, int64_t nnz, const int32_t *const *idx,
                                   const double *vals, const double *const *U, int n, const double *G,
                                   const int64_t *start, const int64_t *list, int64_t nr,
                                   const int32_t *rows, double *out) {
    int64_t st[MAXN];
    core_strides(N, ranks, st);
    int64_t Pm = prod_ranks(N, ranks) / ranks[n]; /* number of k_{-n} */
    (void)nnz;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nr; ++r) {
        int64_t i = rows[r];
        for (int kn = 0; kn < ranks[n]; ++kn) {
            double acc = 0.0;
            for (int64_t e = start[i]; e < start[i + 1]; ++e) {
                int64_t z = list[e];
                int k[MAXN];
                for (int m = 0; m < N; ++m) k[m] = 0;
                for (int64_t q = 0; q < Pm; ++q) {
                    int64_t g = (int64_t)kn * st[n];
                    double t = vals[z];
                    for (int m = 0; m < N; ++m) {
                        if (m == n) continue;
                        g += (int64_t)k[m] * st[m];
                        t *= U[m][(int64_t)idx[m][z] * ranks[m] + k[m]];
                    }
                    acc += t * G[g];
                    /* odometer over k_{-n}, last mode fastest */
                    for (int m = N - 1; m >= 0; --m) {
                        if (m == n) continue;
                        if (++k[m] < ranks[m]) break;
                        k[m] = 0;
                    }
                }
            }
            out[r * ranks[n] + kn] = acc;
        }
    }
}

/*
 * TTMcTC(X, {U}, n), element-wise (Alg. 3): first G <- X x {U^T}, then every
 * A_n(i_n, k_n).  A is I_n x K_n; G_out (optional, P entries) receives the core
 * that was used.
 */
void hoqri_oracle_ttmctc(int N, const int64_t *dims, const int32_t *ranks, int64_t nnz,
                         const int32_t *const *idx, const double *vals, const double *const *U, int n,
                         double *A, double *G_out) {
    int64_t P = prod_ranks(N, ranks);
    double *G = G_out ? G_out : (double *)malloc((size_t)P * sizeof(double));
    hoqri_oracle_core(N, ranks, nnz, idx, vals, U, G);
    int64_t *start, *list;
    mode_index_sets(dims[n], nnz, idx[n], &start, &list);
    int32_t *rows = (int32_t *)malloc((size_t)dims[n] * sizeof(int32_t));
    for (int64_t i = 0; i < dims[n]; ++i) rows[i] = (int32_t)i;
    ttmctc_rows_given_core(N, ranks, nnz, idx, vals, U, n, G, start, list, dims[n], rows, A);
    free(rows);
    free(start);
    free(list);
    if (!G_out) free(G);
}

/* Selected rows of A_n (Alg. 3 restricted to i_n in rows[]), with G computed
 * here from X and U (G_out optional).  out is nr x K_n. */
void hoqri_oracle_ttmctc_rows(int N, const int64_t *dims, const int32_t *ranks, int64_t nnz,
                              const int32_t *const *idx, const double *vals, const double *const *U,
                              int n, int64_t nr, const int32_t *rows, double *out, double *G_out) {
    int64_t P = prod_ranks(N, ranks);
    double *G = G_out ? G_out : (double *)malloc((size_t)P * sizeof(double));
    hoqri_oracle_core(N, ranks, nnz, idx, vals, U, G);
    int64_t *start, *list;
    mode_index_sets(dims[n], nnz, idx[n], &start, &list);
    ttmctc_rows_given_core(N, ranks, nnz, idx, vals, U, n, G, start, list, nr, rows, out);
    free(start);
    free(list);
    if (!G_out) free(G);
}

/* Selected rows of A_n (Alg. 3 restricted to i_n in rows[]) with a core G
 * supplied by the caller (P entries, the layout above) instead of computed
 * here: the element-wise TTMcTC step of Alg. 3 alone.  out is nr x K_n. */
void hoqri_oracle_ttmctc_rows_with_core(int N, const int64_t *dims, const int32_t *ranks, int64_t nnz,
                                        const int32_t *const *idx, const double *vals,
                                        const double *const *U, int n, const double *G, int64_t nr,
                                        const int32_t *rows, double *out) {
    int64_t *start, *list;
    mode_index_sets(dims[n], nnz, idx[n], &start, &list);
    ttmctc_rows_given_core(N, ranks, nnz, idx, vals, U, n, G, start, list, nr, rows, out);
    free(start);
    free(list);
}

/* ----------------------------------------------------- TTMcTC, matrix version */

/*
 * TTMcTC, matrix version (Alg. 4): A_n = sum over k_{-n} of y y^T U_n with
 * y = X x_{-n} {u_{k_v}}, the sparse mode product of X with the columns
 * U_v(:, k_v), v != n.  Independent of Alg. 3 (it never forms G).
 */
void hoqri_oracle_ttmctc_matrix(int N, const int64_t *dims, const int32_t *ranks, int64_t nnz,
                                const int32_t *const *idx, const double *vals, const double *const *U,
                                int n, double *A) {
    int64_t In = dims[n];
    int Kn = ranks[n];
    int64_t Pm = prod_ranks(N, ranks) / Kn;
    double *y = (double *)malloc((size_t)In * sizeof(double));
    double *w = (double *)malloc((size_t)Kn * sizeof(double));
    memset(A, 0, (size_t)In * Kn * sizeof(double));
    int k[MAXN];
    for (int m = 0; m < N; ++m) k[m] = 0;
    for (int64_t q = 0; q < Pm; ++q) {
        memset(y, 0, (size_t)In * sizeof(double));
        for (int64_t z = 0; z < nnz; ++z) {
            double t = vals[z];
            for (int m = 0; m < N; ++m)
                if (m != n) t *= U[m][(int64_t)idx[m][z] * ranks[m] + k[m]];
            y[idx[n][z]] += t;
        }
        for (int c = 0; c < Kn; ++c) {
            double s = 0.0;
            for (int64_t i = 0; i < In; ++i) s += y[i] * U[n][i * Kn + c];
            w[c] = s;
        }
        for (int64_t i = 0; i < In; ++i)
            for (int c = 0; c < Kn; ++c) A[i * Kn + c] += y[i] * w[c];
        for (int m = N - 1; m >= 0; --m) {
            if (m == n) continue;
            if (++k[m] < ranks[m]) break;
            k[m] = 0;
        }
    }
    free(y);
    free(w);
}

/* ------------------------------------------------------------------------- QR */

/*
 * Thin QR of the I x K matrix A (I >= K) by Householder reflections (the "QR"
 * of Alg. 2: an orthonormal basis of the columns of A).  Q is I x K with
 * orthonormal columns, R is K x K upper triangular; columns are signed so that
 * diag(R) >= 0, which makes (Q, R) unique when A has full column rank.  A zero
 * pivot column gets no reflection, and the accumulated reflectors still give a
 * K-column orthonormal Q.  Returns the number of zero pivots.
 */
int hoqri_oracle_qr(int64_t I, int K, const double *A, double *Q, double *R) {
    double *W = (double *)malloc((size_t)I * K * sizeof(double));
    double *V = (double *)calloc((size_t)I * K, sizeof(double)); /* reflector j in column j */
    double *beta = (double *)calloc((size_t)K, sizeof(double));
    memcpy(W, A, (size_t)I * K * sizeof(double));
    int zero = 0;
    double *Rl = R ? R : (double *)malloc((size_t)K * K * sizeof(double));
    memset(Rl, 0, (size_t)K * K * sizeof(double));
    for (int j = 0; j < K; ++j) {
        double nrm2 = 0.0;
        for (int64_t i = j; i < I; ++i) nrm2 += W[i * K + j] * W[i * K + j];
        double nrm = sqrt(nrm2);
        if (nrm == 0.0) {
            ++zero;
            beta[j] = 0.0;
        } else {
            double alpha = W[(int64_t)j * K + j] > 0 ? -nrm : nrm;
            double vn2 = 0.0;
            for (int64_t i = j; i < I; ++i) {
                double v = W[i * K + j] - (i == j ? alpha : 0.0);
                V[i * K + j] = v;
                vn2 += v * v;
            }
            beta[j] = vn2 > 0 ? 2.0 / vn2 : 0.0;
            for (int c = j; c < K; ++c) {
                double s = 0.0;
                for (int64_t i = j; i < I; ++i) s += V[i * K + j] * W[i * K + c];
                s *= beta[j];
                for (int64_t i = j; i < I; ++i) W[i * K + c] -= s * V[i * K + j];
            }
        }
        for (int c = j; c < K; ++c) Rl[j * K + c] = W[(int64_t)j * K + c];
    }
    /* Q = H_0 H_1 ... H_{K-1} [I_K; 0] */
    memset(Q, 0, (size_t)I * K * sizeof(double));
    for (int j = 0; j < K; ++j) Q[(int64_t)j * K + j] = 1.0;
    for (int j = K - 1; j >= 0; --j) {
        if (beta[j] == 0.0) continue;
        for (int c = 0; c < K; ++c) {
            double s = 0.0;
            for (int64_t i = j; i < I; ++i) s += V[i * K + j] * Q[i * K + c];
            s *= beta[j];
            for (int64_t i = j; i < I; ++i) Q[i * K + c] -= s * V[i * K + j];
        }
    }
    for (int j = 0; j < K; ++j) {
        if (Rl[j * K + j] < 0) {
            for (int64_t i = 0; i < I; ++i) Q[i * K + j] = -Q[i * K + j];
            for (int c = j; c < K; ++c) Rl[j * K + c] = -Rl[j * K + c];
        }
    }
    if (!R) free(Rl);
    free(W);
    free(V);
    free(beta);
    return zero;
}

/* -------------------------------------------------------------------- HOQRI */

/*
 * HOQRI (Alg. 2): U holds the initial factors on entry (overwritten with the
 * final ones).  Each of `iters` iterations is one sweep n = 1..N of
 *   A_n <- TTMcTC(X, {U}, n)   (Alg. 3, which recomputes G with the current U)
 *   U_n <- Q of the Householder QR of A_n.
 * After the loop G <- X x {U^T} (G_out, optional).  The input stream may repeat
 * coordinates; it is coalesced first.  Outputs (all optional):
 *   resid[t]      = sqrt(max(0, ||X||^2 - ||G_t||^2)) / ||X||, G_t the core
 *                   after sweep t (the relative error of prob. (tucker) for
 *                   orthonormal U and optimal G, Sec. 2.2);
 *   fblock[t*N+n] = ||G||^2 of the core Alg. 3 computed at the start of block
 *                   (t, n), i.e. the objective f of prob. (main) just before
 *                   that block update (Thm. 1: non-decreasing).
 * Returns the total number of zero QR pivots met.
 */
int hoqri_oracle_hoqri(int N, const int64_t *dims, const int32_t *ranks, int64_t nnz_raw,
                       const int32_t *const *idx_raw, const double *vals_raw, double *const *U,
                       int iters, double *G_out, double *resid, double *fblock) {
    int32_t *cidx[MAXN];
    for (int m = 0; m < N; ++m) cidx[m] = (int32_t *)malloc((size_t)(nnz_raw > 0 ? nnz_raw : 1) * sizeof(int32_t));
    double *cval = (double *)malloc((size_t)(nnz_raw > 0 ? nnz_raw : 1) * sizeof(double));
    int64_t nnz = hoqri_oracle_coalesce(N, nnz_raw, idx_raw, vals_raw, cidx, cval);
    double nx2 = hoqri_oracle_norm2(nnz, cval);
    int64_t P = prod_ranks(N, ranks);
    double *G = (double *)malloc((size_t)P * sizeof(double));
    int64_t maxI = 0;
    for (int m = 0; m < N; ++m) maxI = dims[m] > maxI ? dims[m] : maxI;
    int maxK = 0;
    for (int m = 0; m < N; ++m) maxK = ranks[m] > maxK ? ranks[m] : maxK;
    double *A = (double *)malloc((size_t)maxI * maxK * sizeof(double));
    int zero = 0;
    for (int t = 0; t < iters; ++t) {
        for (int n = 0; n < N; ++n) {
            hoqri_oracle_ttmctc(N, dims, ranks, nnz, (const int32_t *const *)cidx, cval,
                                (const double *const *)U, n, A, G);
            if (fblock) {
                double g2 = 0.0;
                for (int64_t p = 0; p < P; ++p) g2 += G[p] * G[p];
                fblock[t * N + n] = g2;
            }
            zero += hoqri_oracle_qr(dims[n], ranks[n], A, U[n], NULL);
        }
        if (resid || (t == iters - 1 && G_out)) {
            hoqri_oracle_core(N, ranks, nnz, (const int32_t *const *)cidx, cval, (const double *const *)U, G);
            if (resid) {
                double g2 = 0.0;
                for (int64_t p = 0; p < P; ++p) g2 += G[p] * G[p];
                double r2 = nx2 - g2;
                resid[t] = nx2 > 0 ? sqrt(r2 > 0 ? r2 : 0.0) / sqrt(nx2) : 0.0;
            }
        }
    }
    if (G_out) {
        if (iters == 0)
            hoqri_oracle_core(N, ranks, nnz, (const int32_t *const *)cidx, cval, (const double *const *)U, G);
        memcpy(G_out, G, (size_t)P * sizeof(double));
    }
    for (int m = 0; m < N; ++m) free(cidx[m]);
    free(cval);
    free(G);
    free(A);
    return zero;
}
