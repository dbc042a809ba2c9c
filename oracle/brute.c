/*
 * Brute-force FP64 evaluation of restricted U- and V-statistics by enumerating
 * index tuples.  TEST INFRASTRUCTURE ONLY: loaded by the oracle's Python side;
 * the CUDA library never links or calls it.
 *
 * Definitions followed (arXiv 2508.12627):
 *   - V-set V(n, pi) and restricted V-statistic V_pi (Section 3.3, Definitions
 *     "V-Set" and "Restricted V-Statistic"): the sum of h over tuples that are
 *     constant on every block of pi.
 *   - U-set U(n, pi) and restricted U-statistic U_pi (Appendix E, Definitions
 *     "U-Set" and "Restricted U-Statistic"): the sum of h over tuples whose
 *     equality pattern is exactly pi.  U_pi of the finest partition is the
 *     U-statistic of Section 2.1.
 *   - h(x) = prod_k T_k(alpha[A_k]) (Section 3.1, Definition "Multiplicative
 *     Decomposition"), with every T_k already tensorized (Algorithm 1).
 *
 * Signature tuples have length 1 or 2; tensor k is a length-n vector or an
 * n x n row-major matrix.  Sums are accumulated per thread with Neumaier
 * compensation and then added in thread order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double s, c;
} nsum;

static inline void nadd(nsum *a, double x) {
    double t = a->s + x;
    if ((a->s >= 0 ? a->s : -a->s) >= (x >= 0 ? x : -x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

/* h(alpha) for one tuple. */
static inline double kernel_value(int K, const int *arity, const int *idx0, const int *idx1,
                                  const double *const *T, int64_t n, const int64_t *alpha) {
    double h = 1.0;
    for (int k = 0; k < K; ++k) {
        if (arity[k] == 1)
            h *= T[k][alpha[idx0[k]]];
        else
            h *= T[k][alpha[idx0[k]] * n + alpha[idx1[k]]];
    }
    return h;
}

/*
 * All restricted U-statistics U_pi at once: every alpha in [n]^m is visited,
 * its equality pattern is written as a restricted growth string, and h(alpha)
 * is added to that pattern's slot.  rgs_code_to_index maps the base-m code
 * sum_i rgs[i] * m^i of a restricted growth string to its output slot.
 * Returns 0, or -1 on bad arguments.
 */
int oracle_brute_u_patterns(int64_t n, int m, int K, const int *arity, const int *idx0,
                            const int *idx1, const double *const *T,
                            const int *rgs_code_to_index, int n_parts, double *U_out) {
    if (n <= 0 || m <= 0 || m > 8 || K <= 0) return -1;
    int64_t total = 1;
    for (int i = 0; i < m; ++i) total *= n;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    nsum *acc = (nsum *)calloc((size_t)nthreads * n_parts, sizeof(nsum));
    if (!acc) return -1;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        nsum *mine = acc + (size_t)tid * n_parts;
        int64_t alpha[8];
        int lab[8];
#pragma omp for schedule(static)
        for (int64_t t = 0; t < total; ++t) {
            int64_t r = t;
            for (int i = m - 1; i >= 0; --i) {
                alpha[i] = r % n;
                r /= n;
            }
            /* equality pattern: label = first position holding the same value */
            int next = 0;
            int code = 0, base = 1;
            for (int i = 0; i < m; ++i) {
                int l = -1;
                for (int j = 0; j < i; ++j)
                    if (alpha[j] == alpha[i]) {
                        l = lab[j];
                        break;
                    }
                if (l < 0) l = next++;
                lab[i] = l;
                code += l * base;
                base *= m;
            }
            int slot = rgs_code_to_index[code];
            if (slot >= 0 && slot < n_parts)
                nadd(&mine[slot], kernel_value(K, arity, idx0, idx1, T, n, alpha));
        }
    }
    for (int p = 0; p < n_parts; ++p) {
        nsum tot = {0.0, 0.0};
        for (int t = 0; t < nthreads; ++t) {
            nadd(&tot, acc[(size_t)t * n_parts + p].s);
            nadd(&tot, acc[(size_t)t * n_parts + p].c);
        }
        U_out[p] = tot.s + tot.c;
    }
    free(acc);
    return 0;
}

/*
 * V_pi for one partition, straight from the V-set: enumerate beta in [n]^k
 * (k = number of blocks) and set alpha_i = beta[rgs[i]].
 */
int oracle_brute_v(int64_t n, int m, int K, const int *arity, const int *idx0, const int *idx1,
                   const double *const *T, const int *rgs, double *V_out) {
    if (n <= 0 || m <= 0 || m > 8 || K <= 0) return -1;
    int k = 0;
    for (int i = 0; i < m; ++i)
        if (rgs[i] + 1 > k) k = rgs[i] + 1;
    int64_t total = 1;
    for (int i = 0; i < k; ++i) total *= n;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    nsum *acc = (nsum *)calloc((size_t)nthreads, sizeof(nsum));
    if (!acc) return -1;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int64_t beta[8], alpha[8];
#pragma omp for schedule(static)
        for (int64_t t = 0; t < total; ++t) {
            int64_t r = t;
            for (int j = k - 1; j >= 0; --j) {
                beta[j] = r % n;
                r /= n;
            }
            for (int i = 0; i < m; ++i) alpha[i] = beta[rgs[i]];
            nadd(&acc[tid], kernel_value(K, arity, idx0, idx1, T, n, alpha));
        }
    }
    nsum tot = {0.0, 0.0};
    for (int t = 0; t < nthreads; ++t) {
        nadd(&tot, acc[t].s);
        nadd(&tot, acc[t].c);
    }
    *V_out = tot.s + tot.c;
    free(acc);
    return 0;
}
