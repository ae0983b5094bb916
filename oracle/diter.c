/*
 * diter.c - CPU oracle of the D-iteration (TEST INFRASTRUCTURE ONLY).
 *
 * Plain, sequential, FP64 restatement of the method, written to be checked
 * against the paper by eye.  Only tests, the smoke check and the benchmark's
 * CPU-baseline leg may build, load or call it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Problem (Eq. 1): X = P X + B, with P = d Q (Eq. 2) and q_kj = 1/#out_j for
 * every edge j -> k (Sec. 2.2); a dangling column (no out-edge) stays zero.
 * The graph is a CSR of out-edges: row j lists the targets k of j's edges,
 * i.e. the support of column j of P.  Duplicate entries count with their
 * multiplicity and a self-loop j -> j is an ordinary entry p_jj.
 *
 * Method (Eqs. defF/defH and the pseudo-code of Sec. 2.1): F_0 = B, H_0 = 0;
 * diffusing node i moves F_i into H_i and adds p_ki F_i to F_k for every
 * child k.  Node order (Sec. 2.4): a cyclic scan over i = 0..N-1 diffuses
 * every node with |F_i| >= T, then T <- T / alpha (alpha = 1.5 by default).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - T_0 = max_i |F_i| of the initial fluid;
 *   - "above T" is |F_i| >= T on the raw fluid (not the weighted score);
 *   - one cyclic sweep per threshold level; fluid received earlier in the
 *     same sweep counts when its node is reached (Gauss-Seidel order);
 *   - a level whose sweep would find no node is skipped, i.e. T is divided
 *     by alpha until T <= max|F| (an empty sweep changes nothing);
 *   - stop when the L1 residual r = sum_i |F_i|, summed afresh after each
 *     sweep, is <= tol (the paper's own rule r/(1-d) <= Target_Error is the
 *     same test with tol = (1-d) Target_Error);
 *   - warm start: H_0 given, F_0 = B + P H_0 - H_0 (signed fluid is selected
 *     on |F_i| and r is the L1 norm).
 *
 * Optional dangling completion (Sec. 2.2 notes that the dangling columns of
 * Q may be completed by 1/N, which makes Q stochastic): with dangling != 0,
 * column j of Q for a node without out-edges is the uniform 1/N, so
 * diffusing such a node adds d F_j / N to every node k, itself included.
 *
 * Optional weighted selection (Sec. 2.4 names the ideal order as the argmax of
 * F_i / ((#in_i + 1)(#out_i + 1)) and approximates it by a threshold sweep):
 * with weights w_i the sweep selects |F_i| w_i >= T instead, T_0 and the
 * empty-level rule use max_i |F_i| w_i, and r stays sum_i |F_i|.
 */
#include <stdint.h>
#include <math.h>
#include <stddef.h>

typedef struct {
    int64_t levels;           /* non-empty sweeps performed */
    int64_t node_diffusions;  /* nodes diffused */
    int64_t edge_diffusions;  /* elementary node-to-node diffusions (Sec. 2.4) */
    double resid_l1;          /* sum |F_i| at return */
    double threshold;         /* T at return */
} oracle_stats;

/* F = B + P H - H, column by column (FP64); returns sum |F_i|.  With
 * dangling != 0 a column without out-edges is d/N in every row, so those
 * columns add d/N times the sum of H over the dangling nodes to every row. */
double oracle_residual(int64_t n, const int64_t *row_ptr, const int32_t *col,
                       const double *B, double d, const double *H, double *F, int dangling) {
    double h_dangling = 0.0;
    for (int64_t k = 0; k < n; ++k) F[k] = B[k] - H[k];
    for (int64_t j = 0; j < n; ++j) {
        int64_t deg = row_ptr[j + 1] - row_ptr[j];
        if (deg == 0) {
            h_dangling += H[j];
            continue;
        }
        double p = d / (double)deg;
        for (int64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) F[col[e]] += p * H[j];
    }
    if (dangling)
        for (int64_t k = 0; k < n; ++k) F[k] += d / (double)n * h_dangling;
    double r = 0.0;
    for (int64_t k = 0; k < n; ++k) r += fabs(F[k]);
    return r;
}

/*
 * Runs the D-iteration until sum|F| <= tol or max_levels sweeps.
 * H: in = H_0 when warm != 0, out = history.  F: out = residual fluid.
 * trace (optional, capacity trace_cap): r after each sweep.
 * Returns 0 on convergence, 4 when max_levels was reached first,
 * 1 on invalid arguments.
 */
int oracle_diter(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *B,
                 double d, double tol, double alpha, int64_t max_levels, int warm,
                 double *H, double *F, oracle_stats *st, double *trace, int64_t trace_cap,
                 const double *w, int dangling) {
    if (n < 0 || !(alpha > 1.0) || !(tol >= 0.0) || max_levels < 0) return 1;
    if (warm) {
        oracle_residual(n, row_ptr, col, B, d, H, F, dangling);
    } else {
        for (int64_t i = 0; i < n; ++i) { F[i] = B[i]; H[i] = 0.0; }
    }
    double T = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double score = w ? fabs(F[i]) * w[i] : fabs(F[i]);
        if (score > T) T = score;
    }

    oracle_stats s = {0, 0, 0, 0.0, 0.0};
    int status = 4;
    for (;;) {
        double r = 0.0, mx = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double a = fabs(F[i]);
            r += a;
            double score = w ? a * w[i] : a;
            if (score > mx) mx = score;
        }
        s.resid_l1 = r;
        if (r <= tol) { status = 0; break; }
        if (s.levels >= max_levels) { status = 4; break; }
        while (T > mx) T /= alpha;          /* skip sweeps that would be empty */

        for (int64_t i = 0; i < n; ++i) {  /* one cyclic sweep at threshold T */
            double sent = F[i];
            double score = w ? fabs(sent) * w[i] : fabs(sent);
            if (score < T || sent == 0.0) continue;
            H[i] += sent;
            F[i] = 0.0;
            int64_t deg = row_ptr[i + 1] - row_ptr[i];
            s.node_diffusions += 1;
            if (deg == 0) {
                if (dangling)                   /* the uniform column: d/N to every node */
                    for (int64_t k = 0; k < n; ++k) F[k] += sent * (d / (double)n);
                continue;
            }
            double p = d / (double)deg;     /* p_ki, the same for every child k */
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) F[col[e]] += sent * p;
            s.edge_diffusions += deg;
        }
        if (trace && s.levels < trace_cap) {
            double rr = 0.0;
            for (int64_t i = 0; i < n; ++i) rr += fabs(F[i]);
            trace[s.levels] = rr;
        }
        s.levels += 1;
        T /= alpha;
    }
    s.threshold = T;
    if (st) *st = s;
    return status;
}
