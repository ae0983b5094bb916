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
#include <stdlib.h>

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

/*
 * K-PID asynchronous D-iteration (Secs. 2.3-2.6), emulated sequentially.
 *
 * The nodes are split into K ranges Omega_k = [bounds[k], bounds[k+1]) (a
 * uniform or cost-balanced partition, Sec. 2.3), each owned by one PID with
 * its own threshold T_k.  Readings where the paper is silent (each is listed
 * in the design notes):
 *   - the PIDs run in lock-step rounds; in a round every PID makes one cyclic
 *     threshold sweep over its own nodes (the time-stepped model of Sec. 2.4
 *     with equal speeds, at the granularity of one sweep);
 *   - a sweep diffuses a node to its children inside Omega_k only (the
 *     algorithm (*) of Sec. 2.5); the fluid owed to external children is
 *     carried implicitly by the increment H - H_old since the PID's last
 *     transmission;
 *   - after the sweeps, PID k transmits when s_k > r_k / K (Eq. send), with
 *     r_k = sum of |F_i| over Omega_k and s_k = sum over the external edges
 *     j <- i of |p_ji (H_i - H_old_i)|: it adds p_ji (H_i - H_old_i) to F_j
 *     for every external child j and sets H_old = H on Omega_k.  Every PID
 *     decides on the state after the sweeps, then all transmissions land;
 *   - reception (Sec. 2.6): a PID that received fluid rescales its threshold
 *     by (r_k + received) / r_k when r_k > 0 (the printed factor
 *     min((r_k + received) / r_k, received) is garbled; its first term is
 *     taken), and sets T_k = received when r_k = 0, as the paper states; the
 *     empty-sweep rule below then lowers a T_k above every |F_i| of the range;
 *   - T_k starts at max |F_i| over Omega_k and a sweep that would find nothing
 *     is skipped by dividing T_k by alpha first (as in the one-PID oracle); a
 *     PID without fluid idles;
 *   - the stop test is the exact residual |B + P H - H|_1 <= tol after each
 *     round: it includes the fluid still waiting for transmission;
 *   - with dangling != 0 (the 1/N completion of Sec. 2.2) the column of a
 *     node without out-edges is d/N in every row: its part in the PID's own
 *     range is local (added to every node of Omega_k when the node diffuses)
 *     and the rest is owed to the other ranges like any external edge
 *     (counted in s_k, transmitted from H - H_old to every node outside
 *     Omega_k).
 * Costs (Sec. 2.4): ops[k] counts PID k's elementary diffusions, one per local
 * child in its sweeps and one per external edge it transmits (a completed
 * column has n_k local and N - n_k external children).
 * Returns 0 on convergence, 4 when max_rounds was reached, 1 on invalid
 * arguments, 2 when a scratch allocation failed.
 */
int oracle_kpid(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *B, double d,
                double tol, double alpha, int K, const int64_t *bounds, int64_t max_rounds,
                double *H, double *F, double *H_old, int64_t *ops, int64_t *sends,
                int64_t *rounds_out, double *resid_out, double *trace, int64_t trace_cap, double *T_out,
                int dangling) {
    if (n < 0 || K < 1 || !(alpha > 1.0) || !(tol >= 0.0) || max_rounds < 0) return 1;
    if (bounds[0] != 0 || bounds[K] != n) return 1;
    for (int k = 0; k < K; ++k)
        if (bounds[k + 1] < bounds[k]) return 1;
    int32_t *part = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    double *scratch = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *T = (double *)malloc((size_t)K * sizeof(double));
    double *r = (double *)malloc((size_t)K * sizeof(double));
    double *s = (double *)malloc((size_t)K * sizeof(double));
    double *recv = (double *)malloc((size_t)K * sizeof(double));
    int *send = (int *)malloc((size_t)K * sizeof(int));
    if (!part || !scratch || !T || !r || !s || !recv || !send) {
        free(part); free(scratch); free(T); free(r); free(s); free(recv); free(send);
        return 2;
    }
    for (int k = 0; k < K; ++k)
        for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i) part[i] = k;
    for (int64_t i = 0; i < n; ++i) { F[i] = B[i]; H[i] = 0.0; H_old[i] = 0.0; }
    for (int k = 0; k < K; ++k) {
        ops[k] = 0;
        sends[k] = 0;
        T[k] = 0.0;
        for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i)
            if (fabs(F[i]) > T[k]) T[k] = fabs(F[i]);
    }
    int status = 4;
    int64_t round = 0;
    double resid = 0.0;
    for (;;) {
        resid = oracle_residual(n, row_ptr, col, B, d, H, scratch, dangling);
        if (resid <= tol) { status = 0; break; }
        if (round >= max_rounds) { status = 4; break; }
        /* every PID sweeps its own nodes, diffusing to local children only */
        for (int k = 0; k < K; ++k) {
            double mx = 0.0;
            for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i)
                if (fabs(F[i]) > mx) mx = fabs(F[i]);
            if (mx == 0.0) continue;                    /* idle */
            while (T[k] > mx) T[k] /= alpha;
            for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i) {
                double sent = F[i];
                if (fabs(sent) < T[k] || sent == 0.0) continue;
                F[i] = 0.0;
                H[i] += sent;
                int64_t deg = row_ptr[i + 1] - row_ptr[i];
                if (deg == 0) {
                    if (dangling) {                     /* the completed column's local part */
                        for (int64_t c = bounds[k]; c < bounds[k + 1]; ++c) F[c] += sent * (d / (double)n);
                        ops[k] += bounds[k + 1] - bounds[k];
                    }
                    continue;
                }
                double p = d / (double)deg;
                for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                    if (part[col[e]] != k) continue;    /* external: left in H - H_old */
                    F[col[e]] += sent * p;
                    ops[k] += 1;
                }
            }
            T[k] /= alpha;
        }
        /* transmissions: decided on the state after the sweeps (Eq. send) */
        for (int k = 0; k < K; ++k) {
            r[k] = 0.0;
            s[k] = 0.0;
            recv[k] = 0.0;
            for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i) {
                r[k] += fabs(F[i]);
                double dh = H[i] - H_old[i];
                int64_t deg = row_ptr[i + 1] - row_ptr[i];
                if (dh != 0.0 && deg == 0 && dangling)  /* completed column: N - n_k external rows */
                    s[k] += fabs(d / (double)n * dh) * (double)(n - (bounds[k + 1] - bounds[k]));
                if (dh == 0.0 || deg == 0) continue;
                double p = d / (double)deg;
                for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
                    if (part[col[e]] != k) s[k] += fabs(p * dh);
            }
            send[k] = s[k] > 0.0 && s[k] > r[k] / (double)K;
        }
        for (int k = 0; k < K; ++k) {
            if (!send[k]) continue;
            sends[k] += 1;
            for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i) {
                double dh = H[i] - H_old[i];
                int64_t deg = row_ptr[i + 1] - row_ptr[i];
                H_old[i] = H[i];
                if (dh != 0.0 && deg == 0 && dangling) {   /* completed column: every node outside */
                    double q = d / (double)n * dh;
                    for (int64_t j = 0; j < n; ++j) {
                        if (part[j] == k) continue;
                        F[j] += q;
                        recv[part[j]] += fabs(q);
                    }
                    ops[k] += n - (bounds[k + 1] - bounds[k]);
                }
                if (dh == 0.0 || deg == 0) continue;
                double p = d / (double)deg;
                for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                    int32_t j = col[e];
                    if (part[j] == k) continue;
                    F[j] += p * dh;
                    recv[part[j]] += fabs(p * dh);
                    ops[k] += 1;
                }
            }
        }
        /* reception (Sec. 2.6): rescale the threshold of every receiver */
        for (int k = 0; k < K; ++k) {
            if (recv[k] == 0.0) continue;
            if (r[k] > 0.0) T[k] *= (r[k] + recv[k]) / r[k];
            else T[k] = recv[k];
        }
        if (trace && round < trace_cap)
            for (int k = 0; k < K; ++k) {
                double rk = 0.0;
                for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i) rk += fabs(F[i]);
                trace[round * K + k] = rk;
            }
        round += 1;
    }
    *rounds_out = round;
    *resid_out = resid;
    if (T_out)
        for (int k = 0; k < K; ++k) T_out[k] = T[k];
    free(part); free(scratch); free(T); free(r); free(s); free(recv); free(send);
    return status;
}
