/*
 * kpid_sim.c - time-stepped simulation of K asynchronous PIDs running the
 * D-iteration, as the paper evaluates its distributed scheme (Secs. 2.3-2.6
 * for the scheme, Sec. 2.4 "PID modelling" and Sec. 3 for the model).
 *
 * The nodes are split into K ranges Omega_k = [bounds[k], bounds[k+1]) (the
 * uniform or the cost-balanced partition of Sec. 2.3), each owned by one PID.
 * Time advances in steps; in every step each PID can spend PID_Speed_k
 * elementary operations (one operation = one node-to-node diffusion,
 * Sec. 2.4; the default speed is L / K).  A PID works through cyclic
 * threshold sweeps over its own nodes (Sec. 2.4): a sweep visits the nodes of
 * Omega_k in order and diffuses every node with |F_i| >= T_k to its children
 * inside Omega_k only (algorithm (*) of Sec. 2.5), then T_k <- T_k / alpha.
 * A sweep may span several steps (the PID resumes where its budget ran out);
 * a node's diffusion is never split (the budget may go below zero and the
 * debt is paid from the next step).  Before a sweep starts, T_k is lowered to
 * the first T_k / alpha^j <= max |F_i| over Omega_k (an empty sweep changes
 * nothing).  A PID whose residual r_k = sum |F_i| over Omega_k is at most
 * sleep_tol sleeps (Sec. 2.4: it goes to sleep once r_k is below its
 * target); the budget of a step it spends asleep, or leaves unused because a
 * sweep limit was reached, is idle capacity (Sec. 3).
 *
 * At the end of every step each PID evaluates r_k and the fluid it owes to
 * other ranges, s_k = sum over its external edges i -> j of
 * |p_ji (H_i - H_old_i)| (the H-increment form of Sec. 2.5), and transmits
 * P (H - H_old) restricted to external children when s_k > r_k / K
 * (Eq. send); one operation is charged per external edge, and H_old = H on
 * Omega_k.  A transmission is tested once per step (every PID_Speed
 * operations) and held back with probability Delay_Proba at each test, so its
 * delay is geometric with mean PID_Speed * Delay_Proba / (1 - Delay_Proba)
 * operations (Sec. 3).  On delivery the receiver adds the fluid and rescales
 * its threshold (Sec. 2.6): T_k <- T_k (r_k + received) / r_k, or
 * T_k <- received when r_k = 0.  The run stops when the exact residual
 * |B + P H - H|_1, which counts the fluid still owed or in transit, is at
 * most tol (checked at the start of every step).
 *
 * With an unbounded speed, one sweep per step, no delay and sleep_tol = 0 a
 * step is exactly one lock-step round of the sequential emulation of the
 * scheme; the tests pin that case against the CPU oracle bit for bit.
 *
 * This file shares no code with the oracle or with the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Counter-based uniform in [0, 1): SplitMix64 of (seed, message, test). */
static double ks_uniform(uint64_t seed, uint64_t msg, uint64_t test) {
    uint64_t z = seed ^ (msg * 0x9E3779B97F4A7C15ull) ^ (test * 0xD1B54A32D192ED03ull);
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* Exported for the delay-model test: the number of steps a transmission waits. */
int64_t ks_delay_steps(double delay_proba, uint64_t seed, uint64_t msg) {
    int64_t t = 0;
    while (ks_uniform(seed, msg, (uint64_t)t) < delay_proba) ++t;
    return t;
}

typedef struct {
    int64_t first, count;   /* entries in the pool */
    int64_t id;             /* message number (RNG stream) */
    int64_t tests;          /* tests already failed */
} ks_msg;

typedef struct {
    int32_t *node;
    double *amt;
    int64_t size, cap;
} ks_pool;

static int pool_reserve(ks_pool *p, int64_t extra) {
    if (p->size + extra <= p->cap) return 0;
    int64_t cap = p->cap ? p->cap : 1024;
    while (cap < p->size + extra) cap *= 2;
    int32_t *nn = (int32_t *)realloc(p->node, (size_t)cap * sizeof(int32_t));
    if (!nn) return 1;
    p->node = nn;
    double *na = (double *)realloc(p->amt, (size_t)cap * sizeof(double));
    if (!na) return 1;
    p->amt = na;
    p->cap = cap;
    return 0;
}

/* |B + P H - H|_1: every column j adds (d / #out_j) H_j to its children. */
static double ks_exact_residual(int64_t n, const int64_t *rp, const int32_t *col, const double *B, double d,
                                const double *H, double *work) {
    for (int64_t k = 0; k < n; ++k) work[k] = B[k] - H[k];
    for (int64_t j = 0; j < n; ++j) {
        const int64_t deg = rp[j + 1] - rp[j];
        if (deg == 0) continue;
        const double p = d / (double)deg;
        for (int64_t e = rp[j]; e < rp[j + 1]; ++e) work[col[e]] += p * H[j];
    }
    double r = 0.0;
    for (int64_t k = 0; k < n; ++k) r += fabs(work[k]);
    return r;
}

/*
 * Runs the simulation.  speed <= 0 means unbounded; sweeps_per_step = 0
 * means no limit (with an unbounded speed a limit is required).
 * Outputs: H, F (n each); per PID (K each): ops (elementary operations),
 * idle (unused capacity, in operations; bounded speed only), sleep_steps
 * (steps spent asleep), sends (transmissions); steps run, exact residual at
 * return, messages still in transit.  trace (optional, capacity trace_cap
 * steps of K values): r_k + s_k at the end of every step.
 * Returns 0 on convergence, 4 when max_steps was reached, 3 when the
 * simulation stalled above tol (every PID asleep, nothing to transmit and
 * nothing in transit: sleep_tol too large for tol), 1 on invalid arguments,
 * 2 when an allocation failed.
 */
int ks_run(int64_t n, const int64_t *rp, const int32_t *col, const double *B, double d, double tol, double alpha,
           int K, const int64_t *bounds, double speed, int sweeps_per_step, double delay_proba, uint64_t seed,
           double sleep_tol, int64_t max_steps, int threads, double *H, double *F, int64_t *ops, double *idle,
           int64_t *sleep_steps, int64_t *sends, int64_t *steps_out, double *resid_out, int64_t *in_transit,
           double *trace, int64_t trace_cap) {
    if (n < 1 || K < 1 || !(alpha > 1.0) || !(tol >= 0.0) || max_steps < 0) return 1;
    if (!(delay_proba >= 0.0 && delay_proba < 1.0) || !(sleep_tol >= 0.0)) return 1;
    if (speed <= 0.0 && sweeps_per_step < 1) return 1;
    if (bounds[0] != 0 || bounds[K] != n) return 1;
    for (int k = 0; k < K; ++k)
        if (bounds[k + 1] < bounds[k]) return 1;
    const int bounded = speed > 0.0;

    int32_t *part = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    double *H_old = (double *)calloc((size_t)n, sizeof(double));
    double *work = (double *)malloc((size_t)n * sizeof(double));
    double *T = (double *)calloc((size_t)K, sizeof(double));
    double *budget = (double *)calloc((size_t)K, sizeof(double));
    double *r = (double *)calloc((size_t)K, sizeof(double));
    double *s = (double *)calloc((size_t)K, sizeof(double));
    double *recv = (double *)calloc((size_t)K, sizeof(double));
    int64_t *cursor = (int64_t *)malloc((size_t)K * sizeof(int64_t));
    int *send = (int *)calloc((size_t)K, sizeof(int));
    int *moved = (int *)calloc((size_t)K, sizeof(int));   /* this step, the PID diffused a node */
    ks_msg *msgs = NULL;
    int64_t nmsg = 0, msg_cap = 0, next_id = 0;
    ks_pool pool = {NULL, NULL, 0, 0};
    int status = 2;
    if (!part || !H_old || !work || !T || !budget || !r || !s || !recv || !cursor || !send || !moved) goto done;

    for (int k = 0; k < K; ++k) {
        for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i) part[i] = k;
        ops[k] = 0;
        idle[k] = 0.0;
        sleep_steps[k] = 0;
        sends[k] = 0;
        cursor[k] = -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        F[i] = B[i];
        H[i] = 0.0;
    }
    for (int k = 0; k < K; ++k)   /* T_k starts at the largest fluid of the range */
        for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i)
            if (fabs(F[i]) > T[k]) T[k] = fabs(F[i]);

    status = 4;
    int64_t step = 0;
    double resid = 0.0;
    for (;;) {
        resid = ks_exact_residual(n, rp, col, B, d, H, work);
        if (resid <= tol) { status = 0; break; }
        if (step >= max_steps) { status = 4; break; }

        for (int k = 0; k < K; ++k) moved[k] = 0;
        /* the PIDs' local work: disjoint node ranges, so they run in parallel */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : omp_get_max_threads())
#endif
        for (int k = 0; k < K; ++k) {
            const int64_t lo = bounds[k], hi = bounds[k + 1];
            if (bounded) budget[k] += speed;
            int started = 0;
            for (;;) {
                if (bounded && budget[k] <= 0.0) break;
                if (cursor[k] < 0) {
                    if (sweeps_per_step > 0 && started >= sweeps_per_step) {
                        if (bounded) { idle[k] += budget[k]; budget[k] = 0.0; }
                        break;
                    }
                    double mx = 0.0, rk = 0.0;
                    for (int64_t i = lo; i < hi; ++i) {
                        const double a = fabs(F[i]);
                        rk += a;
                        if (a > mx) mx = a;
                    }
                    if (mx == 0.0 || rk <= sleep_tol) {      /* asleep for the rest of the step */
                        if (started == 0) sleep_steps[k] += 1;
                        if (bounded) { idle[k] += budget[k]; budget[k] = 0.0; }
                        break;
                    }
                    while (T[k] > mx) T[k] /= alpha;
                    cursor[k] = lo;
                    started += 1;
                }
                int64_t i = cursor[k];
                for (; i < hi; ++i) {
                    if (bounded && budget[k] <= 0.0) break;
                    const double sent = F[i];
                    if (fabs(sent) < T[k] || sent == 0.0) continue;
                    F[i] = 0.0;
                    H[i] += sent;
                    moved[k] = 1;
                    const int64_t deg = rp[i + 1] - rp[i];
                    if (deg == 0) continue;
                    const double p = d / (double)deg;
                    int64_t local = 0;
                    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                        const int32_t j = col[e];
                        if (part[j] != k) continue;
                        F[j] += sent * p;
                        local += 1;
                    }
                    ops[k] += local;
                    if (bounded) budget[k] -= (double)local;
                }
                if (i >= hi) {                 /* the sweep is complete */
                    cursor[k] = -1;
                    T[k] /= alpha;
                } else {
                    cursor[k] = i;             /* resume here next step */
                    break;
                }
            }
        }

        /* end of the step: residuals, owed fluid and the send decisions (Eq. send) */
        for (int k = 0; k < K; ++k) {
            double rk = 0.0, sk = 0.0;
            for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i) {
                rk += fabs(F[i]);
                const double dh = H[i] - H_old[i];
                const int64_t deg = rp[i + 1] - rp[i];
                if (dh == 0.0 || deg == 0) continue;
                const double p = d / (double)deg;
                for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
                    if (part[col[e]] != k) sk += fabs(p * dh);
            }
            r[k] = rk;
            s[k] = sk;
            recv[k] = 0.0;
            send[k] = sk > 0.0 && sk > rk / (double)K;
        }
        if (trace && step < trace_cap)
            for (int k = 0; k < K; ++k) trace[step * K + k] = r[k] + s[k];
        for (int k = 0; k < K; ++k) {
            if (!send[k]) continue;
            sends[k] += 1;
            if (nmsg == msg_cap) {
                const int64_t cap = msg_cap ? 2 * msg_cap : 64;
                ks_msg *nm = (ks_msg *)realloc(msgs, (size_t)cap * sizeof(ks_msg));
                if (!nm) { status = 2; goto done; }
                msgs = nm;
                msg_cap = cap;
            }
            ks_msg m = {pool.size, 0, next_id++, 0};
            for (int64_t i = bounds[k]; i < bounds[k + 1]; ++i) {
                const double dh = H[i] - H_old[i];
                const int64_t deg = rp[i + 1] - rp[i];
                H_old[i] = H[i];
                if (dh == 0.0 || deg == 0) continue;
                const double p = d / (double)deg;
                if (pool_reserve(&pool, deg)) { status = 2; goto done; }
                for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
                    const int32_t j = col[e];
                    if (part[j] == k) continue;
                    pool.node[pool.size] = j;
                    pool.amt[pool.size] = p * dh;
                    pool.size += 1;
                    m.count += 1;
                }
            }
            ops[k] += m.count;
            if (bounded) budget[k] -= (double)m.count;
            msgs[nmsg++] = m;
        }
        /* deliveries due this step (every message in transit is tested once) */
        int64_t kept = 0;
        for (int64_t q = 0; q < nmsg; ++q) {
            ks_msg m = msgs[q];
            if (delay_proba > 0.0 && ks_uniform(seed, (uint64_t)m.id, (uint64_t)m.tests) < delay_proba) {
                m.tests += 1;
                msgs[kept++] = m;
                continue;
            }
            for (int64_t e = m.first; e < m.first + m.count; ++e) {
                const int32_t j = pool.node[e];
                F[j] += pool.amt[e];
                recv[part[j]] += fabs(pool.amt[e]);
            }
        }
        const int64_t delivered = nmsg - kept;
        nmsg = kept;
        if (nmsg == 0) pool.size = 0;         /* nothing in transit: reuse the pool */
        int any_work = 0;
        for (int k = 0; k < K; ++k) any_work |= moved[k] | send[k];
        if (!any_work && delivered == 0 && nmsg == 0) {
            /* every PID asleep, nothing owed above its send threshold and nothing
               in transit: no later step can change the state */
            step += 1;
            resid = ks_exact_residual(n, rp, col, B, d, H, work);
            status = resid <= tol ? 0 : 3;
            break;
        }
        /* reception (Sec. 2.6): rescale the threshold of every receiver */
        for (int k = 0; k < K; ++k) {
            if (recv[k] == 0.0) continue;
            if (r[k] > 0.0) T[k] *= (r[k] + recv[k]) / r[k];
            else T[k] = recv[k];
        }
        step += 1;
    }
    *steps_out = step;
    *resid_out = resid;
    *in_transit = nmsg;
done:
    if (status == 2) { *steps_out = 0; *resid_out = 0.0; *in_transit = 0; }
    free(part); free(H_old); free(work); free(T); free(budget); free(r); free(s); free(recv);
    free(cursor); free(send); free(moved); free(msgs); free(pool.node); free(pool.amt);
    return status;
}
