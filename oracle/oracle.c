/*
 * FP64 CPU oracle for depth-p QAOA on NAE-k-SAT (arXiv 2401.02852).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library, and it never calls into it.
 *
 * Conventions (readings of the paper, stated once):
 *   - assignment index x = sum_l x_l 2^l: variable l is bit l of x (the
 *     decimal representation of Appendix A.3 is garbled; this is the reading);
 *   - X_j flips bit j: X_j |x> = |x xor 2^j>;
 *   - literal (v, s): its value is bit v of x, complemented when s = 1
 *     (s = 1 is the negated literal, Eq. for the literal Hamiltonian);
 *   - layer i = 0 (the first gamma/beta) acts first on |+>^n (Eq. for the
 *     QAOA output state, product over i = 0..p-1 read right to left);
 *   - mixer sign s = +1: U_B(beta) = exp(+i beta sum_j X_j) = prod_j
 *     [cos(beta) I + i sin(beta) X_j] (Sec. "Efficient Classical Simulation",
 *     Appendix A.3); s = -1 gives exp(-i beta sum_j X_j) (Sec. 2.1's form).
 *
 * Parity pins live in the tests: closed forms (n = 1), dense matrix
 * exponentials (n <= 8), the random-assignment theorem (gamma = 0 or beta = 0),
 * the clause-counting identity and the global-flip symmetry.
 *
 * Everything is FP64 and serial apart from OpenMP loops whose iterations are
 * independent (same arithmetic, same result for any thread count).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OK 0
#define EINVAL_ -1
#define ENOMEM_ -3

/* ------------------------------------------------------------------------ */
/* Cost function, Eq. for C^NAE (Sec. "Problem Hamiltonian") and its De Morgan
 * form (Appendix A.2): clause i is violated under NAE iff all its literals are
 * false (the clause is unsatisfied) or all are true.                          */

static int clause_violated(uint64_t x, int k, const int32_t *var, const uint8_t *neg) {
    int n_true = 0;
    for (int j = 0; j < k; ++j) {
        int bit = (int)((x >> var[j]) & 1u);
        int lit = neg[j] ? 1 - bit : bit;
        n_true += lit;
    }
    return (n_true == 0) || (n_true == k);
}

/* C(x) for one assignment x. */
uint32_t oracle_cost_at(uint64_t x, int m, int k, const int32_t *var, const uint8_t *neg) {
    uint32_t c = 0;
    for (int i = 0; i < m; ++i) c += (uint32_t)clause_violated(x, k, var + (size_t)i * k, neg + (size_t)i * k);
    return c;
}

/* C(x) for a list of assignments (sampled checks at sizes where the full table
 * does not fit). */
int oracle_cost_samples(int m, int k, const int32_t *var, const uint8_t *neg,
                        int64_t count, const uint64_t *xs, uint32_t *out) {
    if (m < 0 || k < 1 || count < 0) return EINVAL_;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t) out[t] = oracle_cost_at(xs[t], m, k, var, neg);
    return OK;
}

/* Full table C[0 .. 2^n - 1] (uint16: exact for m <= 65535). Also returns the
 * number of x with C(x) = 0 and the largest C. */
int oracle_cost_table(int n, int m, int k, const int32_t *var, const uint8_t *neg,
                      uint16_t *cost, uint64_t *n_sol, uint32_t *max_cost) {
    if (n < 1 || n > 34 || m < 0 || m > 65535 || k < 1 || k > n) return EINVAL_;
    for (int i = 0; i < m * k; ++i)
        if (var[i] < 0 || var[i] >= n) return EINVAL_;
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) cost[x] = (uint16_t)oracle_cost_at((uint64_t)x, m, k, var, neg);
    uint64_t sol = 0;
    uint32_t mx = 0;
    for (int64_t x = 0; x < N; ++x) {
        if (cost[x] == 0) ++sol;
        if (cost[x] > mx) mx = cost[x];
    }
    if (n_sol) *n_sol = sol;
    if (max_cost) *max_cost = mx;
    return OK;
}

/* ------------------------------------------------------------------------ */
/* State evolution.  psi is interleaved (re, im) doubles, 2 * 2^n of them.   */

/* Uniform superposition |+>^n = 2^{-n/2} sum_x |x> (Sec. 2.1). */
static void plus_state(int n, double complex *psi) {
    const int64_t N = (int64_t)1 << n;
    const double a = pow(2.0, -0.5 * n);
    for (int64_t x = 0; x < N; ++x) psi[x] = a;
}

/* U_C(gamma) = sum_x exp(-i gamma C(x)) |x><x| (Eq. for U_C, Appendix A.3's
 * diagonalisation).  exp is evaluated per x, no table. */
static void apply_phase(int n, const uint16_t *cost, double gamma, double complex *psi) {
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) psi[x] *= cexp(-I * gamma * (double)cost[x]);
}

/* U_B(beta) = prod_j [cos(beta) I + i s sin(beta) X_j] (Appendix A.3): for each
 * qubit j, every pair (x, x | 2^j) with bit j of x clear is replaced by
 * (c a + i s sn b, i s sn a + c b). */
static void apply_mixer(int n, double beta, int sign, double complex *psi) {
    const int64_t N = (int64_t)1 << n;
    const double c = cos(beta);
    const double complex is = I * (double)sign * sin(beta);
    for (int j = 0; j < n; ++j) {
        const int64_t h = (int64_t)1 << j;
#pragma omp parallel for schedule(static)
        for (int64_t x = 0; x < N; ++x) {
            if (x & h) continue;
            double complex a = psi[x], b = psi[x | h];
            psi[x] = c * a + is * b;
            psi[x | h] = is * a + c * b;
        }
    }
}

/* |gamma, beta>_p = prod_{i=0}^{p-1} U_B(beta_i) U_C(gamma_i) |+>^n
 * (Eq. for the QAOA output state); layer i = 0 first. */
int oracle_evolve(int n, const uint16_t *cost, int p, const double *gamma, const double *beta,
                  int sign, double *psi_out) {
    if (n < 1 || n > 34 || p < 0 || (sign != 1 && sign != -1)) return EINVAL_;
    double complex *psi = (double complex *)psi_out;
    plus_state(n, psi);
    for (int i = 0; i < p; ++i) {
        apply_phase(n, cost, gamma[i], psi);
        apply_mixer(n, beta[i], sign, psi);
    }
    return OK;
}

/* Pairwise (recursive halving) sum of f over [lo, hi). */
static double pairwise_norm(const double complex *psi, int64_t lo, int64_t hi) {
    if (hi - lo <= 8) {
        double s = 0.0;
        for (int64_t x = lo; x < hi; ++x) s += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
        return s;
    }
    int64_t mid = lo + (hi - lo) / 2;
    return pairwise_norm(psi, lo, mid) + pairwise_norm(psi, mid, hi);
}

static double pairwise_psucc(const double complex *psi, const uint16_t *cost, int64_t lo, int64_t hi) {
    if (hi - lo <= 8) {
        double s = 0.0;
        for (int64_t x = lo; x < hi; ++x)
            if (cost[x] == 0) s += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
        return s;
    }
    int64_t mid = lo + (hi - lo) / 2;
    return pairwise_psucc(psi, cost, lo, mid) + pairwise_psucc(psi, cost, mid, hi);
}

/* p_succ = <Psi| {H_C = 0} |Psi> (Def. of the success probability): the mass
 * on assignments with C(x) = 0; the norm <Psi|Psi> is returned beside it. */
int oracle_success_prob(int n, const uint16_t *cost, const double *psi_in, double *p_succ, double *norm) {
    if (n < 1 || n > 34) return EINVAL_;
    const double complex *psi = (const double complex *)psi_in;
    const int64_t N = (int64_t)1 << n;
    if (p_succ) *p_succ = pairwise_psucc(psi, cost, 0, N);
    if (norm) *norm = pairwise_norm(psi, 0, N);
    return OK;
}

/* ------------------------------------------------------------------------ */
/* Gradient of p_succ with respect to (gamma_i, beta_i): reverse-mode
 * differentiation of the layer product with every forward state stored (what
 * automatic differentiation through the simulator computes, Sec. "QAOA
 * Procedure": the angles are trained by gradient ascent on p_succ).
 *
 * Forward: phi_l = D_l psi_{l-1}, psi_l = M_l phi_l with D_l = exp(-i gamma_l C),
 * M_l = exp(i s beta_l B), B = sum_j X_j.  f = <psi_p|P|psi_p>.
 *   df/dbeta_l  = 2 Re <lam_l| i s B |psi_l>,          lam_p = P psi_p
 *   mu_l        = M_l^dagger lam_l
 *   df/dgamma_l = 2 Re <mu_l| (-i C) |phi_l>
 *   lam_{l-1}   = D_l^dagger mu_l
 * The stored phi_l, psi_l are used directly (no recomputation). */
int oracle_grad(int n, const uint16_t *cost, int p, const double *gamma, const double *beta, int sign,
                double *p_succ, double *dgamma, double *dbeta) {
    if (n < 1 || n > 30 || p < 0 || (sign != 1 && sign != -1)) return EINVAL_;
    const int64_t N = (int64_t)1 << n;
    /* states[2l] = psi_l (l = 0..p), states[2l - 1] = phi_l (l = 1..p) */
    double complex *states = (double complex *)malloc(sizeof(double complex) * (size_t)N * (size_t)(2 * p + 1));
    double complex *lam = (double complex *)malloc(sizeof(double complex) * (size_t)N);
    if (!states || !lam) {
        free(states);
        free(lam);
        return ENOMEM_;
    }
    plus_state(n, states);
    for (int l = 1; l <= p; ++l) {
        memcpy(states + (size_t)(2 * l - 1) * N, states + (size_t)(2 * l - 2) * N, sizeof(double complex) * N);
        apply_phase(n, cost, gamma[l - 1], states + (size_t)(2 * l - 1) * N);
        memcpy(states + (size_t)(2 * l) * N, states + (size_t)(2 * l - 1) * N, sizeof(double complex) * N);
        apply_mixer(n, beta[l - 1], sign, states + (size_t)(2 * l) * N);
    }
    const double complex *psi_p = states + (size_t)(2 * p) * N;
    if (p_succ) *p_succ = pairwise_psucc(psi_p, cost, 0, N);
    for (int64_t x = 0; x < N; ++x) lam[x] = cost[x] == 0 ? psi_p[x] : 0.0;
    for (int l = p; l >= 1; --l) {
        const double complex *psi_l = states + (size_t)(2 * l) * N;
        const double complex *phi_l = states + (size_t)(2 * l - 1) * N;
        /* <lam| i s B |psi> = i s sum_j sum_x conj(lam(x)) psi(x xor 2^j) */
        double complex acc = 0.0;
        for (int j = 0; j < n; ++j) {
            const int64_t h = (int64_t)1 << j;
            for (int64_t x = 0; x < N; ++x) acc += conj(lam[x]) * psi_l[x ^ h];
        }
        dbeta[l - 1] = 2.0 * creal(I * (double)sign * acc);
        /* mu_l = M_l^dagger lam_l = exp(-i s beta_l B) lam_l */
        apply_mixer(n, -beta[l - 1], sign, lam);
        /* <mu| -i C |phi> */
        double complex accg = 0.0;
        for (int64_t x = 0; x < N; ++x) accg += conj(lam[x]) * (-I * (double)cost[x]) * phi_l[x];
        dgamma[l - 1] = 2.0 * creal(accg);
        /* lam_{l-1} = D_l^dagger mu_l */
        apply_phase(n, cost, -gamma[l - 1], lam);
    }
    free(states);
    free(lam);
    return OK;
}

/* ------------------------------------------------------------------------ */
/* Bitstrings drawn from the output state (Sec. "Running Times": measuring the
 * final state yields x with probability |Psi(x)|^2, and the running time of an
 * instance is the number of such draws up to and including the first one that
 * satisfies it).  The caller supplies one uniform u_j in [0, 1) per draw, so
 * two implementations given the same uniforms make the same draws.  Draw j is
 * the inverse of the cumulative distribution in index order:
 *   F(x) = sum_{y <= x} |psi(y)|^2,   x_j = min { x : F(x) > u_j F(2^n - 1) },
 * which never returns an x of probability zero. */
int oracle_sample(int n, const double *psi_in, int k, const double *u, uint64_t *x_out) {
    if (n < 1 || n > 30 || k < 0) return EINVAL_;
    const double complex *psi = (const double complex *)psi_in;
    const int64_t N = (int64_t)1 << n;
    double *F = (double *)malloc(sizeof(double) * (size_t)N);
    if (!F) return ENOMEM_;
    double run = 0.0;
    for (int64_t x = 0; x < N; ++x) {
        run += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
        F[x] = run;
    }
    for (int j = 0; j < k; ++j) {
        const double t = u[j] * F[N - 1];
        int64_t lo = 0, hi = N - 1; /* smallest x with F[x] > t (N - 1 if none) */
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (F[mid] > t)
                hi = mid;
            else
                lo = mid + 1;
        }
        x_out[j] = (uint64_t)lo;
    }
    free(F);
    return OK;
}

/* Running time of one instance over the given draws: 1 + the index of the
 * first draw with C(x_j) = 0, or 0 when none of the k draws satisfies. */
int oracle_running_time(int n, const uint16_t *cost, const double *psi_in, int k, const double *u,
                        int64_t *running_time) {
    if (k < 0) return EINVAL_;
    uint64_t *xs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(k > 0 ? k : 1));
    if (!xs) return ENOMEM_;
    int rc = oracle_sample(n, psi_in, k, u, xs);
    if (rc == OK) {
        *running_time = 0;
        for (int j = 0; j < k; ++j)
            if (cost[xs[j]] == 0) {
                *running_time = j + 1;
                break;
            }
    }
    free(xs);
    return rc;
}
