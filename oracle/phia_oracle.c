/*
 * phia_oracle.c -- plain, slow FP64 CPU oracle for PHIA (arXiv 2407.10205).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no code, header, table or constant with the CUDA
 * library; the only thing both sides share is the seeded input generators,
 * which hold none of the method's arithmetic.
 *
 * Every function follows one passage of the paper, named in its comment:
 *   Eq. 2        Ising energy E(s) = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i
 *   Eq. 6        local field (quasi-gradient) I_i = sum_j J_ij sgn(x_j) + h_i
 *   Eq. 4 / A6   H(x,v) = beta E(sgn x) + x.x/2 + v.v/2
 *   Eq. 5, 7, 8  dv/dt = beta * gamma (1 - tanh^2(gamma x)) * I - x
 *   Eq. A7, A8   x <- x + eps v ;  v <- v - eps grad H(x_new)
 *   Table 3      state 4: acceptance test on H at the end of a trajectory (optional)
 *                state 5: keep the best state seen so far
 *   Sec. 2.1     momentum drawn at random at the start of a trajectory;
 *                position prior g(x) is a standard normal (Eq. A3)
 *   Sec. 2.1, 3.2  vanilla GAHMC: the exact solution of the dynamics by zero
 *                crossings (the method PHIA approximates; the paper's ablation)
 *
 * Fixed point (Sec. 2.2, coefficients held as fixed-point constants):
 * J_ij = k_ij * q and h_i = kh_i * q with q = 2^-f, int8 k and int32 kh.
 * Fields and energies are exact int64 integers in units of q.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11) written from its published definition,
 * and the Box-Muller transform (Box & Muller, 1958) in FP64.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox */

/* One Philox4x32-10 block: 10 rounds of the 4x32 S-box with the Weyl key
 * schedule, as defined by Salmon et al. (SC'11, Sec. 3 and Table 2). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mul0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)mul1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += weyl0;
        k1 += weyl1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniforms on 24 bits, so that the same value is exact in FP32 and FP64. */
double orc_u01_open(uint32_t a) { return (double)((a >> 8) + 1u) * (1.0 / 16777216.0); } /* (0,1] */
double orc_u01_half(uint32_t a) { return (double)(a >> 8) * (1.0 / 16777216.0); }        /* [0,1) */

/* Box-Muller: one standard normal from two uniforms (cosine branch). */
double orc_box_muller(uint32_t a, uint32_t b)
{
    double u1 = orc_u01_open(a), u2 = orc_u01_half(b);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* The draw for spin j of replica r, draw index d (0 = initial state, t = momentum refresh
 * before iteration t) of instance `inst`: counter (j, r, d, inst), key = 64-bit seed.
 * Words 0,1 give the position sample (g(x) of Eq. A3), words 2,3 the momentum sample. */
void orc_draw(uint64_t seed, uint32_t inst, uint32_t r, uint32_t j, uint32_t d,
              double *nx, double *nv)
{
    uint32_t ctr[4] = {j, r, d, inst};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    if (nx) *nx = orc_box_muller(o[0], o[1]);
    if (nv) *nv = orc_box_muller(o[2], o[3]);
}

/* ------------------------------------------------------------- instance */

/* One Ising instance: either a dense k matrix (n*n, row-major) or CSR
 * (row_ptr[n+1], col[nnz], val[nnz]); kh has n entries. */
typedef struct {
    int32_t n;
    const int8_t *k;        /* dense, or NULL */
    const int32_t *row_ptr; /* CSR, used when k == NULL */
    const int32_t *col;
    const int8_t *val;
    const int32_t *kh;
} orc_inst;

/* Eq. 2, literally: E = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i (units of q). */
int64_t orc_energy_exact(const orc_inst *P, const int8_t *s)
{
    int64_t e = 0;
    int n = P->n;
    if (P->k) {
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j)
                e -= (int64_t)P->k[(int64_t)i * n + j] * s[i] * s[j];
    } else {
        for (int i = 0; i < n; ++i)
            for (int32_t p = P->row_ptr[i]; p < P->row_ptr[i + 1]; ++p) {
                int j = P->col[p];
                if (j > i) e -= (int64_t)P->val[p] * s[i] * s[j];
            }
    }
    for (int i = 0; i < n; ++i) e -= (int64_t)P->kh[i] * s[i];
    return e;
}

/* Eq. 6: I_i = sum_j J_ij s_j + h_i (units of q). */
void orc_field(const orc_inst *P, const int8_t *s, int64_t *I)
{
    int n = P->n;
    for (int i = 0; i < n; ++i) {
        int64_t acc = 0;
        if (P->k) {
            for (int j = 0; j < n; ++j) acc += (int64_t)P->k[(int64_t)i * n + j] * s[j];
        } else {
            for (int32_t p = P->row_ptr[i]; p < P->row_ptr[i + 1]; ++p)
                acc += (int64_t)P->val[p] * s[P->col[p]];
        }
        I[i] = acc + P->kh[i];
    }
}

/* E from the field: Eq. 2 and Eq. 6 give E = -1/2 sum_i s_i (I_i + h_i). */
int64_t orc_energy_from_field(const orc_inst *P, const int8_t *s, const int64_t *I)
{
    int64_t twice = 0;
    for (int i = 0; i < P->n; ++i) twice += (int64_t)s[i] * (I[i] + P->kh[i]);
    return -twice / 2;
}

/* Exhaustive minimum of Eq. 2 over all 2^n states (n <= 24).  State index b maps
 * to s_i = +1 when bit i of b is set, else -1.  Returns the minimum; writes the
 * number of minimisers and the lowest-index minimiser. */
int64_t orc_brute_force(const orc_inst *P, int64_t *n_min, int8_t *argmin)
{
    int n = P->n;
    int8_t *s = (int8_t *)malloc((size_t)n);
    int64_t best = INT64_MAX, count = 0;
    uint64_t total = 1ull << n;
    for (uint64_t b = 0; b < total; ++b) {
        for (int i = 0; i < n; ++i) s[i] = ((b >> i) & 1u) ? 1 : -1;
        int64_t e = orc_energy_exact(P, s);
        if (e < best) {
            best = e;
            count = 1;
            if (argmin) memcpy(argmin, s, (size_t)n);
        } else if (e == best) {
            ++count;
        }
    }
    free(s);
    if (n_min) *n_min = count;
    return best;
}

/* ----------------------------------------------------------------- update */

/* sgn with sgn(0) = +1 (the paper leaves sgn(0) open). */
static int8_t orc_sgn(double x) { return x >= 0.0 ? 1 : -1; }

/* The derivative factor of Eq. 8 at y = gamma x: 1 - tanh^2(y) (deriv = 0), or
 * (deriv = 1) a quadratic stand-in for it.  Sec. 2.2 says the FPGA approximates the
 * derivative by a quadratic polynomial but prints no coefficients; the ones here are
 * this implementation's own choice: max(0, 1 - (y / 1.5)^2), equal to the exact factor
 * at y = 0 and with the same integral over the real line (4 * 1.5 / 3 = 2). */
double orc_dfactor(double y, int32_t deriv)
{
    if (deriv == 1) {
        double u = y / 1.5;
        return u * u >= 1.0 ? 0.0 : 1.0 - u * u;
    }
    double t = tanh(y);
    return 1.0 - t * t;
}

/* One iteration of Eq. A7 with the gradient of Eq. A8 under the tanh surrogate
 * (Eqs. 7-8):
 *   x <- x + eps v
 *   s  = sgn x
 *   I  = J s + h                                  (Eq. 6)
 *   dH/dx_i = -beta * gamma (1 - tanh^2(gamma x_i)) * q * I_i + x_i   (Eqs. 4, 5, 8)
 *   v <- v - eps dH/dx
 * Writes s and I (units of q); returns E(s) in units of q. */
int64_t orc_step_mode(const orc_inst *P, double q, double beta, double eps, double gamma, int32_t deriv,
                      double *x, double *v, int8_t *s, int64_t *I)
{
    int n = P->n;
    for (int i = 0; i < n; ++i) x[i] = x[i] + eps * v[i];
    for (int i = 0; i < n; ++i) s[i] = orc_sgn(x[i]);
    orc_field(P, s, I);
    for (int i = 0; i < n; ++i) {
        double grad = -beta * gamma * orc_dfactor(gamma * x[i], deriv) * q * (double)I[i] + x[i];
        v[i] = v[i] - eps * grad;
    }
    return orc_energy_from_field(P, s, I);
}

/* The same with the exact derivative factor. */
int64_t orc_step(const orc_inst *P, double q, double beta, double eps, double gamma,
                 double *x, double *v, int8_t *s, int64_t *I)
{
    return orc_step_mode(P, q, beta, eps, gamma, 0, x, v, s, I);
}

/* Annealing schedule (Table 3, state 4: the temperature is adjusted as the run
 * proceeds).  beta goes linearly from beta0 at iteration 0 to beta1 at the last
 * iteration; eps and gamma are constant; refresh > 0 redraws the momentum at the
 * start of every iteration t with t % refresh == 0, t > 0 (a new HMC trajectory
 * from the previous end point, Fig. 1b). */
typedef struct {
    double beta0, beta1, eps, gamma;
    int64_t refresh;
    int32_t has_target;
    int32_t stop_at_target;
    int64_t target;
    int32_t deriv;      /* derivative factor: 0 exact, 1 quadratic stand-in (orc_dfactor) */
    int32_t accept_test;/* 0: every trajectory accepted (App. A); 1: Metropolis test on H (orc_metropolis) */
} orc_sched;

double orc_beta_at(const orc_sched *S, int64_t t, int64_t T)
{
    if (T <= 1) return S->beta0;
    return S->beta0 + (S->beta1 - S->beta0) * (double)t / (double)(T - 1);
}

/* Per-replica result. */
typedef struct {
    int64_t best_e;     /* lowest E seen (units of q) */
    int64_t best_step;  /* first iteration at which it was seen */
    int64_t hit_step;   /* first iteration with E <= target, or -1 */
    int64_t steps_run;  /* iterations executed */
    int64_t proposed;   /* trajectories put to the acceptance test (accept_test = 1) */
    int64_t accepted;   /* of those, accepted */
} orc_replica_out;

/* Eq. 4 (= Eq. A6): H(x, v) = beta E(sgn x) + x.x / 2 + v.v / 2, with E in units of q
 * (beta E = beta q e). */
double orc_hamiltonian(double beta, double q, int64_t e, const double *x, const double *v, int n)
{
    double xx = 0.0, vv = 0.0;
    for (int i = 0; i < n; ++i) {
        xx += x[i] * x[i];
        vv += v[i] * v[i];
    }
    return beta * q * (double)e + 0.5 * xx + 0.5 * vv;
}

/* Table 3, state 4 read as the Metropolis test of HMC (App. A: exact dynamics conserve H,
 * so the test accepts with probability 1; the discretised dynamics of Eq. A7 do not):
 * the proposed end point of a trajectory is accepted with probability
 * min(1, exp(-(H_end - H_start))), i.e. when the uniform u in (0, 1] satisfies
 * u <= exp(-(H_end - H_start)).  Returns 1 to accept. */
int orc_metropolis(double h_start, double h_end, double u)
{
    return u <= exp(-(h_end - h_start)) ? 1 : 0;
}

/* The uniform of the test that ends at the momentum draw d = t of the next trajectory:
 * Philox counter (0xFFFFFFFF, r, t, inst) -- a spin index no instance has -- word 0, on
 * the 24-bit grid of (0, 1]. */
double orc_accept_uniform(uint64_t seed, uint32_t inst, uint32_t r, uint32_t t)
{
    uint32_t ctr[4] = {0xFFFFFFFFu, r, t, inst};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    return orc_u01_open(o[0]);
}

/* One replica of a PHIA run: initial draw (d = 0), then T iterations of
 * orc_step with the momentum redrawn at trajectory starts; the best state is
 * kept with strict improvement (Table 3, state 5).  With S->accept_test = 1 and a
 * refresh period, each trajectory's end point except the first's is put to the
 * Metropolis test of orc_metropolis just before the next momentum draw (Table 3,
 * state 4); a rejected end point sends x back to the trajectory's start (every
 * state visited still counts for the best state).  The run's last trajectory has
 * no test: nothing follows it.  x0/v0, when given, replace the initial draw.  x/v
 * out (optional) receive the final state. */
void orc_anneal_replica(const orc_inst *P, int32_t frac_bits, const orc_sched *S, int64_t T,
                        uint64_t seed, uint32_t inst_id, uint32_t r,
                        const double *x0, const double *v0,
                        orc_replica_out *out, int8_t *best_s, double *x_out, double *v_out,
                        int64_t *energy_trace)
{
    int n = P->n;
    double q = ldexp(1.0, -frac_bits);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *xs = (double *)malloc(sizeof(double) * (size_t)n);  /* trajectory start (accept_test) */
    double *vs = (double *)malloc(sizeof(double) * (size_t)n);
    int8_t *s = (int8_t *)malloc((size_t)n);
    int64_t *I = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int j = 0; j < n; ++j) {
        if (x0 && v0) {
            x[j] = x0[j];
            v[j] = v0[j];
        } else {
            orc_draw(seed, inst_id, r, (uint32_t)j, 0u, &x[j], &v[j]);
        }
    }
    out->best_e = INT64_MAX;
    out->best_step = -1;
    out->hit_step = -1;
    out->steps_run = 0;
    out->proposed = 0;
    out->accepted = 0;
    int64_t e_prev = 0;      /* E of the last iteration */
    int64_t e_start = 0;     /* E(sgn x) at the start of the current trajectory */
    int has_start = 0;       /* the current trajectory's start state is known (not the first) */
    for (int64_t t = 0; t < T; ++t) {
        if (S->refresh > 0 && t > 0 && t % S->refresh == 0) {
            if (S->accept_test == 1) {
                /* End of the trajectory that ran iterations [t - refresh, t): test its end
                 * point against its start under the Hamiltonian of its last iteration.  The
                 * first trajectory starts from the initial draw, whose energy no iteration
                 * evaluated; it is accepted as it stands. */
                if (has_start) {
                    double beta_end = orc_beta_at(S, t - 1, T);
                    double h_start = orc_hamiltonian(beta_end, q, e_start, xs, vs, n);
                    double h_end = orc_hamiltonian(beta_end, q, e_prev, x, v, n);
                    double u = orc_accept_uniform(seed, inst_id, r, (uint32_t)t);
                    out->proposed += 1;
                    if (orc_metropolis(h_start, h_end, u)) {
                        out->accepted += 1;
                        e_start = e_prev;
                    } else {
                        memcpy(x, xs, sizeof(double) * (size_t)n);   /* back to the start point */
                    }
                } else {
                    e_start = e_prev;
                    has_start = 1;
                }
            }
            for (int j = 0; j < n; ++j) orc_draw(seed, inst_id, r, (uint32_t)j, (uint32_t)t, NULL, &v[j]);
            if (S->accept_test == 1) {
                memcpy(xs, x, sizeof(double) * (size_t)n);
                memcpy(vs, v, sizeof(double) * (size_t)n);
            }
        }
        double beta = orc_beta_at(S, t, T);
        int64_t e = orc_step_mode(P, q, beta, S->eps, S->gamma, S->deriv, x, v, s, I);
        e_prev = e;
        if (energy_trace) energy_trace[t] = e;
        out->steps_run = t + 1;
        int frozen = S->stop_at_target && out->hit_step >= 0;
        if (!frozen && e < out->best_e) {
            out->best_e = e;
            out->best_step = t;
            if (best_s) memcpy(best_s, s, (size_t)n);
        }
        if (S->has_target && out->hit_step < 0 && e <= S->target) {
            out->hit_step = t;
            if (S->stop_at_target) break;
        }
    }
    if (x_out) memcpy(x_out, x, sizeof(double) * (size_t)n);
    if (v_out) memcpy(v_out, v, sizeof(double) * (size_t)n);
    free(x); free(v); free(xs); free(vs); free(s); free(I);
}

/* ------------------------------------------------------ threaded replicas */

typedef struct {
    const orc_inst *P;
    int32_t frac_bits;
    const orc_sched *S;
    int64_t T;
    uint64_t seed;
    uint32_t inst_id;
    int32_t R;
    int32_t next;  /* protected by mu */
    pthread_mutex_t mu;
    orc_replica_out *outs;
    int8_t *best_s;   /* R*n or NULL */
    int32_t r0;       /* replica index offset */
} orc_pool;

static void *orc_worker(void *arg)
{
    orc_pool *pool = (orc_pool *)arg;
    for (;;) {
        pthread_mutex_lock(&pool->mu);
        int r = pool->next++;
        pthread_mutex_unlock(&pool->mu);
        if (r >= pool->R) break;
        int8_t *bs = pool->best_s ? pool->best_s + (int64_t)r * pool->P->n : NULL;
        orc_anneal_replica(pool->P, pool->frac_bits, pool->S, pool->T, pool->seed, pool->inst_id,
                           (uint32_t)(pool->r0 + r), NULL, NULL, &pool->outs[r], bs, NULL, NULL, NULL);
    }
    return NULL;
}

/* Replicas r0 .. r0+R-1 of one instance, spread over `threads` POSIX threads. */
void orc_anneal_replicas(const orc_inst *P, int32_t frac_bits, const orc_sched *S, int64_t T,
                         uint64_t seed, uint32_t inst_id, int32_t r0, int32_t R, int32_t threads,
                         orc_replica_out *outs, int8_t *best_s)
{
    orc_pool pool;
    pool.P = P; pool.frac_bits = frac_bits; pool.S = S; pool.T = T; pool.seed = seed;
    pool.inst_id = inst_id; pool.R = R; pool.next = 0; pool.outs = outs; pool.best_s = best_s;
    pool.r0 = r0;
    pthread_mutex_init(&pool.mu, NULL);
    if (threads < 1) threads = 1;
    if (threads > R) threads = R;
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int t = 0; t < threads; ++t) pthread_create(&tid[t], NULL, orc_worker, &pool);
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
    free(tid);
    pthread_mutex_destroy(&pool.mu);
}

/* ---------------------------------------------------------- vanilla GAHMC */

/* The exact solution of the dynamics of H(x, v) = beta E(sgn x) + x.x/2 + v.v/2 (Eq. 4,
 * App. A) by zero crossings -- the Gaussian-augmented HMC of the paper's reference
 * [Pakman & Paninski 2013] that Sec. 2.1 names as the exact alternative to the
 * approximate gradient and Sec. 3.2 uses as an ablation.
 *
 * Inside an orthant sgn x = s is fixed and the potential is x.x/2 (+ a constant), so each
 * coordinate moves on the unit circle: x_i(t) = x_i cos t + v_i sin t,
 * v_i(t) = -x_i sin t + v_i cos t.  When x_j reaches 0 the potential would jump by
 * dU = beta q dE with dE = E(s with s_j flipped) - E(s) = 2 s_j I_j (Eqs. 2, 6; units of
 * q).  Energy conservation decides: the speed there is A_j = sqrt(x_j^2 + v_j^2); if
 * A_j^2 / 2 > dU the coordinate crosses into the other orthant with speed
 * sqrt(A_j^2 - 2 dU) (s_j flips, the field follows), else it is reflected (speed A_j,
 * direction reversed).  Either way x_j = 0 afterwards, so its next zero is exactly pi
 * later: with a travel time <= pi each coordinate meets the wall at most once per
 * trajectory, at the time its start state fixes.  The events are taken in time order
 * (ties: lower index first); each decision uses the field left by the earlier ones.
 *
 * A run: the initial draw (Philox d = 0, as PHIA), then `trajectories` trajectories of
 * time `travel` each; trajectory k > 0 starts with the momentum draw d = k; beta is
 * linear from beta0 (k = 0) to beta1 (k = K - 1).  The best energy over every state
 * visited (the initial one and one per crossing) is kept with strict improvement;
 * best_traj is the trajectory in which it was first reached (0 for the initial state). */
typedef struct {
    double beta0, beta1;
    double travel;          /* time per trajectory, 0 < travel <= pi */
    int64_t trajectories;
    int32_t has_target;
    int32_t pad;
    int64_t target;
} orc_gahmc_sched;

typedef struct {
    int64_t best_e;
    int64_t best_traj;
    int64_t crossings;
    int64_t reflections;
    int64_t hit_traj;       /* first trajectory reaching E <= target (0: the initial state), or -1 */
} orc_gahmc_out;

/* First time t in [0, pi] at which x(t) = x0 cos t + v0 sin t leaves the orthant of sign
 * s (the zero of x with x moving from sign s to -s). */
double orc_gahmc_cross_time(double x0, double v0, int8_t s)
{
    /* x(t) = 0 where (cos t, sin t) is parallel to (v0, -x0); of the two roots per period
     * the one where x goes from s to -s has s * v(t) < 0. */
    return s > 0 ? atan2(x0, -v0) : atan2(-x0, v0);
}

void orc_gahmc_replica(const orc_inst *P, int32_t frac_bits, const orc_gahmc_sched *S, uint64_t seed,
                       uint32_t inst_id, uint32_t r, const double *x0, const double *v0, orc_gahmc_out *out,
                       int8_t *best_s, double *x_out, double *v_out, int8_t *s_out, int32_t *events,
                       int64_t events_cap)
{
    int n = P->n;
    double q = ldexp(1.0, -frac_bits);
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *tev = (double *)malloc(sizeof(double) * (size_t)n);
    double *vnew = (double *)malloc(sizeof(double) * (size_t)n);
    int *order = (int *)malloc(sizeof(int) * (size_t)n);
    int8_t *s = (int8_t *)malloc((size_t)n);
    int64_t *I = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int j = 0; j < n; ++j) {
        if (x0 && v0) {
            x[j] = x0[j];
            v[j] = v0[j];
        } else {
            orc_draw(seed, inst_id, r, (uint32_t)j, 0u, &x[j], &v[j]);
        }
        s[j] = orc_sgn(x[j]);
    }
    orc_field(P, s, I);
    int64_t e = orc_energy_exact(P, s);
    out->best_e = e;
    out->best_traj = 0;
    out->crossings = 0;
    out->reflections = 0;
    out->hit_traj = (S->has_target && e <= S->target) ? 0 : -1;
    if (best_s) memcpy(best_s, s, (size_t)n);
    int64_t nev = 0;
    int64_t K = S->trajectories;
    double T = S->travel;
    for (int64_t k = 0; k < K; ++k) {
        if (k > 0)
            for (int j = 0; j < n; ++j) orc_draw(seed, inst_id, r, (uint32_t)j, (uint32_t)k, NULL, &v[j]);
        double beta = K > 1 ? S->beta0 + (S->beta1 - S->beta0) * (double)k / (double)(K - 1) : S->beta0;
        /* event times of this trajectory, in order (insertion sort: plain and stable) */
        int m = 0;
        for (int j = 0; j < n; ++j) {
            tev[j] = orc_gahmc_cross_time(x[j], v[j], s[j]);
            vnew[j] = 0.0;
            if (tev[j] < T) {
                int p = m++;
                while (p > 0 && (tev[order[p - 1]] > tev[j])) {
                    order[p] = order[p - 1];
                    --p;
                }
                order[p] = j;
            }
        }
        for (int a = 0; a < m; ++a) {
            int j = order[a];
            double A = sqrt(x[j] * x[j] + v[j] * v[j]);      /* speed at the wall */
            int64_t dE = 2 * (int64_t)s[j] * I[j];             /* flip identity (Eqs. 2, 6) */
            double dU = beta * q * (double)dE;
            if (0.5 * A * A > dU) {
                int8_t sn = (int8_t)(-s[j]);
                vnew[j] = (double)sn * sqrt(A * A - 2.0 * dU);  /* moving into the orthant of sn */
                s[j] = sn;
                for (int i = 0; i < n; ++i) {
                    int64_t kij;
                    if (P->k) {
                        kij = P->k[(int64_t)i * n + j];
                    } else {
                        kij = 0;
                        for (int32_t p2 = P->row_ptr[i]; p2 < P->row_ptr[i + 1]; ++p2)
                            if (P->col[p2] == j) kij = P->val[p2];
                    }
                    I[i] += 2 * kij * sn;
                }
                e += dE;
                out->crossings += 1;
                if (events && nev < events_cap) events[nev] = j;
                if (e < out->best_e) {
                    out->best_e = e;
                    out->best_traj = k;
                    if (best_s) memcpy(best_s, s, (size_t)n);
                }
                if (S->has_target && out->hit_traj < 0 && e <= S->target) out->hit_traj = k;
            } else {
                vnew[j] = (double)s[j] * A;                      /* reflected back into its orthant */
                out->reflections += 1;
                if (events && nev < events_cap) events[nev] = -(j + 1);
            }
            ++nev;
        }
        /* every coordinate to the end of the trajectory */
        for (int j = 0; j < n; ++j) {
            if (tev[j] < T) {
                double u = T - tev[j];
                x[j] = vnew[j] * sin(u);
                v[j] = vnew[j] * cos(u);
            } else {
                double xj = x[j] * cos(T) + v[j] * sin(T);
                double vj = -x[j] * sin(T) + v[j] * cos(T);
                x[j] = xj;
                v[j] = vj;
            }
        }
    }
    if (x_out) memcpy(x_out, x, sizeof(double) * (size_t)n);
    if (v_out) memcpy(v_out, v, sizeof(double) * (size_t)n);
    if (s_out) memcpy(s_out, s, (size_t)n);
    free(x); free(v); free(tev); free(vnew); free(order); free(s); free(I);
}
