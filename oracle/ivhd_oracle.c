/*
 * ivhd_oracle.c -- plain, slow FP64 CPU oracle for the IVHD embedding iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two are compared on the same seeded
 * inputs.
 *
 * What it follows (B. Minch, "In search of the most efficient and
 * memory-saving visualization of high dimensional data", 2023):
 *   - binary target distances D_ij in {0, 1}            Sec. 3.3.1, Eq. 3.15
 *   - the IVHD stress over nn and rn pairs              Sec. 3.3.1, Eq. 3.16
 *   - the force as the negative gradient of the stress   Sec. 3.3.1, Eq. 3.14;
 *     Sec. 3.3.3, Eq. 3.32 (see READINGS below)
 *   - the force-directed / momentum update              Sec. 3.3.3, Eq. 3.34;
 *     Sec. 3.3.2, Eq. 3.20
 *   - Nesterov and Adadelta updates                     Sec. 3.3.2
 *   - random neighbours: a vertex connected to i is never its random
 *     neighbour                                        Sec. 3.3.3 (last paragraph)
 *   - the synchronous force-then-update step            Sec. 5.2, simplified
 *     IVHD-CUDA scheme (Algorithm in Sec. 5.2)
 *   - neighbourhood preservation Q_NX(k)                Sec. 4.1 (rank criteria)
 *   - neighbour hit cf_nn                               Sec. 4.1, Eq. 4.4
 *   - placement of new points at the embedding of their
 *     nearest base neighbour(s)                        Sec. 2.4.3 (Progressive UMAP)
 *
 * READINGS where the paper is silent, garbled or inconsistent:
 *   R1  d_ij is the Euclidean norm ||y_i - y_j||_2 (Sec. 3.3 prints a square
 *       root of the norm; Eq. 3.16 and the MDS stress need the plain norm).
 *   R2  The force is F = -1/2 grad E, i.e. the nn term pulls with
 *       -(y_i - y_j) and the rn term pushes with +c (1 - d)/d (y_i - y_k).
 *       Eq. 3.14 / 3.32 print a minus sign on the rn term, which would
 *       attract pairs closer than 1 and contradict the stress c (1 - d)^2.
 *       Constant factors (2, 2 k_nn) are absorbed into b.
 *   R3  Every term acts on both endpoints (Newton's third law, as in the
 *       "positive / negative slot" description of IVHD-CUDA, Sec. 5.2), so F
 *       is the exact gradient of E and sums to zero.
 *   R4  Multiplicity (default): the literal double sum of Eq. 3.16, so a
 *       mutual kNN pair contributes two nn terms.  dedup=1 counts each
 *       unordered nn pair once (an "undirected kNN graph").
 *   R5  Random neighbours are fixed for the whole run, drawn once from
 *       SplitMix64 (below); self, out-kNN, in-kNN and earlier draws are
 *       rejected.
 *   R6  d = 0 in an rn term contributes zero force.
 *   R7  Momentum / Nesterov as descent: v <- a v + b F, y <- y + v
 *       (the printed "+ alpha grad f" would ascend).
 *   R8  Adadelta in Zeiler's form: g = -F, eps inside both RMS terms, both
 *       accumulators start at zero, no learning rate.
 *   R9  Q_NX ties are broken by the lower index (Sec. 4.1 rank definition);
 *       the 2-D distance that decides the neighbour set is taken in FP32 as
 *       dx*dx rounded, then fma(dy, dy, .), the precision of the GPU kernel.
 *   R10 kNN ties are broken by the lower index; the squared distance that
 *       decides the set is the FP32 chain acc = fma(x_d - y_d, x_d - y_d, acc)
 *       over d = 0..N-1 for float data, exact integers for uint8 data.
 *   R11 kNN rows may hold -1 for an absent entry (a vertex with fewer than
 *       k neighbours keeps those it has, Sec. 3.3.3).
 *   R12 A redraw of the random neighbours with epoch e > 0 replaces the seed
 *       s by s ^ mix(e) (mix = the SplitMix64 finaliser).
 *   R13 L1 late stage (Sec. 3.4.1): d = |dx| + |dy| in the stress; the force
 *       is -1/2 of its gradient taken coordinate-wise with sign(0) = 0.
 *   R14 Reverse-neighbour mechanism (Sec. 3.4.2): nn term (i, j) is kept iff
 *       i is among the neighbours of j in the helper graph.
 *   R15 Self-adaptive b (Sec. 3.3.3): dT = sum |v'|^2 - sum |v|^2 over the
 *       candidate step; if |dT| > tau * sum |v|^2 (and sum |v|^2 > 0) the step
 *       is rejected (positions and velocities unchanged) and b is multiplied
 *       by gamma1 (dT < 0) or gamma2 (dT > 0); otherwise it is accepted.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), state advanced by the golden
 * gamma and finalised by the variant-13 mixer.  Output t (t = 0, 1, ...) of
 * the generator seeded with s is mix(s + (t+1) * gamma).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IVO_GAMMA 0x9E3779B97F4A7C15ULL
#define IVO_DOMAIN_RN 0x726E5F6C69737473ULL   /* "rn_lists" */
#define IVO_DOMAIN_INIT 0x696E69745F706F73ULL /* "init_pos" */

static uint64_t ivo_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output number t of SplitMix64 seeded with `seed`. */
uint64_t ivo_splitmix64(uint64_t seed, uint64_t t)
{
    return ivo_mix64(seed + (t + 1) * IVO_GAMMA);
}

/* floor(x * M / 2^64): maps a 64-bit draw onto [0, M). */
static int64_t ivo_range(uint64_t x, int64_t M)
{
    return (int64_t)(((unsigned __int128)x * (unsigned __int128)(uint64_t)M) >> 64);
}

static int ivo_row_has(const int32_t *row, int n, int64_t j)
{
    for (int s = 0; s < n; ++s)
        if (row[s] == j) return 1;
    return 0;
}

/* True when j is i itself or joined to i by a kNN edge in either direction. */
static int ivo_connected(const int32_t *knn, int k, int64_t i, int64_t j)
{
    if (i == j) return 1;
    if (ivo_row_has(knn + i * (int64_t)k, k, j)) return 1;
    if (ivo_row_has(knn + j * (int64_t)k, k, i)) return 1;
    return 0;
}

/*
 * Random neighbours O_rn(i) (Sec. 3.3.1 "generated ad hoc"; Sec. 3.3.3: a
 * vertex connected to i cannot be its random neighbour).
 *
 * For vertex i the draws are x_t = output t of SplitMix64 seeded with
 * s_i = output i of SplitMix64 seeded with (seed ^ "rn_lists"); the candidate
 * is floor(x_t * M / 2^64).  A candidate is kept unless it is i, connected to
 * i, or already kept.  After 64*r draws any still-missing slots are filled by
 * scanning j = 0, 1, ..., M-1 with the same rule; slots that cannot be filled
 * hold -1.  Returns the number of -1 slots written.
 */
int64_t ivo_random_neighbors(const int32_t *knn, int64_t M, int k, int r, uint64_t seed,
                             int32_t *rn)
{
    int64_t empty = 0;
    if (r == 0) return 0;
    for (int64_t i = 0; i < M; ++i) {
        int32_t *row = rn + i * (int64_t)r;
        int got = 0;
        uint64_t s_i = ivo_splitmix64(seed ^ IVO_DOMAIN_RN, (uint64_t)i);
        for (int64_t t = 0; t < 64 * (int64_t)r && got < r; ++t) {
            int64_t j = ivo_range(ivo_splitmix64(s_i, (uint64_t)t), M);
            if (ivo_connected(knn, k, i, j) || ivo_row_has(row, got, j)) continue;
            row[got++] = (int32_t)j;
        }
        for (int64_t j = 0; j < M && got < r; ++j) {
            if (ivo_connected(knn, k, i, j) || ivo_row_has(row, got, j)) continue;
            row[got++] = (int32_t)j;
        }
        for (int s = got; s < r; ++s) {
            row[s] = -1;
            ++empty;
        }
    }
    return empty;
}

/* Random neighbours of draw epoch e (R12); e = 0 is the first draw. */
int64_t ivo_random_neighbors_epoch(const int32_t *knn, int64_t M, int k, int r, uint64_t seed,
                                   uint64_t epoch, int32_t *rn)
{
    uint64_t s = epoch ? (seed ^ ivo_mix64(epoch)) : seed;
    return ivo_random_neighbors(knn, M, k, r, s, rn);
}

/*
 * Reverse-neighbour restriction (R14): out[i][s] = knn[i][s] when i appears in
 * helper row knn[i][s], else -1.
 */
void ivo_restrict(const int32_t *knn, const int32_t *helper, int64_t M, int k, int kh,
                  int32_t *out)
{
    for (int64_t i = 0; i < M; ++i)
        for (int s = 0; s < k; ++s) {
            int32_t j = knn[i * (int64_t)k + s];
            out[i * (int64_t)k + s] = (j >= 0 && ivo_row_has(helper + (int64_t)j * kh, kh, i)) ? j : -1;
        }
}

/*
 * Initial positions y_i ~ U(0,1)^2: with s_i = output i of SplitMix64 seeded
 * with (seed ^ "init_pos"), coordinate q (q = 0, 1) is the top 24 bits of
 * output q of SplitMix64 seeded with s_i, times 2^-24.
 */
void ivo_init_positions(int64_t M, uint64_t seed, double *Y)
{
    for (int64_t i = 0; i < M; ++i) {
        uint64_t s_i = ivo_splitmix64(seed ^ IVO_DOMAIN_INIT, (uint64_t)i);
        for (int q = 0; q < 2; ++q) {
            uint64_t x = ivo_splitmix64(s_i, (uint64_t)q);
            Y[2 * i + q] = (double)(x >> 40) * (1.0 / 16777216.0);
        }
    }
}

/*
 * The term list of Eq. 3.16: one nn term per kNN entry (i, j) and one rn term
 * per kept random neighbour (i, k).  kind[t] = 0 for nn, 1 for rn.
 * dedup = 0 keeps multiplicity (R4); dedup = 1 keeps a mutual nn pair only in
 * the row of its lower-index endpoint.  Arrays must hold M*(k+r) entries.
 * Returns the number of terms.
 */
int64_t ivo_build_terms(const int32_t *knn, const int32_t *rn, int64_t M, int k, int r,
                        int dedup, int64_t *ti, int64_t *tj, int8_t *kind)
{
    int64_t T = 0;
    for (int64_t i = 0; i < M; ++i) {
        for (int s = 0; s < k; ++s) {
            int64_t j = knn[i * (int64_t)k + s];
            if (j < 0) continue;
            if (dedup && j < i && ivo_row_has(knn + j * (int64_t)k, k, i)) continue;
            ti[T] = i;
            tj[T] = j;
            kind[T] = 0;
            ++T;
        }
        for (int s = 0; s < r; ++s) {
            int64_t j = rn[i * (int64_t)r + s];
            if (j < 0) continue;
            ti[T] = i;
            tj[T] = j;
            kind[T] = 1;
            ++T;
        }
    }
    return T;
}

/* Euclidean distance between rows i and j of Y (R1). */
static double ivo_dist(const double *Y, int64_t i, int64_t j)
{
    double dx = Y[2 * i] - Y[2 * j];
    double dy = Y[2 * i + 1] - Y[2 * j + 1];
    return sqrt(dx * dx + dy * dy);
}

/* Stress E of Eq. 3.16: sum of d^2 over nn terms plus c (1 - d)^2 over rn terms. */
double ivo_stress(const double *Y, const int64_t *ti, const int64_t *tj, const int8_t *kind,
                  int64_t T, double c)
{
    double E = 0.0;
    for (int64_t t = 0; t < T; ++t) {
        double d = ivo_dist(Y, ti[t], tj[t]);
        if (kind[t] == 0)
            E += d * d;
        else
            E += c * (1.0 - d) * (1.0 - d);
    }
    return E;
}

/*
 * F = -1/2 grad E (R2, R3).  nn term (i, j): F_i -= (y_i - y_j), F_j += (y_i - y_j).
 * rn term (i, k) with u = y_i - y_k, d = |u|: g = c (1 - d) / d * u,
 * F_i += g, F_k -= g; zero when d = 0 (R6).
 */
void ivo_forces(const double *Y, int64_t M, const int64_t *ti, const int64_t *tj,
                const int8_t *kind, int64_t T, double c, double *F)
{
    memset(F, 0, sizeof(double) * 2 * (size_t)M);
    for (int64_t t = 0; t < T; ++t) {
        int64_t i = ti[t], j = tj[t];
        double ux = Y[2 * i] - Y[2 * j];
        double uy = Y[2 * i + 1] - Y[2 * j + 1];
        double gx, gy;
        if (kind[t] == 0) {
            gx = -ux;
            gy = -uy;
        } else {
            double d = sqrt(ux * ux + uy * uy);
            if (d == 0.0) continue;
            double s = c * (1.0 - d) / d;
            gx = s * ux;
            gy = s * uy;
        }
        F[2 * i] += gx;
        F[2 * i + 1] += gy;
        F[2 * j] -= gx;
        F[2 * j + 1] -= gy;
    }
}

/*
 * One synchronous step (all forces from the same configuration, then all
 * updates; Sec. 5.2 scheme).  opt: 0 momentum / force-directed (Eq. 3.34),
 * 1 Nesterov (Sec. 3.3.2), 2 Adadelta (Sec. 3.3.2, R8).
 * S1 = velocity (opt 0, 1) or E[g^2] (opt 2); S2 = E[dx^2] (opt 2 only).
 * F and W are caller scratch of 2*M doubles each.
 */
void ivo_step(int opt, double *Y, double *S1, double *S2, int64_t M, const int64_t *ti,
              const int64_t *tj, const int8_t *kind, int64_t T, double c, double a, double b,
              double rho, double eps, double *F, double *W)
{
    int64_t n = 2 * M;
    if (opt == 0) {
        ivo_forces(Y, M, ti, tj, kind, T, c, F);
        for (int64_t q = 0; q < n; ++q) {
            S1[q] = a * S1[q] + b * F[q];
            Y[q] += S1[q];
        }
    } else if (opt == 1) {
        for (int64_t q = 0; q < n; ++q) W[q] = Y[q] + a * S1[q];
        ivo_forces(W, M, ti, tj, kind, T, c, F);
        for (int64_t q = 0; q < n; ++q) {
            S1[q] = a * S1[q] + b * F[q];
            Y[q] += S1[q];
        }
    } else {
        ivo_forces(Y, M, ti, tj, kind, T, c, F);
        for (int64_t q = 0; q < n; ++q) {
            double g = -F[q];
            S1[q] = rho * S1[q] + (1.0 - rho) * g * g;
            double dx = -sqrt(S2[q] + eps) / sqrt(S1[q] + eps) * g;
            S2[q] = rho * S2[q] + (1.0 - rho) * dx * dx;
            Y[q] += dx;
        }
    }
}

static double ivo_sgn(double u) { return (double)((u > 0.0) - (u < 0.0)); }

/* Stress with the L1 distance (R13). */
double ivo_stress_l1(const double *Y, const int64_t *ti, const int64_t *tj, const int8_t *kind,
                     int64_t T, double c)
{
    double E = 0.0;
    for (int64_t t = 0; t < T; ++t) {
        int64_t i = ti[t], j = tj[t];
        double d = fabs(Y[2 * i] - Y[2 * j]) + fabs(Y[2 * i + 1] - Y[2 * j + 1]);
        E += (kind[t] == 0) ? d * d : c * (1.0 - d) * (1.0 - d);
    }
    return E;
}

/*
 * F = -1/2 grad of the L1 stress (R13).  With u = y_i - y_j and d = |u_x| + |u_y|:
 * nn term: F_i -= d sign(u), F_j += d sign(u); rn term: g = c (1 - d) sign(u),
 * F_i += g, F_j -= g.
 */
void ivo_forces_l1(const double *Y, int64_t M, const int64_t *ti, const int64_t *tj,
                   const int8_t *kind, int64_t T, double c, double *F)
{
    memset(F, 0, sizeof(double) * 2 * (size_t)M);
    for (int64_t t = 0; t < T; ++t) {
        int64_t i = ti[t], j = tj[t];
        double ux = Y[2 * i] - Y[2 * j], uy = Y[2 * i + 1] - Y[2 * j + 1];
        double d = fabs(ux) + fabs(uy);
        double s = (kind[t] == 0) ? -d : c * (1.0 - d);
        double gx = s * ivo_sgn(ux), gy = s * ivo_sgn(uy);
        F[2 * i] += gx;
        F[2 * i + 1] += gy;
        F[2 * j] -= gx;
        F[2 * j + 1] -= gy;
    }
}

/*
 * One attempt of a momentum (opt 0) or Nesterov (opt 1) step with the
 * self-adaptive b of R15, metric 0 = L2, 1 = L1.  Y, V are updated only when
 * the step is accepted; *b is scaled when it is rejected.  Returns 1 when
 * accepted, 0 when rejected.  F, W, Yn, Vn are caller scratch of 2*M doubles.
 */
int ivo_step_adaptive(int opt, int metric, double *Y, double *V, int64_t M, const int64_t *ti,
                      const int64_t *tj, const int8_t *kind, int64_t T, double c, double a,
                      double *b, double tau, double gamma1, double gamma2, double *F, double *W,
                      double *Yn, double *Vn)
{
    int64_t n = 2 * M;
    const double *at = Y;
    if (opt == 1) {
        for (int64_t q = 0; q < n; ++q) W[q] = Y[q] + a * V[q];
        at = W;
    }
    if (metric == 1)
        ivo_forces_l1(at, M, ti, tj, kind, T, c, F);
    else
        ivo_forces(at, M, ti, tj, kind, T, c, F);
    double told = 0.0, tnew = 0.0;
    for (int64_t q = 0; q < n; ++q) {
        Vn[q] = a * V[q] + *b * F[q];
        Yn[q] = Y[q] + Vn[q];
        told += V[q] * V[q];
        tnew += Vn[q] * Vn[q];
    }
    double dT = tnew - told;
    if (told > 0.0 && fabs(dT) > tau * told) {
        *b *= (dT < 0.0) ? gamma1 : gamma2;
        return 0;
    }
    memcpy(Y, Yn, sizeof(double) * (size_t)n);
    memcpy(V, Vn, sizeof(double) * (size_t)n);
    return 1;
}

/* Momentum / Nesterov step with the L1 forces (R13); same state as ivo_step. */
void ivo_step_l1(int opt, double *Y, double *V, int64_t M, const int64_t *ti, const int64_t *tj,
                 const int8_t *kind, int64_t T, double c, double a, double b, double *F, double *W)
{
    int64_t n = 2 * M;
    const double *at = Y;
    if (opt == 1) {
        for (int64_t q = 0; q < n; ++q) W[q] = Y[q] + a * V[q];
        at = W;
    }
    ivo_forces_l1(at, M, ti, tj, kind, T, c, F);
    for (int64_t q = 0; q < n; ++q) {
        V[q] = a * V[q] + b * F[q];
        Y[q] += V[q];
    }
}

/* n_iter steps of ivo_step; scratch is allocated here.  Returns 0, or -1 on OOM. */
int ivo_run(int opt, double *Y, double *S1, double *S2, int64_t M, const int64_t *ti,
            const int64_t *tj, const int8_t *kind, int64_t T, double c, double a, double b,
            double rho, double eps, int64_t n_iter)
{
    double *F = (double *)malloc(sizeof(double) * 2 * (size_t)M);
    double *W = (double *)malloc(sizeof(double) * 2 * (size_t)M);
    if (!F || !W) {
        free(F);
        free(W);
        return -1;
    }
    for (int64_t it = 0; it < n_iter; ++it)
        ivo_step(opt, Y, S1, S2, M, ti, tj, kind, T, c, a, b, rho, eps, F, W);
    free(F);
    free(W);
    return 0;
}

/*
 * ivo_run on n_threads host threads (the multi-core CPU timing of the same
 * oracle; POSIX threads).  Every step runs the phases of ivo_step with the
 * same arithmetic: thread t sums the forces of its contiguous share of the
 * term list into its own buffer, then F = sum over t of those buffers, added
 * in thread order for every coordinate, and each thread updates its share of
 * the coordinates.  Only the order in which the terms' contributions are
 * added differs from ivo_run; with one thread the result is bit for bit
 * ivo_run's.  Returns 0, or -1 on OOM or a failed thread start.
 */
/* Start gate of the worker threads: 0 = wait, 1 = run, 2 = return at once. */
typedef struct {
    pthread_mutex_t mu;
    pthread_cond_t cv;
    int state;
} ivo_gate;

typedef struct {
    int opt, t, nt;
    double *Y, *S1, *S2, *F, *W, *Fp;
    int64_t M, T, n_iter;
    const int64_t *ti, *tj;
    const int8_t *kind;
    double c, a, b, rho, eps;
    pthread_barrier_t *bar;
    ivo_gate *gate;
} ivo_thread_arg;

static void *ivo_thread_main(void *p)
{
    ivo_thread_arg *A = (ivo_thread_arg *)p;
    if (A->t > 0) {
        pthread_mutex_lock(&A->gate->mu);
        while (A->gate->state == 0) pthread_cond_wait(&A->gate->cv, &A->gate->mu);
        int go = A->gate->state == 1;
        pthread_mutex_unlock(&A->gate->mu);
        if (!go) return NULL;
    }
    int64_t n = 2 * A->M;
    int64_t q0 = n * A->t / A->nt, q1 = n * (A->t + 1) / A->nt;
    int64_t t0 = A->T * A->t / A->nt, t1 = A->T * (A->t + 1) / A->nt;
    double *Fmine = A->Fp + (size_t)A->t * (size_t)n;
    for (int64_t it = 0; it < A->n_iter; ++it) {
        const double *Yf = A->Y;
        if (A->opt == 1) {
            for (int64_t q = q0; q < q1; ++q) A->W[q] = A->Y[q] + A->a * A->S1[q];
            pthread_barrier_wait(A->bar);
            Yf = A->W;
        }
        ivo_forces(Yf, A->M, A->ti + t0, A->tj + t0, A->kind + t0, t1 - t0, A->c, Fmine);
        pthread_barrier_wait(A->bar);
        for (int64_t q = q0; q < q1; ++q) {
            double f = 0.0;
            for (int u = 0; u < A->nt; ++u) f += A->Fp[(size_t)u * (size_t)n + (size_t)q];
            A->F[q] = f;
        }
        for (int64_t q = q0; q < q1; ++q) {
            if (A->opt != 2) {
                A->S1[q] = A->a * A->S1[q] + A->b * A->F[q];
                A->Y[q] += A->S1[q];
            } else {
                double g = -A->F[q];
                A->S1[q] = A->rho * A->S1[q] + (1.0 - A->rho) * g * g;
                double dx = -sqrt(A->S2[q] + A->eps) / sqrt(A->S1[q] + A->eps) * g;
                A->S2[q] = A->rho * A->S2[q] + (1.0 - A->rho) * dx * dx;
                A->Y[q] += dx;
            }
        }
        pthread_barrier_wait(A->bar);
    }
    return NULL;
}

int ivo_run_threads(int opt, double *Y, double *S1, double *S2, int64_t M, const int64_t *ti,
                    const int64_t *tj, const int8_t *kind, int64_t T, double c, double a,
                    double b, double rho, double eps, int64_t n_iter, int n_threads)
{
    if (n_threads < 1) return -1;
    size_t n = 2 * (size_t)M;
    double *F = (double *)malloc(sizeof(double) * n);
    double *W = (double *)malloc(sizeof(double) * n);
    double *Fp = (double *)malloc(sizeof(double) * n * (size_t)n_threads);
    ivo_thread_arg *args = (ivo_thread_arg *)malloc(sizeof(ivo_thread_arg) * (size_t)n_threads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    ivo_gate gate = {PTHREAD_MUTEX_INITIALIZER, PTHREAD_COND_INITIALIZER, 0};
    pthread_barrier_t bar;
    int rc = -1, started = 0;
    if (!F || !W || !Fp || !args || !th) goto out;
    if (pthread_barrier_init(&bar, NULL, (unsigned)n_threads) != 0) goto out;
    for (int t = 0; t < n_threads; ++t) {
        ivo_thread_arg A = {opt, t, n_threads, Y, S1, S2, F, W, Fp, M, T, n_iter,
                            ti, tj, kind, c, a, b, rho, eps, &bar, &gate};
        args[t] = A;
    }
    /* share 0 runs on the calling thread; the others wait at the gate until
       every thread has started, so a failed start stops them all */
    for (int t = 1; t < n_threads; ++t) {
        if (pthread_create(&th[t], NULL, ivo_thread_main, &args[t]) != 0) break;
        ++started;
    }
    pthread_mutex_lock(&gate.mu);
    gate.state = (started == n_threads - 1) ? 1 : 2;
    pthread_cond_broadcast(&gate.cv);
    pthread_mutex_unlock(&gate.mu);
    if (gate.state == 1) {
        ivo_thread_main(&args[0]);
        rc = 0;
    }
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    pthread_barrier_destroy(&bar);
out:
    free(F);
    free(W);
    free(Fp);
    free(args);
    free(th);
    return rc;
}

/* Insert (d, j) into a list of n best (ascending d, ties by lower j) of capacity k. */
static void ivo_topk_insert_f(float *bd, int32_t *bj, int *n, int k, float d, int32_t j)
{
    int pos = *n;
    while (pos > 0 && (bd[pos - 1] > d || (bd[pos - 1] == d && bj[pos - 1] > j))) --pos;
    if (pos >= k) return;
    int last = (*n < k) ? *n : k - 1;
    for (int s = last; s > pos; --s) {
        bd[s] = bd[s - 1];
        bj[s] = bj[s - 1];
    }
    bd[pos] = d;
    bj[pos] = j;
    if (*n < k) ++*n;
}

static void ivo_topk_insert_i(int64_t *bd, int32_t *bj, int *n, int k, int64_t d, int32_t j)
{
    int pos = *n;
    while (pos > 0 && (bd[pos - 1] > d || (bd[pos - 1] == d && bj[pos - 1] > j))) --pos;
    if (pos >= k) return;
    int last = (*n < k) ? *n : k - 1;
    for (int s = last; s > pos; --s) {
        bd[s] = bd[s - 1];
        bj[s] = bj[s - 1];
    }
    bd[pos] = d;
    bj[pos] = j;
    if (*n < k) ++*n;
}

/*
 * Exact kNN of float rows (R10): for each query q in `rows` (all rows when
 * rows == NULL), the k nearest other rows by the FP32 sequential squared
 * distance, ascending, ties by lower index.  out is nrows x k.
 */
int ivo_knn_f32(const float *X, int64_t M, int N, int k, const int64_t *rows, int64_t nrows,
                int32_t *out)
{
    if (k < 1 || k > M - 1) return -1;
    float *bd = (float *)malloc(sizeof(float) * (size_t)k);
    if (!bd) return -1;
    int64_t nq = rows ? nrows : M;
    for (int64_t qi = 0; qi < nq; ++qi) {
        int64_t q = rows ? rows[qi] : qi;
        int32_t *bj = out + qi * (int64_t)k;
        int n = 0;
        const float *xq = X + q * (int64_t)N;
        for (int64_t j = 0; j < M; ++j) {
            if (j == q) continue;
            const float *xj = X + j * (int64_t)N;
            float acc = 0.0f;
            for (int d = 0; d < N; ++d) {
                float diff = xq[d] - xj[d];
                acc = fmaf(diff, diff, acc);
            }
            ivo_topk_insert_f(bd, bj, &n, k, acc, (int32_t)j);
        }
    }
    free(bd);
    return 0;
}

/* Exact kNN of uint8 rows with integer squared distances (R10). */
int ivo_knn_u8(const uint8_t *X, int64_t M, int N, int k, const int64_t *rows, int64_t nrows,
               int32_t *out)
{
    if (k < 1 || k > M - 1) return -1;
    int64_t *bd = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (!bd) return -1;
    int64_t nq = rows ? nrows : M;
    for (int64_t qi = 0; qi < nq; ++qi) {
        int64_t q = rows ? rows[qi] : qi;
        int32_t *bj = out + qi * (int64_t)k;
        int n = 0;
        const uint8_t *xq = X + q * (int64_t)N;
        for (int64_t j = 0; j < M; ++j) {
            if (j == q) continue;
            const uint8_t *xj = X + j * (int64_t)N;
            int64_t acc = 0;
            for (int d = 0; d < N; ++d) {
                int64_t diff = (int64_t)xq[d] - (int64_t)xj[d];
                acc += diff * diff;
            }
            ivo_topk_insert_i(bd, bj, &n, k, acc, (int32_t)j);
        }
    }
    free(bd);
    return 0;
}

/*
 * Exact kNN of query rows against a separate base set: the nearest-neighbour
 * search of the Progressive UMAP placement (Sec. 2.4.3, Progressive UMAP
 * scheme), made exact.  For each of the Mq queries, the k base rows nearest by
 * the same FP32 sequential squared distance as ivo_knn_f32 (uint8: the exact
 * integer distance), ascending, ties by lower index.  No row is excluded: a
 * query equal to a base row finds it at distance 0.  out is Mq x k.
 */
int ivo_knn_query_f32(const float *Q, int64_t Mq, const float *X, int64_t M, int N, int k,
                      int32_t *out)
{
    if (k < 1 || k > M) return -1;
    float *bd = (float *)malloc(sizeof(float) * (size_t)k);
    if (!bd) return -1;
    for (int64_t q = 0; q < Mq; ++q) {
        int32_t *bj = out + q * (int64_t)k;
        int n = 0;
        const float *xq = Q + q * (int64_t)N;
        for (int64_t j = 0; j < M; ++j) {
            const float *xj = X + j * (int64_t)N;
            float acc = 0.0f;
            for (int d = 0; d < N; ++d) {
                float diff = xq[d] - xj[d];
                acc = fmaf(diff, diff, acc);
            }
            ivo_topk_insert_f(bd, bj, &n, k, acc, (int32_t)j);
        }
    }
    free(bd);
    return 0;
}

int ivo_knn_query_u8(const uint8_t *Q, int64_t Mq, const uint8_t *X, int64_t M, int N, int k,
                     int32_t *out)
{
    if (k < 1 || k > M) return -1;
    int64_t *bd = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (!bd) return -1;
    for (int64_t q = 0; q < Mq; ++q) {
        int32_t *bj = out + q * (int64_t)k;
        int n = 0;
        const uint8_t *xq = Q + q * (int64_t)N;
        for (int64_t j = 0; j < M; ++j) {
            const uint8_t *xj = X + j * (int64_t)N;
            int64_t acc = 0;
            for (int d = 0; d < N; ++d) {
                int64_t diff = (int64_t)xq[d] - (int64_t)xj[d];
                acc += diff * diff;
            }
            ivo_topk_insert_i(bd, bj, &n, k, acc, (int32_t)j);
        }
    }
    free(bd);
    return 0;
}

/*
 * Placement of new points from the embedding Y of their base neighbours:
 * y_q = (1/k) sum_s Y[ids[q][s]] in FP64.  k = 1 is the Progressive UMAP
 * initialisation (a new point starts at the embedding of its nearest
 * neighbour, Sec. 2.4.3).  out is n x 2.
 */
void ivo_place_nn(const float *Y, const int32_t *ids, int64_t n, int k, double *out)
{
    for (int64_t q = 0; q < n; ++q) {
        double sx = 0.0, sy = 0.0;
        for (int s = 0; s < k; ++s) {
            int64_t j = ids[q * (int64_t)k + s];
            sx += (double)Y[2 * j];
            sy += (double)Y[2 * j + 1];
        }
        out[2 * q] = sx / k;
        out[2 * q + 1] = sy / k;
    }
}

/* The FP32 2-D squared distance that decides low-dimensional neighbours (R9). */
static float ivo_d2_f32(const float *Y, int64_t i, int64_t j)
{
    float dx = Y[2 * j] - Y[2 * i];
    float dy = Y[2 * j + 1] - Y[2 * i + 1];
    float p = dx * dx;
    return fmaf(dy, dy, p);
}

/* The kk nearest other points of row q in the 2-D embedding Y (R9). */
static void ivo_lowd_knn(const float *Y, int64_t M, int64_t q, int kk, float *bd, int32_t *bj)
{
    int n = 0;
    for (int64_t j = 0; j < M; ++j) {
        if (j == q) continue;
        ivo_topk_insert_f(bd, bj, &n, kk, ivo_d2_f32(Y, q, j), (int32_t)j);
    }
}

/*
 * Hits of Q_NX(k) (Sec. 4.1) over sampled rows qi in [r0, r1): for each, the
 * k nearest other points n_i of y_i in the embedding, and |v_i ∩ n_i| with
 * v_i the given high-dimensional kNN row.  lowd_out (optional) receives n_i
 * at row qi.  bd, bj: scratch of k entries.
 */
static int64_t ivo_qnx_hits(const float *Y, int64_t M, const int32_t *knn, int k,
                            const int64_t *rows, int64_t r0, int64_t r1, int32_t *lowd_out,
                            float *bd, int32_t *bj)
{
    int64_t hits = 0;
    for (int64_t qi = r0; qi < r1; ++qi) {
        int64_t q = rows ? rows[qi] : qi;
        ivo_lowd_knn(Y, M, q, k, bd, bj);
        for (int s = 0; s < k; ++s) {
            if (lowd_out) lowd_out[qi * (int64_t)k + s] = bj[s];
            if (ivo_row_has(knn + q * (int64_t)k, k, bj[s])) ++hits;
        }
    }
    return hits;
}

/* Hits of cf_nn (Sec. 4.1, Eq. 4.4) over sampled rows qi in [r0, r1). */
static int64_t ivo_cf_hits(const float *Y, int64_t M, const int32_t *labels, int nn,
                           const int64_t *rows, int64_t r0, int64_t r1, float *bd, int32_t *bj)
{
    int64_t hits = 0;
    for (int64_t qi = r0; qi < r1; ++qi) {
        int64_t q = rows ? rows[qi] : qi;
        ivo_lowd_knn(Y, M, q, nn, bd, bj);
        for (int s = 0; s < nn; ++s)
            if (labels[bj[s]] == labels[q]) ++hits;
    }
    return hits;
}

/*
 * Q_NX(k) (Sec. 4.1): the mean over the sampled rows of |v_i ∩ n_i| / k,
 * where v_i is the given high-dimensional kNN row and n_i the k nearest
 * points of y_i in the embedding.  lowd_out (optional, nrows x k) receives n_i.
 */
double ivo_qnx(const float *Y, int64_t M, const int32_t *knn, int k, const int64_t *rows,
               int64_t nrows, int32_t *lowd_out)
{
    float *bd = (float *)malloc(sizeof(float) * (size_t)k);
    int32_t *bj = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    if (!bd || !bj) {
        free(bd);
        free(bj);
        return -1.0;
    }
    int64_t nq = rows ? nrows : M;
    int64_t hits = ivo_qnx_hits(Y, M, knn, k, rows, 0, nq, lowd_out, bd, bj);
    free(bd);
    free(bj);
    return (double)hits / ((double)k * (double)nq);
}

/*
 * Neighbour hit cf_nn (Sec. 4.1, Eq. 4.4): the fraction of the nn nearest
 * embedded neighbours of each sampled point that share its class label.
 */
double ivo_cf(const float *Y, int64_t M, const int32_t *labels, int nn, const int64_t *rows,
              int64_t nrows)
{
    float *bd = (float *)malloc(sizeof(float) * (size_t)nn);
    int32_t *bj = (int32_t *)malloc(sizeof(int32_t) * (size_t)nn);
    if (!bd || !bj) {
        free(bd);
        free(bj);
        return -1.0;
    }
    int64_t nq = rows ? nrows : M;
    int64_t hits = ivo_cf_hits(Y, M, labels, nn, rows, 0, nq, bd, bj);
    free(bd);
    free(bj);
    return (double)hits / ((double)nn * (double)nq);
}

/*
 * The same two criteria on several host threads, for the large sampled sets
 * of full-size runs: thread t counts the hits of the t-th contiguous share of
 * the sampled rows exactly as above, and the integer hit counts are added, so
 * the result equals the serial one exactly for any number of threads.
 */
typedef struct {
    const float *Y;
    int64_t M;
    const int32_t *knn, *labels;
    int k;
    const int64_t *rows;
    int64_t r0, r1;
    int32_t *lowd_out;
    int64_t hits;
    int rc;
} ivo_eval_arg;

static void *ivo_eval_main(void *p)
{
    ivo_eval_arg *A = (ivo_eval_arg *)p;
    float *bd = (float *)malloc(sizeof(float) * (size_t)A->k);
    int32_t *bj = (int32_t *)malloc(sizeof(int32_t) * (size_t)A->k);
    A->rc = -1;
    if (bd && bj) {
        A->hits = A->labels
                      ? ivo_cf_hits(A->Y, A->M, A->labels, A->k, A->rows, A->r0, A->r1, bd, bj)
                      : ivo_qnx_hits(A->Y, A->M, A->knn, A->k, A->rows, A->r0, A->r1,
                                     A->lowd_out, bd, bj);
        A->rc = 0;
    }
    free(bd);
    free(bj);
    return NULL;
}

static double ivo_eval_threads(const float *Y, int64_t M, const int32_t *knn,
                               const int32_t *labels, int k, const int64_t *rows, int64_t nrows,
                               int32_t *lowd_out, int n_threads)
{
    if (n_threads < 1) return -1.0;
    int64_t nq = rows ? nrows : M;
    ivo_eval_arg *args = (ivo_eval_arg *)malloc(sizeof(ivo_eval_arg) * (size_t)n_threads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    char *started = (char *)calloc((size_t)n_threads, 1);
    double out = -1.0;
    if (!args || !th || !started) goto done;
    for (int t = 0; t < n_threads; ++t) {
        ivo_eval_arg A = {Y, M, knn, labels, k, rows, nq * t / n_threads,
                          nq * (t + 1) / n_threads, lowd_out, 0, -1};
        args[t] = A;
    }
    for (int t = 1; t < n_threads; ++t)
        started[t] = pthread_create(&th[t], NULL, ivo_eval_main, &args[t]) == 0;
    ivo_eval_main(&args[0]);
    for (int t = 1; t < n_threads; ++t) {
        if (started[t])
            pthread_join(th[t], NULL);
        else
            ivo_eval_main(&args[t]);  /* a share whose thread did not start runs here */
    }
    int64_t hits = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (args[t].rc != 0) goto done;
        hits += args[t].hits;
    }
    out = (double)hits / ((double)k * (double)nq);
done:
    free(args);
    free(th);
    free(started);
    return out;
}

double ivo_qnx_threads(const float *Y, int64_t M, const int32_t *knn, int k, const int64_t *rows,
                       int64_t nrows, int32_t *lowd_out, int n_threads)
{
    return ivo_eval_threads(Y, M, knn, NULL, k, rows, nrows, lowd_out, n_threads);
}

double ivo_cf_threads(const float *Y, int64_t M, const int32_t *labels, int nn,
                      const int64_t *rows, int64_t nrows, int n_threads)
{
    return ivo_eval_threads(Y, M, NULL, labels, nn, rows, nrows, NULL, n_threads);
}
