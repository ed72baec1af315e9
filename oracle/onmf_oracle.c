/*
 * FP64 CPU oracle for online and batch IS-NMF (Lefevre, Bach, Fevotte,
 * "Online algorithms for Nonnegative Matrix Factorization with the
 * Itakura-Saito divergence", arXiv:1106.4198).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA path is checked against. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header, table
 * or helper with the CUDA library; neither includes nor links the other.
 *
 * Conventions: every matrix is column-major. V is F x N (frame = column,
 * leading dimension ldv >= F), W and A, B are F x K (ld = F), H is K x N
 * (ld = K). All arithmetic is IEEE double; V arrives as float (the precision
 * the data is stored in) and is widened on read.
 *
 * Readings of the paper that the code takes (the paper is silent or
 * ambiguous at these points):
 *   - h update: the majorization-minimization multiplicative update with
 *     exponent gamma (default 1/2), h_k <- h_k * ((W^T p)_k/(W^T q)_k)^gamma,
 *     where p = y/x^2, q = 1/x. Section 2.1 only says "similar updates can be
 *     found for h_n"; gamma = 1/2 is the MM exponent for IS, gamma = 1 the
 *     heuristic multiplicative update.
 *   - h start point of a fresh restart (Section 2.3, "Fresh or warm
 *     restarts"): h0_k = sum_f y_f / sum_{f,k} W_fk for every k.
 *   - forgetting factor (Algorithm 1, eq. in "Scaling past data"): the past is
 *     scaled, A <- rho*A + sum a, with rho = r^(beta'/n_ref) (rho = 1 when
 *     n_ref <= 0). The literal form A <- A + rho*sum a is selectable.
 *   - guards: a W entry with B_fk = 0, an h entry with (W^T q)_k = 0 and a
 *     column with s_k = 0 are left unchanged.
 *   - the statistics a, b of a minibatch use the final h of each frame and the
 *     W that the h-solve used (Algorithm 1).
 *   - penalties (Section 2.2, "Extensions", which names the two kinds but gives
 *     no updates): on h, lambda * psi(sum_k h_k) with psi(s) = log(a + s),
 *     majorized by its tangent (a linear term in the h update's denominator);
 *     on W, the linear mu * sum W, which turns the dictionary step into
 *     sqrt(A/(B + mu)). lambda = mu = 0 is the plain algorithm. The projection
 *     (or_project) uses the same penalized h-solve; the batch functions are
 *     unpenalized.
 *
 * Parity status: every function here is pinned by tests against closed
 * forms, brute force and identities (d_IS properties, K = 1 closed-form
 * trajectory, block-diagonal W, F = K = 2 brute force, monotone descent,
 * the sqrt(A/B) minimizer, the online-equals-batch identity, power-of-two
 * scale equivariance, the noiseless fixed point, order invariance; for the
 * penalties the K = 1 stationary point in closed form, an F = K = 2 grid
 * minimum, descent of the penalized objective and the penalized dictionary
 * step's minimizer).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

/* Number of host threads used for the per-frame h-solves and per-row
 * statistics (the arithmetic of each output is unchanged). */
void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int or_get_threads(void) { return g_threads; }

int or_have_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* ratio^gamma with the two common exponents taken exactly */
static double powg(double ratio, double gamma) {
    if (gamma == 0.5) return sqrt(ratio);
    if (gamma == 1.0) return ratio;
    return pow(ratio, gamma);
}

/* Itakura-Saito divergence, Section 2.1:
 *   d_IS(y, x) = sum_i ( y_i/x_i - log(y_i/x_i) - 1 ). */
double or_dis(const double *y, const double *x, int64_t n) {
    double d = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = y[i] / x[i];
        d += (r - 1.0) - log(r);
    }
    return d;
}

/* Objective of Eq. (is_nmf) with the epsilon smoothing of Section 2.3:
 *   (1/N) sum_n d_IS(eps + v_n, eps + W h_n). */
double or_objective(int F, int K, int64_t N, const float *V, int64_t ldv,
                    const double *W, const double *H, double eps) {
    double total = 0.0;
    double *y = (double *)malloc(sizeof(double) * F);
    double *x = (double *)malloc(sizeof(double) * F);
    for (int64_t n = 0; n < N; ++n) {
        for (int f = 0; f < F; ++f) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += W[f + (int64_t)k * F] * H[k + n * K];
            x[f] = eps + acc;
            y[f] = eps + (double)V[f + n * ldv];
        }
        total += or_dis(y, x, F);
    }
    free(y);
    free(x);
    return N > 0 ? total / (double)N : 0.0;
}

/* h-solve of Algorithm 1, h_t <- argmin_h d_IS(eps + v_t, eps + W h), run as
 * n_in majorization-minimization steps from the fresh-restart point, with the
 * optional penalty on h of Section 2.2 ("Extensions"), lambda * psi(sum_k h_k)
 * with the concave increasing psi(s) = log(a + s). The concave penalty is
 * majorized by its tangent at the current h, a linear term
 * lambda * psi'(s~) * sum_k h_k, whose gradient joins the positive part of the
 * IS gradient in the update's denominator:
 *   h_k <- h_k * ((W^T p)_k / ((W^T q)_k + lambda / (a + s~)))^gamma,
 * s~ = sum_k h_k before the step (lambda = 0: the plain update).
 *   v: F frame values; W: F x K; h: K outputs.
 *   h_init: if non-NULL, start from it (warm start / batch H step) instead of
 *           the fresh-restart point.
 *   trace: if non-NULL, n_in + 1 entries: the objective d_IS(y, eps + W h)
 *          (+ lambda * log(a + sum_k h_k)) before the first step and after
 *          each step. */
void or_hsolve_pen(int F, int K, const double *W, const float *v, double eps,
                   double gamma, int n_in, double lambda, double a_pen,
                   const double *h_init, double *h, double *trace) {
    double *y = (double *)malloc(sizeof(double) * F);
    double *x = (double *)malloc(sizeof(double) * F);
    double *p = (double *)malloc(sizeof(double) * F);
    double *q = (double *)malloc(sizeof(double) * F);
    for (int f = 0; f < F; ++f) y[f] = eps + (double)v[f];
    if (h_init) {
        for (int k = 0; k < K; ++k) h[k] = h_init[k];
    } else {
        double sy = 0.0, sw = 0.0;
        for (int f = 0; f < F; ++f) sy += y[f];
        for (int k = 0; k < K; ++k)
            for (int f = 0; f < F; ++f) sw += W[f + (int64_t)k * F];
        double h0 = sy / sw;
        for (int k = 0; k < K; ++k) h[k] = h0;
    }
    for (int it = 0; it <= n_in; ++it) {
        /* x = eps + W h */
        for (int f = 0; f < F; ++f) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += W[f + (int64_t)k * F] * h[k];
            x[f] = eps + acc;
        }
        double hs = 0.0; /* s~ = sum_k h_k of the current h */
        for (int k = 0; k < K; ++k) hs += h[k];
        if (trace) trace[it] = or_dis(y, x, F) + (lambda > 0.0 ? lambda * log(a_pen + hs) : 0.0);
        if (it == n_in) break;
        /* p = y / x^2, q = 1 / x */
        for (int f = 0; f < F; ++f) {
            q[f] = 1.0 / x[f];
            p[f] = y[f] / (x[f] * x[f]);
        }
        /* h_k <- h_k * ((W^T p)_k / ((W^T q)_k + lambda psi'(s~)))^gamma */
        const double pen = lambda > 0.0 ? lambda / (a_pen + hs) : 0.0;
        for (int k = 0; k < K; ++k) {
            double num = 0.0, den = 0.0;
            for (int f = 0; f < F; ++f) {
                num += W[f + (int64_t)k * F] * p[f];
                den += W[f + (int64_t)k * F] * q[f];
            }
            den += pen;
            if (den > 0.0) h[k] = h[k] * powg(num / den, gamma);
        }
    }
    free(y);
    free(x);
    free(p);
    free(q);
}

/* The unpenalized h-solve (lambda = 0). */
void or_hsolve(int F, int K, const double *W, const float *v, double eps,
               double gamma, int n_in, const double *h_init, double *h,
               double *trace) {
    or_hsolve_pen(F, K, W, v, eps, gamma, n_in, 0.0, 1.0, h_init, h, trace);
}

/* One dictionary step of Algorithm 1 given the activations of a minibatch:
 *   X = eps + W H;  a = ((Y/X^2) H^T) o W^2;  b = (1/X) H^T;
 *   A <- rho*A + a, B <- rho*B + b   (or A <- A + rho*a with rho_on_new);
 *   W = sqrt(A/B);  then for each k: s = sum_f W_fk, W_:k /= s, A_:k /= s,
 *   B_:k *= s  (when normalize).
 * loss_out (may be NULL) receives sum_n d_IS(Y_n, X_n) over the minibatch. */
void or_stats_step_pen(int F, int K, int64_t n, const float *V, int64_t ldv,
                       const double *H, double eps, double rho, int normalize,
                       int rho_on_new, double mu, double *W, double *A, double *B,
                       double *loss_out) {
    double *X = (double *)malloc(sizeof(double) * F * (size_t)(n > 0 ? n : 1));
    double *P = (double *)malloc(sizeof(double) * F * (size_t)(n > 0 ? n : 1));
    double *Q = (double *)malloc(sizeof(double) * F * (size_t)(n > 0 ? n : 1));
    double loss = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        for (int f = 0; f < F; ++f) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += W[f + (int64_t)k * F] * H[k + j * K];
            double x = eps + acc;
            double y = eps + (double)V[f + j * ldv];
            X[f + j * F] = x;
            Q[f + j * F] = 1.0 / x;
            P[f + j * F] = y / (x * x);
            double r = y / x;
            loss += (r - 1.0) - log(r);
        }
    }
    if (loss_out) *loss_out = loss;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int f = 0; f < F; ++f) {
        for (int k = 0; k < K; ++k) {
            double ph = 0.0, qh = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                ph += P[f + j * F] * H[k + j * K];
                qh += Q[f + j * F] * H[k + j * K];
            }
            double w = W[f + (int64_t)k * F];
            double a = ph * w * w;
            double b = qh;
            size_t i = f + (size_t)k * F;
            if (rho_on_new) {
                A[i] = A[i] + rho * a;
                B[i] = B[i] + rho * b;
            } else {
                A[i] = rho * A[i] + a;
                B[i] = rho * B[i] + b;
            }
        }
    }
    /* W = sqrt(A/B) (Section 2.1), the minimizer of A/W + B W; with the
     * linear dictionary penalty mu * sum W of Section 2.2 ("Extensions")
     * the auxiliary function is A/W + (B + mu) W, minimized by
     * sqrt(A/(B + mu)). Entries with B + mu = 0 are kept. */
    for (size_t i = 0; i < (size_t)F * K; ++i)
        if (B[i] + mu > 0.0) W[i] = sqrt(A[i] / (B[i] + mu));
    if (normalize) {
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int f = 0; f < F; ++f) s += W[f + (size_t)k * F];
            if (s > 0.0) {
                for (int f = 0; f < F; ++f) {
                    size_t i = f + (size_t)k * F;
                    W[i] = W[i] / s;
                    A[i] = A[i] / s;
                    B[i] = B[i] * s;
                }
            }
        }
    }
    free(X);
    free(P);
    free(Q);
}

/* The unpenalized dictionary step (mu = 0). */
void or_stats_step(int F, int K, int64_t n, const float *V, int64_t ldv,
                   const double *H, double eps, double rho, int normalize,
                   int rho_on_new, double *W, double *A, double *B,
                   double *loss_out) {
    or_stats_step_pen(F, K, n, V, ldv, H, eps, rho, normalize, rho_on_new, 0.0, W, A, B,
                      loss_out);
}

/* Forgetting factor of "Scaling past data": rho = r^(beta'/n_ref), or 1 when
 * no reference length is given. */
double or_rho(double r, int64_t nb, int64_t n_ref) {
    if (n_ref <= 0) return 1.0;
    return pow(r, (double)nb / (double)n_ref);
}

/* One minibatch of Algorithm 1 with fresh restarts: solve h for every frame
 * against the fixed W, then take the dictionary step.
 *   H_out: K x nb (ld K) or NULL; loss_out: sum of d_IS over the minibatch. */
void or_online_minibatch(int F, int K, int64_t nb, const float *V, int64_t ldv,
                         int n_in, double eps, double gamma, double r,
                         int64_t n_ref, int normalize, int rho_on_new,
                         double lambda, double a_pen, double mu,
                         double *W, double *A, double *B, const double *H_init,
                         double *H_out, double *loss_out) {
    double *H = (double *)malloc(sizeof(double) * K * (size_t)(nb > 0 ? nb : 1));
    /* fresh restarts (H_init NULL) or warm restarts from the kept h of each
     * frame (Section 2.3, "Fresh or warm restarts") */
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t j = 0; j < nb; ++j)
        or_hsolve_pen(F, K, W, V + j * ldv, eps, gamma, n_in, lambda, a_pen,
                      H_init ? H_init + j * K : NULL, H + j * K, NULL);
    double rho = or_rho(r, nb, n_ref);
    or_stats_step_pen(F, K, nb, V, ldv, H, eps, rho, normalize, rho_on_new, mu, W, A, B,
                      loss_out);
    if (H_out) memcpy(H_out, H, sizeof(double) * K * (size_t)nb);
    free(H);
}

/* One pass of Algorithm 1 over N frames in order, a dictionary step every
 * beta frames. The N mod beta frames left at the end form a partial
 * minibatch that is processed only when `flush` is set.
 *   W, A, B: state, updated in place. H_init: K x N start points (warm
 *   restarts) or NULL (fresh restarts). H_out: K x N or NULL.
 *   mb_loss: per-minibatch d_IS sums, or NULL. Returns frames processed. */
int64_t or_online_pass(int F, int K, int64_t N, const float *V, int64_t ldv,
                       int beta, int n_in, double eps, double gamma, double r,
                       int64_t n_ref, int normalize, int rho_on_new, int flush,
                       double lambda, double a_pen, double mu,
                       double *W, double *A, double *B, const double *H_init,
                       double *H_out, double *loss_sum, double *mb_loss) {
    int64_t done = 0;
    int64_t m = 0;
    while (done < N) {
        int64_t nb = N - done < beta ? N - done : beta;
        if (nb < beta && !flush) break;
        double l = 0.0;
        or_online_minibatch(F, K, nb, V + done * ldv, ldv, n_in, eps, gamma, r,
                            n_ref, normalize, rho_on_new, lambda, a_pen, mu, W, A, B,
                            H_init ? H_init + done * K : NULL,
                            H_out ? H_out + done * K : NULL, &l);
        if (mb_loss) mb_loss[m] = l;
        /* running sum of the online loss L_T (Eq. online_loss), one term per
         * minibatch, so a pass split over several calls adds in the same order */
        if (loss_sum) *loss_sum += l;
        done += nb;
        ++m;
    }
    return done;
}

/* Projection with W fixed (held-out evaluation): the h-solve of every frame.
 * obj_sum (may be NULL): sum_n d_IS(eps + v_n, eps + W h_n). */
void or_project(int F, int K, int64_t N, const float *V, int64_t ldv,
                const double *W, double eps, double gamma, int n_in, double lambda,
                double a_pen, double *H, double *obj_sum) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (int64_t j = 0; j < N; ++j)
        or_hsolve_pen(F, K, W, V + j * ldv, eps, gamma, n_in, lambda, a_pen, NULL, H + j * K,
                      NULL);
    if (obj_sum) *obj_sum = or_objective(F, K, N, V, ldv, W, H, eps) * (double)N;
}

/* Batch start point: the fresh-restart rule applied to every column,
 * H0_kn = sum_f (eps + V_fn) / sum_{f,k} W_fk. */
void or_batch_h0(int F, int K, int64_t N, const float *V, int64_t ldv,
                 const double *W, double eps, double *H) {
    double sw = 0.0;
    for (int k = 0; k < K; ++k)
        for (int f = 0; f < F; ++f) sw += W[f + (int64_t)k * F];
    for (int64_t n = 0; n < N; ++n) {
        double sy = 0.0;
        for (int f = 0; f < F; ++f) sy += eps + (double)V[f + n * ldv];
        for (int k = 0; k < K; ++k) H[k + n * K] = sy / sw;
    }
}

/* Batch IS-NMF cycles (Section 2.1): every iteration updates all of H with
 * W fixed, recomputes the auxiliary function, and updates W:
 *   X = eps + W H;  H <- H o ((W^T P)/(W^T Q))^gamma   (P = Y/X^2, Q = 1/X)
 *   X = eps + W H;  W <- W o sqrt((P H^T)/(Q H^T))     (= sqrt(A/B), Eq. aux_fun)
 *   normalize: s_k = sum_f W_fk, W_:k /= s_k, H_k: *= s_k
 * obj_out (n_iter entries or NULL): the objective after each iteration.
 * which: 0 = full iterations, 1 = H step only, 2 = W step only. */
void or_batch(int F, int K, int64_t N, const float *V, int64_t ldv, double *W,
              double *H, double eps, double gamma, int n_iter, int normalize,
              double *obj_out, int which) {
    size_t FN = (size_t)F * (size_t)(N > 0 ? N : 1);
    double *P = (double *)malloc(sizeof(double) * FN);
    double *Q = (double *)malloc(sizeof(double) * FN);
    double *Wn = (double *)malloc(sizeof(double) * (size_t)F * K);
    for (int it = 0; it < n_iter; ++it) {
        for (int step = 0; step < 2; ++step) {
            if (which == 1 && step == 1) continue;
            if (which == 2 && step == 0) continue;
            /* X, P, Q from the current W, H */
#pragma omp parallel for num_threads(g_threads) schedule(static)
            for (int64_t n = 0; n < N; ++n) {
                for (int f = 0; f < F; ++f) {
                    double acc = 0.0;
                    for (int k = 0; k < K; ++k) acc += W[f + (int64_t)k * F] * H[k + n * K];
                    double x = eps + acc;
                    double y = eps + (double)V[f + n * ldv];
                    Q[f + n * F] = 1.0 / x;
                    P[f + n * F] = y / (x * x);
                }
            }
            if (step == 0) {
                /* H step */
#pragma omp parallel for num_threads(g_threads) schedule(static)
                for (int64_t n = 0; n < N; ++n) {
                    for (int k = 0; k < K; ++k) {
                        double num = 0.0, den = 0.0;
                        for (int f = 0; f < F; ++f) {
                            num += W[f + (int64_t)k * F] * P[f + n * F];
                            den += W[f + (int64_t)k * F] * Q[f + n * F];
                        }
                        if (den > 0.0) H[k + n * K] = H[k + n * K] * powg(num / den, gamma);
                    }
                }
            } else {
                /* W step */
#pragma omp parallel for num_threads(g_threads) schedule(static)
                for (int f = 0; f < F; ++f) {
                    for (int k = 0; k < K; ++k) {
                        double ph = 0.0, qh = 0.0;
                        for (int64_t n = 0; n < N; ++n) {
                            ph += P[f + n * F] * H[k + n * K];
                            qh += Q[f + n * F] * H[k + n * K];
                        }
                        size_t i = f + (size_t)k * F;
                        Wn[i] = qh > 0.0 ? W[i] * sqrt(ph / qh) : W[i];
                    }
                }
                memcpy(W, Wn, sizeof(double) * (size_t)F * K);
                if (normalize) {
                    for (int k = 0; k < K; ++k) {
                        double s = 0.0;
                        for (int f = 0; f < F; ++f) s += W[f + (size_t)k * F];
                        if (s > 0.0) {
                            for (int f = 0; f < F; ++f) W[f + (size_t)k * F] /= s;
                            for (int64_t n = 0; n < N; ++n) H[k + n * K] *= s;
                        }
                    }
                }
            }
        }
        if (obj_out) obj_out[it] = or_objective(F, K, N, V, ldv, W, H, eps);
    }
    free(P);
    free(Q);
    free(Wn);
}
