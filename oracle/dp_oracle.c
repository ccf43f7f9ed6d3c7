/*
 * dp_oracle.c -- plain FP64 CPU oracle for feedforward decentralized WF / ZF
 * precoding (arXiv:1804.10987).  TEST INFRASTRUCTURE ONLY: only the tests,
 * the smoke check and the CPU baseline leg of the benchmark load it.  It
 * shares nothing with the CUDA library.
 *
 * Every step is the plain definition the paper states, in the paper's
 * order, with plain loops:
 *   Sec. III-B   G_c = H_c H_c^H, G = sum_c G_c (feedforward adder tree)
 *   Eq. (14)     A = G + kappa I_U, Q = H^H A^{-1}   (Appendix B, Woodbury)
 *   Thm. 1       kappa = U N0 / rho^2, beta = sqrt(tr(Q^H Q) Es / rho^2)
 *   Lemma 1      tr(Q^H Q) = tr(A^{-1}) - kappa ||A^{-1}||_F^2
 *   Sec. III-B   z = A^{-1} s / beta, x_c = H_c^H z
 *   Sec. III-D   FD-WF: rho_c^2 = rho^2 / C (or rho^2 w_c / sum w with
 *                per-cluster weights), kappa_c = tau_c U N0 / rho_c^2,
 *                Q_c by the B_c x B_c inverse when B_c < U, else by the
 *                U x U one, x_c = sqrt(rho_c^2 / (tr(Q_c^H Q_c) Es)) Q_c s
 * ZF is the kappa = 0 case of the WF formulas (the paper names ZF only).
 * The library's "scale" is 1 / beta, so x_c = scale * H_c^H A^{-1} s.
 *
 * Build: gcc -O2 -ffp-contract=off -fcx-limited-range (the textbook complex
 * product; no fused multiply-add, so results agree across host ISAs).
 */
#include "dp_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define RE(z) creal(z)
#define IM(z) cimag(z)

static int cfinite(orc_cplx z) { return isfinite(RE(z)) && isfinite(IM(z)); }

/* G = H_c H_c^H with H_c the columns b in [lo, hi) of the U x B channel.
 * With H stored [B][U]: G[i][j] = sum_b H[b][i] conj(H[b][j]). */
void orc_gram(int U, const orc_cplx *H, int lo, int hi, orc_cplx *G) {
  for (int i = 0; i < U; ++i)
    for (int j = 0; j < U; ++j) {
      orc_cplx acc = 0;
      for (int b = lo; b < hi; ++b)
        acc += H[(size_t)b * U + i] * conj(H[(size_t)b * U + j]);
      G[i * U + j] = acc;
    }
}

/* G' = H_c^H H_c (B_c x B_c): G'[a][b] = sum_u conj(H[lo+a][u]) H[lo+b][u]. */
void orc_gram_antenna(int U, const orc_cplx *H, int lo, int hi, orc_cplx *Gp) {
  int n = hi - lo;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      orc_cplx acc = 0;
      for (int u = 0; u < U; ++u)
        acc += conj(H[(size_t)(lo + a) * U + u]) * H[(size_t)(lo + b) * U + u];
      Gp[a * n + b] = acc;
    }
}

/* Textbook Cholesky-Banachiewicz: A = L L^H, L lower with real positive
 * diagonal.  A is Hermitian; only its lower triangle is read. */
int orc_cholesky(int n, const orc_cplx *A, orc_cplx *L) {
  for (int i = 0; i < n * n; ++i) L[i] = 0;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      orc_cplx sum = A[i * n + j];
      for (int k = 0; k < j; ++k) sum -= L[i * n + k] * conj(L[j * n + k]);
      if (i == j) {
        double d = RE(sum);
        if (!(d > 0.0) || !isfinite(d)) return ORC_NOT_PD;
        L[i * n + i] = sqrt(d);
      } else {
        L[i * n + j] = sum / RE(L[j * n + j]);
      }
    }
  }
  return ORC_OK;
}

/* W = L^{-1} by forward substitution on the identity, then T = W^H W. */
void orc_inverse_from_cholesky(int n, const orc_cplx *L, orc_cplx *T) {
  orc_cplx *W = (orc_cplx *)calloc((size_t)n * n, sizeof(orc_cplx));
  for (int j = 0; j < n; ++j) {          /* column j of W solves L w = e_j */
    for (int i = j; i < n; ++i) {
      orc_cplx sum = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) sum -= L[i * n + k] * W[k * n + j];
      W[i * n + j] = sum / RE(L[i * n + i]);
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      orc_cplx acc = 0;
      for (int k = 0; k < n; ++k) acc += conj(W[k * n + i]) * W[k * n + j];
      T[i * n + j] = acc;
    }
  free(W);
}

double orc_t_lemma(int n, const orc_cplx *T, double kappa) {
  double tr = 0.0, fro = 0.0;
  for (int i = 0; i < n; ++i) tr += RE(T[i * n + i]);
  for (int i = 0; i < n * n; ++i) fro += RE(T[i]) * RE(T[i]) + IM(T[i]) * IM(T[i]);
  return tr - kappa * fro;
}

double orc_t_direct(int n, const orc_cplx *T, const orc_cplx *G) {
  orc_cplx *TG = (orc_cplx *)malloc((size_t)n * n * sizeof(orc_cplx));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      orc_cplx acc = 0;
      for (int k = 0; k < n; ++k) acc += T[i * n + k] * G[k * n + j];
      TG[i * n + j] = acc;
    }
  orc_cplx tr = 0;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) tr += TG[i * n + k] * T[k * n + i];
  free(TG);
  return RE(tr);
}

/* ------------------------------------------------------------------ */

typedef struct {
  const orc_desc *d;
  const int *off;
  const orc_cplx *H, *S;
  orc_cplx *X, *Z, *G, *Gloc;
  double *scale, *t, *t_alt;
  int *status;
  int sc_lo, sc_hi;
} job;

/* One U-form WF/ZF system on antennas [lo, hi): A = Gc + kappa I, T = A^{-1},
 * t by Lemma 1, scale = sqrt(rho2 / (Es t)), z_k = T s_k,
 * x_k[b] = scale * sum_u conj(H[b][u]) z_k[u]  for b in [lo, hi). */
static int solve_u_form(const orc_desc *d, const orc_cplx *Hn, const orc_cplx *Sn,
                        int lo, int hi, const orc_cplx *Gc, double kappa, double rho2,
                        orc_cplx *A, orc_cplx *L, orc_cplx *T, orc_cplx *zbuf,
                        orc_cplx *Xn, orc_cplx *Zc, double *scale_out,
                        double *t_out, double *td_out) {
  int U = d->U, K = d->K, B = d->B;
  for (int i = 0; i < U * U; ++i) A[i] = Gc[i];
  for (int i = 0; i < U; ++i) A[i * U + i] += kappa;
  if (orc_cholesky(U, A, L) != ORC_OK) return ORC_NOT_PD;
  orc_inverse_from_cholesky(U, L, T);
  double t = orc_t_lemma(U, T, kappa);
  double td = orc_t_direct(U, T, Gc);
  if (!(t > 0.0) || !isfinite(t)) return ORC_NOT_PD;
  double scale = sqrt(rho2 / (d->Es * t));
  for (int k = 0; k < K; ++k) {
    const orc_cplx *s = Sn + (size_t)k * U;
    for (int i = 0; i < U; ++i) {
      orc_cplx acc = 0;
      for (int j = 0; j < U; ++j) acc += T[i * U + j] * s[j];
      zbuf[i] = acc;
      if (Zc) Zc[(size_t)k * U + i] = acc;
    }
    for (int b = lo; b < hi; ++b) {
      orc_cplx acc = 0;
      for (int u = 0; u < U; ++u) acc += conj(Hn[(size_t)b * U + u]) * zbuf[u];
      Xn[(size_t)k * B + b] = scale * acc;
    }
  }
  *scale_out = scale;
  *t_out = t;
  *td_out = td;
  return ORC_OK;
}

/* MRT (Sec. I; the fully distributed baseline of Sec. III-E): P = H^H / beta
 * with E||x||^2 = rho^2, i.e. t = tr(H H^H) = tr(G), scale = rho / sqrt(Es t);
 * z = s.  td: ||H||_F^2 summed over the entries of H. */
static int solve_mrt(const orc_desc *d, const orc_cplx *Hn, const orc_cplx *Sn,
                     const orc_cplx *G, orc_cplx *Xn, orc_cplx *Zc, double *scale_out,
                     double *t_out, double *td_out) {
  int U = d->U, K = d->K, B = d->B;
  double t = 0.0, td = 0.0;
  for (int i = 0; i < U; ++i) t += RE(G[i * U + i]);
  for (size_t i = 0; i < (size_t)B * U; ++i) td += RE(Hn[i]) * RE(Hn[i]) + IM(Hn[i]) * IM(Hn[i]);
  if (!(t > 0.0) || !isfinite(t)) return ORC_NOT_PD;
  double scale = sqrt(d->rho2 / (d->Es * t));
  for (int k = 0; k < K; ++k) {
    const orc_cplx *s = Sn + (size_t)k * U;
    if (Zc)
      for (int i = 0; i < U; ++i) Zc[(size_t)k * U + i] = s[i];
    for (int b = 0; b < B; ++b) {
      orc_cplx acc = 0;
      for (int u = 0; u < U; ++u) acc += conj(Hn[(size_t)b * U + u]) * s[u];
      Xn[(size_t)k * B + b] = scale * acc;
    }
  }
  *scale_out = scale;
  *t_out = t;
  *td_out = td;
  return ORC_OK;
}

/* FD-WF with B_c < U (Sec. III-D, first case):
 * Q_c = (H_c^H H_c + kappa_c I_{B_c})^{-1} H_c^H, t = tr(Q_c^H Q_c),
 * x_c = sqrt(rho_c^2 / (t Es)) Q_c s.  Q[a][u] for antenna a, user u. */
static int solve_bc_form(const orc_desc *d, const orc_cplx *Hn, const orc_cplx *Sn,
                         int lo, int hi, double kappa, double rho2,
                         orc_cplx *Gp, orc_cplx *Ap, orc_cplx *Lp, orc_cplx *Tp,
                         orc_cplx *Q, orc_cplx *Xn, double *scale_out,
                         double *t_out, double *td_out) {
  int U = d->U, K = d->K, B = d->B, n = hi - lo;
  orc_gram_antenna(U, Hn, lo, hi, Gp);
  for (int i = 0; i < n * n; ++i) Ap[i] = Gp[i];
  for (int i = 0; i < n; ++i) Ap[i * n + i] += kappa;
  if (orc_cholesky(n, Ap, Lp) != ORC_OK) return ORC_NOT_PD;
  orc_inverse_from_cholesky(n, Lp, Tp);
  for (int a = 0; a < n; ++a)
    for (int u = 0; u < U; ++u) {
      orc_cplx acc = 0;
      for (int j = 0; j < n; ++j) acc += Tp[a * n + j] * conj(Hn[(size_t)(lo + j) * U + u]);
      Q[a * U + u] = acc;
    }
  double tq = 0.0;
  for (int i = 0; i < n * U; ++i) tq += RE(Q[i]) * RE(Q[i]) + IM(Q[i]) * IM(Q[i]);
  double t = orc_t_lemma(n, Tp, kappa);
  if (!(tq > 0.0) || !isfinite(tq)) return ORC_NOT_PD;
  double scale = sqrt(rho2 / (tq * d->Es));
  for (int k = 0; k < K; ++k) {
    const orc_cplx *s = Sn + (size_t)k * U;
    for (int a = 0; a < n; ++a) {
      orc_cplx acc = 0;
      for (int u = 0; u < U; ++u) acc += Q[a * U + u] * s[u];
      Xn[(size_t)k * B + lo + a] = scale * acc;
    }
  }
  *scale_out = scale;
  *t_out = tq;
  *td_out = t;
  return ORC_OK;
}

static void *worker(void *arg) {
  job *jb = (job *)arg;
  const orc_desc *d = jb->d;
  int U = d->U, B = d->B, C = d->C, K = d->K;
  int bcmax = 0;
  for (int c = 0; c < C; ++c)
    if (d->cluster_sizes[c] > bcmax) bcmax = d->cluster_sizes[c];
  size_t uu = (size_t)U * U, bb = (size_t)bcmax * bcmax;
  orc_cplx *Gs = (orc_cplx *)calloc(uu, sizeof(orc_cplx));
  orc_cplx *Gc = (orc_cplx *)calloc(uu * C, sizeof(orc_cplx));
  orc_cplx *A = (orc_cplx *)calloc(uu, sizeof(orc_cplx));
  orc_cplx *L = (orc_cplx *)calloc(uu, sizeof(orc_cplx));
  orc_cplx *T = (orc_cplx *)calloc(uu, sizeof(orc_cplx));
  orc_cplx *zb = (orc_cplx *)calloc(U, sizeof(orc_cplx));
  orc_cplx *Gp = (orc_cplx *)calloc(bb, sizeof(orc_cplx));
  orc_cplx *Ap = (orc_cplx *)calloc(bb, sizeof(orc_cplx));
  orc_cplx *Lp = (orc_cplx *)calloc(bb, sizeof(orc_cplx));
  orc_cplx *Tp = (orc_cplx *)calloc(bb, sizeof(orc_cplx));
  orc_cplx *Q = (orc_cplx *)calloc((size_t)bcmax * U, sizeof(orc_cplx));
  int nsys = (d->mode == ORC_FDWF) ? C : 1;

  for (int n = jb->sc_lo; n < jb->sc_hi; ++n) {
    const orc_cplx *Hn = jb->H + (size_t)n * B * U;
    const orc_cplx *Sn = jb->S + (size_t)n * K * U;
    orc_cplx *Xn = jb->X ? jb->X + (size_t)n * K * B : NULL;
    orc_cplx *Xtmp = Xn;
    orc_cplx *Xown = NULL;
    if (!Xtmp) Xtmp = Xown = (orc_cplx *)calloc((size_t)K * B, sizeof(orc_cplx));
    int st = ORC_OK;

    for (size_t i = 0; i < (size_t)B * U && st == ORC_OK; ++i)
      if (!cfinite(Hn[i])) st = ORC_NONFINITE;
    for (size_t i = 0; i < (size_t)K * U && st == ORC_OK; ++i)
      if (!cfinite(Sn[i])) st = ORC_NONFINITE;

    /* Sec. III-B: local Grams, then the feedforward sum in cluster order. */
    for (int i = 0; i < (int)uu; ++i) Gs[i] = 0;
    for (int c = 0; c < C; ++c) {
      orc_gram(U, Hn, jb->off[c], jb->off[c + 1], Gc + c * uu);
      for (size_t i = 0; i < uu; ++i) Gs[i] += Gc[c * uu + i];
      if (jb->Gloc) memcpy(jb->Gloc + ((size_t)c * d->n_sc + n) * uu, Gc + c * uu,
                           uu * sizeof(orc_cplx));
    }
    if (jb->G) memcpy(jb->G + (size_t)n * uu, Gs, uu * sizeof(orc_cplx));

    for (int g = 0; g < nsys && st == ORC_OK; ++g) {
      double sc_v = 0, t_v = 0, td_v = 0;
      if (d->mode == ORC_MRT) {
        orc_cplx *Zn = jb->Z ? jb->Z + (size_t)n * K * U : NULL;
        st = solve_mrt(d, Hn, Sn, Gs, Xtmp, Zn, &sc_v, &t_v, &td_v);
      } else if (d->mode != ORC_FDWF) {
        double kappa = (d->mode == ORC_WF) ? d->U * d->N0 / d->rho2 : 0.0;
        orc_cplx *Zn = jb->Z ? jb->Z + (size_t)n * K * U : NULL;
        st = solve_u_form(d, Hn, Sn, 0, B, Gs, kappa, d->rho2, A, L, T, zb, Xtmp, Zn,
                          &sc_v, &t_v, &td_v);
      } else {
        double rho2c = d->rho2 / C;
        if (d->cluster_power) {
          double wsum = 0;
          for (int c = 0; c < C; ++c) wsum += d->cluster_power[c];
          rho2c = d->rho2 * d->cluster_power[g] / wsum;
        }
        double kappa = d->tau * d->U * d->N0 / rho2c;
        int lo = jb->off[g], hi = jb->off[g + 1], bc = hi - lo;
        int small = d->fd_form == ORC_FORM_BCXBC ||
                    (d->fd_form == ORC_FORM_PAPER && bc < U);
        orc_cplx *Zc = jb->Z ? jb->Z + (((size_t)n * C + g) * K) * U : NULL;
        if (!small) {
          st = solve_u_form(d, Hn, Sn, lo, hi, Gc + g * uu, kappa, rho2c, A, L, T, zb,
                            Xtmp, Zc, &sc_v, &t_v, &td_v);
        } else {
          st = solve_bc_form(d, Hn, Sn, lo, hi, kappa, rho2c, Gp, Ap, Lp, Tp, Q, Xtmp,
                             &sc_v, &t_v, &td_v);
          /* The whitened vector of this cluster in the equal U x U form
           * (push-through identity), defined when kappa_c > 0. */
          if (st == ORC_OK && Zc) {
            for (size_t i = 0; i < (size_t)K * U; ++i) Zc[i] = 0;
            if (kappa > 0.0) {
              for (size_t i = 0; i < uu; ++i) A[i] = Gc[g * uu + i];
              for (int i = 0; i < U; ++i) A[i * U + i] += kappa;
              if (orc_cholesky(U, A, L) == ORC_OK) {
                orc_inverse_from_cholesky(U, L, T);
                for (int k = 0; k < K; ++k)
                  for (int i = 0; i < U; ++i) {
                    orc_cplx acc = 0;
                    for (int j = 0; j < U; ++j) acc += T[i * U + j] * Sn[(size_t)k * U + j];
                    Zc[(size_t)k * U + i] = acc;
                  }
              }
            }
          }
        }
      }
      size_t si = (size_t)n * nsys + g;
      if (jb->scale) jb->scale[si] = (st == ORC_OK) ? sc_v : 0.0;
      if (jb->t) jb->t[si] = (st == ORC_OK) ? t_v : 0.0;
      if (jb->t_alt) jb->t_alt[si] = (st == ORC_OK) ? td_v : 0.0;
    }
    if (st != ORC_OK) {
      for (size_t i = 0; i < (size_t)K * B; ++i) Xtmp[i] = 0;
      for (int g = 0; g < nsys; ++g) {
        size_t si = (size_t)n * nsys + g;
        if (jb->scale) jb->scale[si] = 0.0;
        if (jb->t) jb->t[si] = 0.0;
        if (jb->t_alt) jb->t_alt[si] = 0.0;
      }
    }
    if (jb->status) jb->status[n] = st;
    free(Xown);
  }
  free(Gs); free(Gc); free(A); free(L); free(T); free(zb);
  free(Gp); free(Ap); free(Lp); free(Tp); free(Q);
  return NULL;
}

int orc_precode(const orc_desc *d, const orc_cplx *H, const orc_cplx *S,
                orc_cplx *X, double *scale, double *t, double *t_alt,
                orc_cplx *Z, orc_cplx *G, orc_cplx *Gloc, int *status,
                int nthreads) {
  if (!d || !H || !S || d->U < 1 || d->B < 1 || d->C < 1 || d->n_sc < 0 || d->K < 0 ||
      !d->cluster_sizes || !(d->rho2 > 0) || !(d->Es > 0) || d->N0 < 0 || d->tau < 0)
    return ORC_BAD_ARG;
  if (d->mode != ORC_ZF && d->mode != ORC_WF && d->mode != ORC_FDWF && d->mode != ORC_MRT)
    return ORC_BAD_ARG;
  int *off = (int *)malloc(sizeof(int) * (d->C + 1));
  off[0] = 0;
  for (int c = 0; c < d->C; ++c) {
    if (d->cluster_sizes[c] < 1) { free(off); return ORC_BAD_ARG; }
    off[c + 1] = off[c] + d->cluster_sizes[c];
  }
  if (off[d->C] != d->B) { free(off); return ORC_BAD_ARG; }
  if (d->cluster_power) {
    for (int c = 0; c < d->C; ++c)
      if (d->mode != ORC_FDWF || !(d->cluster_power[c] > 0) || !isfinite(d->cluster_power[c])) {
        free(off);
        return ORC_BAD_ARG;
      }
  }
  if (nthreads < 1) nthreads = 1;
  if (nthreads > d->n_sc) nthreads = d->n_sc > 0 ? d->n_sc : 1;
  job *jobs = (job *)calloc(nthreads, sizeof(job));
  pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
  for (int i = 0; i < nthreads; ++i) {
    jobs[i] = (job){d, off, H, S, X, Z, G, Gloc, scale, t, t_alt, status,
                    (int)((long long)d->n_sc * i / nthreads),
                    (int)((long long)d->n_sc * (i + 1) / nthreads)};
  }
  for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, worker, &jobs[i]);
  worker(&jobs[0]);
  for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
  free(th);
  free(jobs);
  free(off);
  return ORC_OK;
}
