/*
 * dp_oracle.h -- plain FP64 CPU oracle for feedforward decentralized
 * Wiener-filter (WF) and zero-forcing (ZF) precoding (Li, Jeon, Cavallaro,
 * Studer, "Feedforward Architectures for Decentralized Precoding in Massive
 * MU-MIMO Systems", arXiv:1804.10987).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two are compared
 * element by element on the same seeded inputs.
 *
 * Layouts (all arrays row-major, complex = two doubles re, im):
 *   H    [n_sc][B][U]   the U x B channel of one subcarrier stored with the
 *                       user index fastest (column b of H is contiguous);
 *                       cluster c owns antennas [off_c, off_c + B_c)
 *   S    [n_sc][K][U]   transmit symbol vectors s[k]
 *   X    [n_sc][K][B]   precoded vectors x[k] = [x_1; ...; x_C]
 *   G    [n_sc][U][U]   G = sum_c G_c
 *   Gloc [C][n_sc][U][U]
 *   Z    WF/ZF [n_sc][K][U],  FD [n_sc][C][K][U]   z = A^{-1} s (unscaled)
 *   scale WF/ZF [n_sc],       FD [n_sc][C]         scale = 1 / beta
 *   t     same shape as scale: the tr(Q^H Q) the scale was formed from
 *         (Lemma 1 in the U x U form; the definition ||Q_c||_F^2 in the FD
 *         B_c x B_c form; tr(G) for MRT)
 *   t_alt same shape: the other formula for the same quantity (the direct
 *         tr(A^{-1} G A^{-1}) of Appendix B, resp. Lemma 1 on the B_c x B_c
 *         inverse, resp. ||H||_F^2 summed over H for MRT), kept for the pins
 *         that the two agree
 */
#ifndef DP_ORACLE_H
#define DP_ORACLE_H

#include <complex.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef double _Complex orc_cplx;

/* ORC_MRT: maximum ratio transmission, the fully distributed baseline the
 * paper compares against (Sec. I, Sec. III-E): x = scale H^H s with
 * scale = rho / sqrt(Es tr(H^H H)); z = s. */
enum { ORC_ZF = 0, ORC_WF = 1, ORC_FDWF = 2, ORC_MRT = 3 };
enum { ORC_OK = 0, ORC_NOT_PD = 1, ORC_NONFINITE = 2, ORC_BAD_ARG = 3 };
/* FD-WF form selection: the rule of Sec. III-D (B_c < U uses the B_c x B_c
 * inverse, otherwise the U x U one), or one form forced for the pin that the
 * two forms agree. */
enum { ORC_FORM_PAPER = 0, ORC_FORM_UXU = 1, ORC_FORM_BCXBC = 2 };

typedef struct {
  int U, B, C;
  const int *cluster_sizes; /* C entries, each >= 1, summing to B */
  int n_sc, K;
  int mode;                 /* ORC_ZF, ORC_WF, ORC_FDWF, ORC_MRT */
  double rho2, N0, Es, tau; /* tau: FD-WF regularization factor tau_c */
  int fd_form;              /* ORC_FORM_* */
  const double *cluster_power; /* FD-WF: C weights w_c > 0, rho_c^2 =
                                  rho^2 w_c / sum w (Sec. III-D: the
                                  per-cluster powers sum to rho^2); NULL:
                                  rho_c^2 = rho^2 / C */
} orc_desc;

/* Per-cluster Gram G_c = H_c H_c^H over antennas [lo, hi) (Sec. III-B). */
void orc_gram(int U, const orc_cplx *H, int lo, int hi, orc_cplx *G);
/* Antenna-side Gram H_c^H H_c (B_c x B_c) for the FD-WF B_c < U form. */
void orc_gram_antenna(int U, const orc_cplx *H, int lo, int hi, orc_cplx *Gp);
/* Cholesky factor A = L L^H (lower); returns ORC_NOT_PD on a pivot <= 0. */
int orc_cholesky(int n, const orc_cplx *A, orc_cplx *L);
/* T = A^{-1} = L^{-H} L^{-1}. */
void orc_inverse_from_cholesky(int n, const orc_cplx *L, orc_cplx *T);
/* Lemma 1: tr(T) - kappa ||T||_F^2. */
double orc_t_lemma(int n, const orc_cplx *T, double kappa);
/* Appendix B definition: tr(T G T). */
double orc_t_direct(int n, const orc_cplx *T, const orc_cplx *G);

/* The whole precoder for all subcarriers, split over nthreads threads.
 * Any output pointer may be NULL.  Returns ORC_OK or ORC_BAD_ARG; per
 * subcarrier failures go to status[n_sc] (X of that subcarrier zeroed). */
int orc_precode(const orc_desc *d, const orc_cplx *H, const orc_cplx *S,
                orc_cplx *X, double *scale, double *t, double *t_alt,
                orc_cplx *Z, orc_cplx *G, orc_cplx *Gloc, int *status,
                int nthreads);

#ifdef __cplusplus
}
#endif
#endif
