/*
 * mhc_oracle.c -- plain, slow, obviously correct CPU reference for the multi-hadron
 * correlator of Vachaspati & Detmold, "Fast Evaluation of Multi-Hadron Correlation
 * Functions" (Lattice 2014).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The library under
 * paper_1411_3691_gb300/ never includes, links or calls it, and it shares no code with
 * the library.
 *
 * What it computes (Sec. 1, the restated correlator equation and the block-diagonal
 * remark that closes Sec. 1):
 *
 *     C = sum_{i in src} sum_{j in snk} w_i w_j prod_f det G_f^{(ij)},
 *     G_f^{(ij)}[m][n] = S_f[a_i^{f,m}][a_j^{f,n}]            (Sec. 1, definition of G)
 *
 * every determinant from a FRESH LU factorisation with partial pivoting of its own
 * matrix (Sec. 2, first paragraph: det from the LU decomposition, i.e. the product of
 * U's diagonal times the sign of the row permutation).  No determinant-update scheme
 * is used here; that is exactly what the library is checked against.
 *
 * Readings taken where the paper is silent:
 *   - pivot = row with the largest |re|+|im| in the pivot column, ties to the lowest
 *     row index; an exactly zero pivot column gives det = 0.
 *   - the permutation double sum of Sec. 1 equals n! det; C uses det (no n!).
 *   - sums over terms are Neumaier-compensated, real and imaginary parts separately.
 *
 * Layouts (shared with the library's C ABI, so one set of test inputs serves both):
 *   S_f      : complex128, L_f x L_f, row-major, interleaved (re, im).
 *   labels   : int32 [N][sum_f n_f], flavour-major inside a term.
 *   weights  : float64 [N].
 *
 * Build: gcc -O2 -fPIC -shared -o _mhc_oracle.so mhc_oracle.c -lm
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ORACLE_MUTANT (default 0) plants one deliberate mistake; only the mutation test of the
 * pins compiles with it, to show that every planted mistake fails some pin. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#define ORACLE_NMAX 64

/* ---------------------------------------------------------------------------------- */
/* Compensated (Neumaier) summation of reals.                                           */
/* ---------------------------------------------------------------------------------- */
typedef struct {
  double s; /* running sum         */
  double c; /* running compensation */
} neumaier;

static void neu_add(neumaier* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

static double neu_value(const neumaier* a) { return a->s + a->c; }

static double abs1(cplx z) { return fabs(creal(z)) + fabs(cimag(z)); }

/* a / b written out as a conj(b) / |b|^2, so that b / b is exactly 1 on every host (the C
 * library's complex division is not exact there on all targets); the entries of S are
 * of order one, far from overflow. */
static cplx cdiv(cplx a, cplx b) {
  const double br = creal(b), bi = cimag(b), ar = creal(a), ai = cimag(a);
  const double d = br * br + bi * bi;
  return CMPLX((ar * br + ai * bi) / d, (ai * br - ar * bi) / d);
}

/* ---------------------------------------------------------------------------------- */
/* Determinant by LU with partial pivoting (Sec. 2, first paragraph).                   */
/* A is n x n row-major and is overwritten by the factors.                              */
/* ---------------------------------------------------------------------------------- */
static cplx lu_det(int n, cplx* A) {
  cplx det = 1.0;
  for (int k = 0; k < n; k++) {
    int p = k;
    double best = abs1(A[k * n + k]);
    for (int i = k + 1; i < n; i++) {
      double m = abs1(A[i * n + k]);
      if (m > best) {
        best = m;
        p = i;
      }
    }
    if (best == 0.0) return 0.0; /* the pivot column is exactly zero: singular */
    if (p != k) {
      for (int j = 0; j < n; j++) {
        cplx t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
#if ORACLE_MUTANT != 1 /* mutant 1: forget the sign of a row swap */
      det = -det;
#endif
    }
    cplx piv = A[k * n + k];
#if ORACLE_MUTANT == 2 /* mutant 2: multiply by the pivot of the next row */
    if (k + 1 < n) piv = A[(k + 1) * n + k];
#endif
    det *= piv;
    for (int i = k + 1; i < n; i++) {
      cplx l = cdiv(A[i * n + k], piv);
      A[i * n + k] = l;
      for (int j = k + 1; j < n; j++) A[i * n + j] -= l * A[k * n + j];
    }
  }
  return det;
}

/* G[m][n] = S[src[m]][snk[n]]  (Sec. 1, definition of G^{(ij)}) */
static void gather(int n, int L, const cplx* S, const int32_t* src, const int32_t* snk, cplx* G) {
  for (int m = 0; m < n; m++)
    for (int q = 0; q < n; q++)
#if ORACLE_MUTANT == 3 /* mutant 3: transposed gather */
      G[m * n + q] = S[(int64_t)snk[q] * L + src[m]];
#else
      G[m * n + q] = S[(int64_t)src[m] * L + snk[q]];
#endif
}

/* det of one n x n matrix (interleaved re/im, row-major); out[0..1] = re, im */
void oracle_det(int n, const double* G_in, double* out) {
  cplx A[ORACLE_NMAX * ORACLE_NMAX];
  memcpy(A, G_in, sizeof(cplx) * n * n);
  cplx d = lu_det(n, A);
  out[0] = creal(d);
  out[1] = cimag(d);
}

static int64_t total_labels(int F, const int32_t* n_f) {
  int64_t t = 0;
  for (int f = 0; f < F; f++) t += n_f[f];
  return t;
}

/* prod_f det G_f^{(ij)} for one (source term, sink term) pair */
static cplx pair_product(int F, const int32_t* n_f, const int32_t* L_f, const double* const* S_f,
                         const int32_t* a_i, const int32_t* a_j, cplx* dets_out) {
  cplx G[ORACLE_NMAX * ORACLE_NMAX];
  cplx prod = 1.0;
  int off = 0;
#if ORACLE_MUTANT == 8 /* mutant 8: last flavour dropped from the product */
  for (int f = 0; f < F; f++) {
    int n = n_f[f];
    cplx d = 1.0;
    if (f == F - 1 && F > 1) {
      if (dets_out) dets_out[f] = d;
      continue;
    }
#else
  for (int f = 0; f < F; f++) {
    int n = n_f[f];
    cplx d = 1.0; /* an empty flavour block contributes a factor 1 */
#endif
    if (n > 0) {
      gather(n, L_f[f], (const cplx*)S_f[f], a_i + off, a_j + off, G);
      d = lu_det(n, G);
    }
    if (dets_out) dets_out[f] = d;
    prod *= d;
    off += n;
  }
  return prod;
}

/*
 * The correlator restricted to source terms [i0, i1) (all sink terms).  Writes
 *   sums[0..3] = (sum_re, comp_re, sum_im, comp_im)  -- Neumaier state, so that
 *                 several source blocks can be combined exactly by the caller;
 *   scale[0]   = sum |w_i w_j prod_f det|             -- the tolerance scale.
 * Returns 0, or -1 on a bad argument.
 */
int oracle_correlator(int F, const int32_t* n_f, const int32_t* L_f, const double* const* S_f,
                      int64_t n_src, const int32_t* labels_src, const double* w_src, int64_t n_snk,
                      const int32_t* labels_snk, const double* w_snk, int64_t i0, int64_t i1,
                      double* sums, double* scale) {
  for (int f = 0; f < F; f++)
    if (n_f[f] < 0 || n_f[f] > ORACLE_NMAX) return -1;
  if (i0 < 0 || i1 > n_src || i0 > i1) return -1;
  int64_t T = total_labels(F, n_f);
  neumaier re = {0, 0}, im = {0, 0};
  double sc = 0.0;
  for (int64_t i = i0; i < i1; i++) {
    for (int64_t j = 0; j < n_snk; j++) {
      cplx p = pair_product(F, n_f, L_f, S_f, labels_src + i * T, labels_snk + j * T, NULL);
#if ORACLE_MUTANT == 4 /* mutant 4: source weight used twice */
      cplx v = w_src[i] * w_src[i] * p;
#else
      cplx v = w_src[i] * w_snk[j] * p;
#endif
      neu_add(&re, creal(v));
      neu_add(&im, cimag(v));
      sc += cabs(v);
    }
  }
  sums[0] = re.s;
  sums[1] = re.c;
  sums[2] = im.s;
  sums[3] = im.c;
#if ORACLE_MUTANT == 5 /* mutant 5: drop the compensation */
  sums[1] = sums[3] = 0.0;
#endif
  scale[0] = sc;
  return 0;
}

/* Per-pair, per-flavour determinants for a list of (i, j) pairs: out[p][f][re, im]. */
int oracle_pair_dets(int F, const int32_t* n_f, const int32_t* L_f, const double* const* S_f,
                     const int32_t* labels_src, const int32_t* labels_snk, int64_t n_pairs,
                     const int64_t* i_idx, const int64_t* j_idx, double* out) {
  for (int f = 0; f < F; f++)
    if (n_f[f] < 0 || n_f[f] > ORACLE_NMAX) return -1;
  int64_t T = total_labels(F, n_f);
  cplx dets[64];
  if (F > 64) return -1;
  for (int64_t p = 0; p < n_pairs; p++) {
    pair_product(F, n_f, L_f, S_f, labels_src + i_idx[p] * T, labels_snk + j_idx[p] * T, dets);
    for (int f = 0; f < F; f++) {
      out[(p * F + f) * 2 + 0] = creal(dets[f]);
      out[(p * F + f) * 2 + 1] = cimag(dets[f]);
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Gradient.  Jacobi's formula: d det G / d G[m][q] = cof(G)[m][q], the signed minor.    */
/* The cofactor is taken from its definition, (-1)^(m+q) det(G without row m, col q),    */
/* each minor by a fresh LU, so that singular G (repeated labels) is handled exactly.   */
/* ---------------------------------------------------------------------------------- */
static void cofactors(int n, const cplx* G, cplx* cof) {
  cplx M[ORACLE_NMAX * ORACLE_NMAX];
  if (n == 1) {
    cof[0] = 1.0;
    return;
  }
  for (int m = 0; m < n; m++) {
    for (int q = 0; q < n; q++) {
      int r = 0;
      for (int mm = 0; mm < n; mm++) {
        if (mm == m) continue;
        int c = 0;
        for (int qq = 0; qq < n; qq++) {
          if (qq == q) continue;
          M[r * (n - 1) + c] = G[mm * n + qq];
          c++;
        }
        r++;
      }
      cplx d = lu_det(n - 1, M);
#if ORACLE_MUTANT == 6 /* mutant 6: cofactor sign from the row only */
      cof[m * n + q] = (m % 2 == 0) ? d : -d;
#else
      cof[m * n + q] = ((m + q) % 2 == 0) ? d : -d;
#endif
    }
  }
}

/*
 * Holomorphic derivatives of C restricted to source terms [i0, i1):
 *   dS_f[a][b] += sum over pairs and over (m, q) with a_i^{f,m} = a, a_j^{f,q} = b of
 *                 w_i w_j (prod_{f' != f} det_{f'}) cof(G_f)[m][q]
 *   dw_src[i]  += sum_j w_j prod_f det_f          (complex)
 *   dw_snk[j]  += sum_i w_i prod_f det_f          (complex)
 * and the matching absolute scales (sums of moduli of the same contributions).
 * dS_f and its scale are complex128 / float64 arrays of L_f x L_f per flavour, in
 * flavour order, packed one after the other.  All outputs are ACCUMULATED into (the
 * caller zeroes them), with plain summation: the caller compares them with a tolerance
 * proportional to the scales.
 */
int oracle_correlator_grad(int F, const int32_t* n_f, const int32_t* L_f, const double* const* S_f,
                           int64_t n_src, const int32_t* labels_src, const double* w_src,
                           int64_t n_snk, const int32_t* labels_snk, const double* w_snk, int64_t i0,
                           int64_t i1, double* dS, double* dS_scale, double* dw_src,
                           double* dw_src_scale, double* dw_snk, double* dw_snk_scale) {
  if (F > 64) return -1;
  for (int f = 0; f < F; f++)
    if (n_f[f] < 0 || n_f[f] > ORACLE_NMAX) return -1;
  if (i0 < 0 || i1 > n_src || i0 > i1) return -1;
  int64_t T = total_labels(F, n_f);
  int64_t s_off[65];
  s_off[0] = 0;
  for (int f = 0; f < F; f++) s_off[f + 1] = s_off[f] + (int64_t)L_f[f] * L_f[f];
  cplx G[ORACLE_NMAX * ORACLE_NMAX], cof[ORACLE_NMAX * ORACLE_NMAX];
  cplx dets[64];
  cplx* dSc = (cplx*)dS;
  cplx* dwi = (cplx*)dw_src;
  cplx* dwj = (cplx*)dw_snk;
  for (int64_t i = i0; i < i1; i++) {
    const int32_t* a_i = labels_src + i * T;
    for (int64_t j = 0; j < n_snk; j++) {
      const int32_t* a_j = labels_snk + j * T;
      cplx prod = pair_product(F, n_f, L_f, S_f, a_i, a_j, dets);
      /* d C / d w_i and d C / d w_j */
#if ORACLE_MUTANT == 9 /* mutant 9: wrong weight in dC/dw_src */
      dwi[i] += w_src[i] * prod;
#else
      dwi[i] += w_snk[j] * prod;
#endif
      dw_src_scale[i] += cabs(w_snk[j] * prod);
      dwj[j] += w_src[i] * prod;
      dw_snk_scale[j] += cabs(w_src[i] * prod);
      int off = 0;
      for (int f = 0; f < F; f++) {
        int n = n_f[f];
        if (n == 0) continue;
        cplx others = 1.0;
        for (int g = 0; g < F; g++)
          if (g != f) others *= dets[g];
        cplx gamma = w_src[i] * w_snk[j] * others;
        gather(n, L_f[f], (const cplx*)S_f[f], a_i + off, a_j + off, G);
        cofactors(n, G, cof);
        for (int m = 0; m < n; m++)
          for (int q = 0; q < n; q++) {
#if ORACLE_MUTANT == 7 /* mutant 7: gradient scattered to the transposed entry */
            int64_t idx = s_off[f] + (int64_t)a_j[off + q] * L_f[f] + a_i[off + m];
#else
            int64_t idx = s_off[f] + (int64_t)a_i[off + m] * L_f[f] + a_j[off + q];
#endif
            cplx c = gamma * cof[m * n + q];
            dSc[idx] += c;
            dS_scale[idx] += cabs(c);
          }
        off += n;
      }
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Double-double determinant (reference for ill-conditioned pairs).                     */
/* Error-free transformations: Knuth's TwoSum and the FMA-based TwoProd (Dekker's        */
/* product written with a fused multiply-add); double-double add/mul/div as in the       */
/* textbook double-double arithmetic of Dekker (1971).  Same pivot rule as lu_det.       */
/* ---------------------------------------------------------------------------------- */
typedef struct {
  double hi, lo;
} dd;

static dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  dd r = {s, e};
  return r;
}
static dd quick_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  dd r = {s, e};
  return r;
}
static dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  dd r = {p, e};
  return r;
}
static dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
static dd dd_neg(dd a) {
  dd r = {-a.hi, -a.lo};
  return r;
}
static dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
static dd dd_div(dd a, dd b) {
  /* long division: q1 = a/b, r = a - q1 b, q2 = r/b, ... */
  double q1 = a.hi / b.hi;
  dd r = dd_sub(a, dd_mul((dd){q1, 0.0}, b));
  double q2 = r.hi / b.hi;
  r = dd_sub(r, dd_mul((dd){q2, 0.0}, b));
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return dd_add(q, (dd){q3, 0.0});
}
static double dd_abs_approx(dd a) { return fabs(a.hi); }

typedef struct {
  dd re, im;
} cdd;

static cdd cdd_mul(cdd a, cdd b) {
  cdd r;
  r.re = dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im));
  r.im = dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re));
  return r;
}
static cdd cdd_sub(cdd a, cdd b) {
  cdd r = {dd_sub(a.re, b.re), dd_sub(a.im, b.im)};
  return r;
}
static cdd cdd_div(cdd a, cdd b) {
  /* a / b = a conj(b) / |b|^2 */
  dd den = dd_add(dd_mul(b.re, b.re), dd_mul(b.im, b.im));
  cdd bc = {b.re, dd_neg(b.im)};
  cdd num = cdd_mul(a, bc);
  cdd r = {dd_div(num.re, den), dd_div(num.im, den)};
  return r;
}

/* det in double-double; out[0..3] = (re.hi, re.lo, im.hi, im.lo) */
void oracle_det_dd(int n, const double* G_in, double* out) {
  cdd A[ORACLE_NMAX * ORACLE_NMAX];
  for (int k = 0; k < n * n; k++) {
    A[k].re = (dd){G_in[2 * k], 0.0};
    A[k].im = (dd){G_in[2 * k + 1], 0.0};
  }
  cdd det = {{1.0, 0.0}, {0.0, 0.0}};
  for (int k = 0; k < n; k++) {
    int p = k;
    double best = dd_abs_approx(A[k * n + k].re) + dd_abs_approx(A[k * n + k].im);
    for (int i = k + 1; i < n; i++) {
      double m = dd_abs_approx(A[i * n + k].re) + dd_abs_approx(A[i * n + k].im);
      if (m > best) {
        best = m;
        p = i;
      }
    }
    if (best == 0.0) {
      out[0] = out[1] = out[2] = out[3] = 0.0;
      return;
    }
    if (p != k) {
      for (int j = 0; j < n; j++) {
        cdd t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
      det.re = dd_neg(det.re);
      det.im = dd_neg(det.im);
    }
    cdd piv = A[k * n + k];
    det = cdd_mul(det, piv);
    for (int i = k + 1; i < n; i++) {
      cdd l = cdd_div(A[i * n + k], piv);
      A[i * n + k] = l;
      for (int j = k + 1; j < n; j++) A[i * n + j] = cdd_sub(A[i * n + j], cdd_mul(l, A[k * n + j]));
    }
  }
  out[0] = det.re.hi;
  out[1] = det.re.lo;
  out[2] = det.im.hi;
  out[3] = det.im.lo;
}

/*
 * Infinity-norm condition number kappa(G) = ||G||_inf ||G^{-1}||_inf (row sums of
 * moduli), with G^{-1} from the LU factors by n forward/backward solves.  Returns
 * +inf when a pivot column is exactly zero.
 */
double oracle_cond_inf(int n, const double* G_in) {
  cplx A[ORACLE_NMAX * ORACLE_NMAX], X[ORACLE_NMAX * ORACLE_NMAX];
  int perm[ORACLE_NMAX];
  memcpy(A, G_in, sizeof(cplx) * n * n);
  double gnorm = 0.0;
  for (int m = 0; m < n; m++) {
    double s = 0.0;
    for (int q = 0; q < n; q++) s += cabs(A[m * n + q]);
    if (s > gnorm) gnorm = s;
  }
  for (int k = 0; k < n; k++) perm[k] = k;
  for (int k = 0; k < n; k++) {
    int p = k;
    double best = abs1(A[k * n + k]);
    for (int i = k + 1; i < n; i++) {
      double m = abs1(A[i * n + k]);
      if (m > best) {
        best = m;
        p = i;
      }
    }
    if (best == 0.0) return INFINITY;
    if (p != k) {
      for (int j = 0; j < n; j++) {
        cplx t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
      int t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
    for (int i = k + 1; i < n; i++) {
      cplx l = cdiv(A[i * n + k], A[k * n + k]);
      A[i * n + k] = l;
      for (int j = k + 1; j < n; j++) A[i * n + j] -= l * A[k * n + j];
    }
  }
  /* column c of G^{-1}: solve L U x = P e_c */
  for (int c = 0; c < n; c++) {
    cplx z[ORACLE_NMAX];
    for (int m = 0; m < n; m++) z[m] = (perm[m] == c) ? 1.0 : 0.0;
    for (int m = 0; m < n; m++)
      for (int k = 0; k < m; k++) z[m] -= A[m * n + k] * z[k];
    for (int m = n - 1; m >= 0; m--) {
      for (int k = m + 1; k < n; k++) z[m] -= A[m * n + k] * z[k];
      z[m] = cdiv(z[m], A[m * n + m]);
    }
    for (int m = 0; m < n; m++) X[m * n + c] = z[m];
  }
  double inorm = 0.0;
  for (int m = 0; m < n; m++) {
    double s = 0.0;
    for (int q = 0; q < n; q++) s += cabs(X[m * n + q]);
    if (s > inorm) inorm = s;
  }
  return gnorm * inorm;
}
