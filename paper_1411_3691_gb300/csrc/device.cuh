// device.cuh -- complex FP64 device arithmetic and the per-thread factorisations of the
// determinant-update scheme.
//
// GB300 executes FP64 at 2 DFMA per clock per SM (a warp-wide DFMA occupies a
// sub-partition's FP64 pipe for 64 cycles, predicated-off lanes included), while integer,
// select, shuffle and load instructions are ~60x cheaper.  Every routine here therefore
// (1) gives each thread its own matrix, so all 32 lanes do useful FP64 work, (2) keeps the
// FP64 instruction count minimal (a complex multiply-add is 4 DFMA, pivot comparisons and
// guard tests run on the IEEE bit patterns in the integer pipe), and (3) is fully unrolled
// for a compile-time n, so the factors live in registers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mhc {
namespace dev {

typedef double2 cd;

__device__ __forceinline__ cd cmul(cd a, cd b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a b
__device__ __forceinline__ cd cfma(cd a, cd b, cd acc) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc - a b
__device__ __forceinline__ cd cfms(cd a, cd b, cd acc) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ cd cneg(cd a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ cd cadd(cd a, cd b) { return make_double2(a.x + b.x, a.y + b.y); }

// pivot measure |re| + |im| (one DADD; the absolute values are free operand modifiers)
__device__ __forceinline__ double abs1(cd a) { return fabs(a.x) + fabs(a.y); }

// a > b for non-negative, non-NaN doubles, compared as integers (no FP64 instruction)
__device__ __forceinline__ bool gt_nonneg(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}

// unbiased binary exponent of |x| from the bit pattern (zero and subnormals give -1023)
__device__ __forceinline__ int expo(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1023; }
__device__ __forceinline__ int expo(cd z) { return max(expo(z.x), expo(z.y)); }

// 1/d by Newton-Raphson iteration (x <- x + x(1 - d x), quadratic convergence), seeded
// with the PTX approximate reciprocal; two steps reach full double precision.
__device__ __forceinline__ double rcp_nr(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  r = fma(r, e, r);
  e = fma(-d, r, 1.0);
  return fma(r, e, r);
}
// 1/z = conj(z) / |z|^2
__device__ __forceinline__ cd crcp(cd z) {
  const double d = fma(z.x, z.x, z.y * z.y);
  const double r = rcp_nr(d);
  return make_double2(z.x * r, -z.y * r);
}

__device__ __forceinline__ cd ldS(const cd* __restrict__ p) { return __ldg(p); }

// ------------------------------------------------------------------------------------
// Shared-row factorisation of one (family, sink, flavour) block.
//
// A = S[arow[i]][col[q]], i < M = n - RHO shared rows, q < n sink columns.  The family's
// changed rows are ordered last, so the LU of the parent (Sec. 2) with partial pivoting
// among the shared rows leaves U = [U1 | U2] (U1 M x M upper triangular), the forward
// solve of the permuted unit vector e_r is trivial, and one back substitution per
// changed row gives the null vectors  z_t = [-U1^{-1} U2 e_t ; e_t]  of A.  Then for any
// member B (RHO rows),
//     det [A ; B] = sd * det(B Z),   sd = sign(P) det(U1),
// which for RHO = 1 is the cofactor form of the matrix determinant lemma (Sec. 2.1):
// y = sd z = det(G) G^{-1} e_r and det(G + e_r v^T) = g' . y.
//
// Output (slot stride ys):
//   RHO = 1: y[0..n) = sd z                                 (n slots)
//   RHO = 2: z1[0..n), z2[0..n), sd                          (2n + 1 slots)
// Returns true when the pivot guard fires: an exactly zero pivot, or
// max/min pivot magnitude above 2^kp (magnitudes compared by binary exponent).
// *ey receives the exponent scale used by the member guard (see member_det).
// ------------------------------------------------------------------------------------
template <int NC, int NFIX, int RHO>
__device__ __forceinline__ bool shared_rows(const cd* __restrict__ S, int L, int n_rt,
                                            const int32_t* __restrict__ arow,
                                            const int32_t* __restrict__ colp, cd* __restrict__ Y,
                                            int ys, int* ey, int kp) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const int M = n - RHO;
  constexpr int MC = (NC - RHO) > 0 ? (NC - RHO) : 1;
  int col[NC];
#pragma unroll UNR
  for (int q = 0; q < n; q++) col[q] = colp[q];
  cd A[MC][NC];
#pragma unroll UNR
  for (int i = 0; i < M; i++) {
    const cd* row = S + (size_t)arow[i] * L;
#pragma unroll UNR
    for (int q = 0; q < n; q++) A[i][q] = ldS(row + col[q]);
  }
  int parity = 0, emin = 4096, emax = -4096;
  bool zero = false;
  cd rc[MC];
  cd det = make_double2(1.0, 0.0);
#pragma unroll UNR
  for (int k = 0; k < M; k++) {
    // partial pivoting: bring the first row of largest |re|+|im| to position k
    double best = abs1(A[k][k]);
#pragma unroll UNR
    for (int i = k + 1; i < M; i++) {
      const double m = abs1(A[i][k]);
      const bool sw = gt_nonneg(m, best);
      best = sw ? m : best;
      parity ^= (int)sw;
#pragma unroll UNR
      for (int q = k; q < n; q++) {
        const cd t = A[k][q];
        A[k][q] = sw ? A[i][q] : t;
        A[i][q] = sw ? t : A[i][q];
      }
    }
    const int e = expo(best);
    zero |= (__double_as_longlong(best) == 0);
    emin = min(emin, e);
    emax = max(emax, e);
    const cd piv = A[k][k];
    det = (k == 0) ? piv : cmul(det, piv);
    rc[k] = crcp(piv);
#pragma unroll UNR
    for (int i = k + 1; i < M; i++) {
      const cd l = cmul(A[i][k], rc[k]);
#pragma unroll UNR
      for (int q = k + 1; q < n; q++) A[i][q] = cfms(l, A[k][q], A[i][q]);
    }
  }
  const cd sd = parity ? cneg(det) : det;
  int ez = -4096;
#pragma unroll
  for (int t = 0; t < RHO; t++) {
    cd z[NC];
#pragma unroll UNR
    for (int k = M - 1; k >= 0; k--) {
      cd s = A[k][M + t];
#pragma unroll UNR
      for (int q = k + 1; q < M; q++) s = cfma(A[k][q], z[q], s);
      z[k] = cmul(s, cneg(rc[k]));
    }
    if (RHO == 1) {
#pragma unroll UNR
      for (int q = 0; q < M; q++) {
        const cd y = cmul(sd, z[q]);
        Y[q * ys] = y;
        ez = max(ez, expo(y));
      }
      Y[M * ys] = sd;
      ez = max(ez, expo(sd));
    } else {
#pragma unroll UNR
      for (int q = 0; q < M; q++) {
        Y[(t * n + q) * ys] = z[q];
        ez = max(ez, expo(z[q]));
      }
#pragma unroll
      for (int u = 0; u < RHO; u++)  // z_t = [.. ; e_t]
        Y[(t * n + M + u) * ys] = make_double2(u == t ? 1.0 : 0.0, 0.0);
    }
  }
  if (RHO >= 2) {
    Y[(RHO * n) * ys] = sd;
    ez = max(ez, 0);  // the unit entries of z
    *ey = expo(sd) + RHO * ez;
  } else {
    *ey = ez;
  }
  return M > 0 && (zero || emax - emin > kp);
}

// Determinant of a K x K matrix in registers by LU with partial pivoting (largest
// |re| + |im|, the first such row on ties); an exactly zero pivot column gives 0.  D is
// destroyed.  Used for the K x K block B Z of a rank-K family (K >= 4).
template <int K>
__device__ __forceinline__ cd small_det(cd (&D)[K][K]) {
  cd det = make_double2(1.0, 0.0);
  int parity = 0;
  bool zero = false;
#pragma unroll
  for (int k = 0; k < K; k++) {
    double best = abs1(D[k][k]);
#pragma unroll
    for (int i = k + 1; i < K; i++) {
      const double m = abs1(D[i][k]);
      const bool sw = gt_nonneg(m, best);
      best = sw ? m : best;
      parity ^= (int)sw;
#pragma unroll
      for (int q = k; q < K; q++) {
        const cd t = D[k][q];
        D[k][q] = sw ? D[i][q] : t;
        D[i][q] = sw ? t : D[i][q];
      }
    }
    zero |= __double_as_longlong(best) == 0;
    det = k == 0 ? D[k][k] : cmul(det, D[k][k]);
    if (k + 1 < K) {
      const cd rc = crcp(D[k][k]);
#pragma unroll
      for (int i = k + 1; i < K; i++) {
        const cd l = cmul(D[i][k], rc);
#pragma unroll
        for (int q = k + 1; q < K; q++) D[i][q] = cfms(l, D[k][q], D[i][q]);
      }
    }
  }
  if (zero) return make_double2(0.0, 0.0);
  return parity ? cneg(det) : det;
}

// det of member rows B against the cached solve: RHO = 1: b . y; RHO >= 2: sd det(B Z).
// *fail is set when |det| < 2^-kc |b| |y| (the normalised lemma factor, by exponents).
template <int NC, int NFIX, int RHO>
__device__ __forceinline__ cd member_det(const cd* __restrict__ S, int L, int n_rt,
                                         const int32_t* __restrict__ lab,
                                         const int32_t* __restrict__ colp,
                                         const cd* __restrict__ Y, int ys, int ey, int kc,
                                         bool* fail) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  if (RHO == 1) {
    const cd* row = S + (size_t)lab[0] * L;
    cd b = ldS(row + colp[0]);
    int eb = expo(b);
    cd d = cmul(b, Y[0]);
#pragma unroll UNR
    for (int q = 1; q < n; q++) {
      b = ldS(row + colp[q]);
      eb = max(eb, expo(b));
      d = cfma(b, Y[q * ys], d);
    }
    *fail = expo(d) < eb + ey - kc;
    return d;
  } else if (RHO == 3) {
    // sd det(B Z), B the three member rows, Z = [z1 z2 z3]: nine dots, a 3 x 3 det by
    // cofactors of the first row
    const cd* r[3] = {S + (size_t)lab[0] * L, S + (size_t)lab[1] * L, S + (size_t)lab[2] * L};
    cd D[3][3];
    int eb = 0;
#pragma unroll
    for (int u = 0; u < 3; u++)
#pragma unroll
      for (int v = 0; v < 3; v++) D[u][v] = make_double2(0.0, 0.0);
#pragma unroll
    for (int u = 0; u < 3; u++) {
      int e = -4096;
#pragma unroll UNR
      for (int q = 0; q < n; q++) {
        const cd b = ldS(r[u] + colp[q]);
        e = max(e, expo(b));
#pragma unroll
        for (int v = 0; v < 3; v++) D[u][v] = cfma(b, Y[(v * n + q) * ys], D[u][v]);
      }
      eb += e;
    }
    const cd m0 = cfms(D[1][2], D[2][1], cmul(D[1][1], D[2][2]));
    const cd m1 = cfms(D[1][2], D[2][0], cmul(D[1][0], D[2][2]));
    const cd m2 = cfms(D[1][1], D[2][0], cmul(D[1][0], D[2][1]));
    const cd dd = cfma(D[0][2], m2, cfms(D[0][1], m1, cmul(D[0][0], m0)));
    const cd d = cmul(Y[3 * n * ys], dd);
    *fail = expo(d) < eb + ey - kc;
    return d;
  } else if (RHO >= 4) {
    // sd det(B Z), B the RHO member rows: RHO x RHO dots, then a small LU
    cd D[RHO][RHO];
    int eb = 0;
#pragma unroll
    for (int u = 0; u < RHO; u++)
#pragma unroll
      for (int v = 0; v < RHO; v++) D[u][v] = make_double2(0.0, 0.0);
#pragma unroll
    for (int u = 0; u < RHO; u++) {
      const cd* ru = S + (size_t)lab[u] * L;
      int e = -4096;
#pragma unroll UNR
      for (int q = 0; q < n; q++) {
        const cd b = ldS(ru + colp[q]);
        e = max(e, expo(b));
#pragma unroll
        for (int v = 0; v < RHO; v++) D[u][v] = cfma(b, Y[(v * n + q) * ys], D[u][v]);
      }
      eb += e;
    }
    const cd dd = small_det<RHO>(D);
    const cd d = cmul(Y[RHO * n * ys], dd);
    *fail = expo(d) < eb + ey - kc;
    return d;
  } else {
    const cd* r1 = S + (size_t)lab[0] * L;
    const cd* r2 = S + (size_t)lab[1] * L;
    cd d11 = make_double2(0.0, 0.0), d12 = d11, d21 = d11, d22 = d11;
    int e1 = -4096, e2 = -4096;
#pragma unroll UNR
    for (int q = 0; q < n; q++) {
      const int c = colp[q];
      const cd b1 = ldS(r1 + c), b2 = ldS(r2 + c);
      const cd z1 = Y[q * ys], z2 = Y[(n + q) * ys];
      e1 = max(e1, expo(b1));
      e2 = max(e2, expo(b2));
      d11 = cfma(b1, z1, d11);
      d12 = cfma(b1, z2, d12);
      d21 = cfma(b2, z1, d21);
      d22 = cfma(b2, z2, d22);
    }
    const cd dd = cfms(d12, d21, cmul(d11, d22));
    const cd d = cmul(Y[2 * n * ys], dd);
    *fail = expo(d) < e1 + e2 + ey - kc;
    return d;
  }
}

// Rank-2 members against a two-sided block with one changed column (kapply2): the first null
// vector z1 = [-U1^{-1} u ; 1 ; 0] is the same for every sink of the sink family, so the dots
// b1 . z1 and b2 . z1 of a member are too (the sink's changed column meets z1's zero).
// member_dots_z1 forms them (in member_det's order, so the results are bitwise the same) and
// member_det_z1 finishes the member's determinant from them with b1 . z2, b2 . z2.
template <int NC, int NFIX>
__device__ __forceinline__ void member_dots_z1(const cd* __restrict__ S, int L, int n_rt,
                                               const int32_t* __restrict__ lab,
                                               const int32_t* __restrict__ colp,
                                               const cd* __restrict__ Y, int ys, cd* d11, cd* d21) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const cd* r1 = S + (size_t)lab[0] * L;
  const cd* r2 = S + (size_t)lab[1] * L;
  cd a = make_double2(0.0, 0.0), b = a;
#pragma unroll UNR
  for (int q = 0; q < n; q++) {
    const int c = colp[q];
    const cd z1 = Y[q * ys];
    a = cfma(ldS(r1 + c), z1, a);
    b = cfma(ldS(r2 + c), z1, b);
  }
  *d11 = a;
  *d21 = b;
}

template <int NC, int NFIX>
__device__ __forceinline__ cd member_det_z1(const cd* __restrict__ S, int L, int n_rt,
                                            const int32_t* __restrict__ lab,
                                            const int32_t* __restrict__ colp, const cd* __restrict__ Y,
                                            int ys, int ey, int kc, bool* fail, cd d11, cd d21) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const cd* r1 = S + (size_t)lab[0] * L;
  const cd* r2 = S + (size_t)lab[1] * L;
  cd d12 = make_double2(0.0, 0.0), d22 = d12;
  int e1 = -4096, e2 = -4096;
#pragma unroll UNR
  for (int q = 0; q < n; q++) {
    const int c = colp[q];
    const cd b1 = ldS(r1 + c), b2 = ldS(r2 + c);
    const cd z2 = Y[(n + q) * ys];
    e1 = max(e1, expo(b1));
    e2 = max(e2, expo(b2));
    d12 = cfma(b1, z2, d12);
    d22 = cfma(b2, z2, d22);
  }
  const cd dd = cfms(d12, d21, cmul(d11, d22));
  const cd d = cmul(Y[2 * n * ys], dd);
  *fail = expo(d) < e1 + e2 + ey - kc;
  return d;
}

// Row-difference update of a one-row member whose lemma guard failed.  Adding a multiple of
// one row of a matrix to another leaves its determinant unchanged, so for any shared row a_r
//   det [A; b] = det [A; b - a_r] = (b - a_r) . y      (y: the member row's cofactors, A y = 0).
// A member that is near-singular because its row b nearly repeats a shared row (two labels
// whose propagator rows almost coincide) loses its determinant to cancellation in b . y; the
// rounded difference b - a_r is the small remainder itself, correct to one rounding per
// entry (a floating-point subtraction rounds the exact difference once), so its dot with y
// does not cancel.  a_r: the shared row nearest to b in the sink's first column (|re| + |im|
// of the difference, lowest row on ties).  The lemma guard is taken again on the difference
// row; when it fails too the caller refactors.  Off the hot path (one call per failed pair),
// so not inlined.
static __device__ __noinline__ cd rowdiff_det(const cd* __restrict__ S, int L, int n, int32_t blab,
                                       const int32_t* __restrict__ arow,
                                       const int32_t* __restrict__ colp, const cd* __restrict__ Y,
                                       int ys, int ey, int kc, bool* fail) {
  const cd* rb = S + (size_t)blab * L;
  const int c0 = colp[0];
  const cd b0 = ldS(rb + c0);
  int r = 0;
  double best = -1.0;
  for (int i = 0; i < n - 1; i++) {
    const cd x = ldS(S + (size_t)arow[i] * L + c0);
    const double v = abs1(make_double2(b0.x - x.x, b0.y - x.y));
    if (best < 0.0 || v < best) {
      best = v;
      r = i;
    }
  }
  const cd* ra = S + (size_t)arow[r] * L;
  cd d = make_double2(0.0, 0.0);
  int eb = -4096;
  for (int q = 0; q < n; q++) {
    const int c = colp[q];
    const cd x = ldS(rb + c), z = ldS(ra + c);
    const cd del = make_double2(x.x - z.x, x.y - z.y);
    eb = max(eb, expo(del));
    d = cfma(del, Y[q * ys], d);
  }
  *fail = expo(d) < eb + ey - kc;
  return d;
}

// Flops of one rowdiff_det call (planner's rule): the search (a complex difference and
// |re| + |im| per shared row), the differences and the dot.
__host__ __device__ constexpr int rowdiff_flops(int n) { return 3 * (n - 1) + 10 * n; }

// The same for a two-row member (rows b_0, b_1) of a family of rank 2: with the shared rows'
// null vectors z_1, z_2 (Y[q], Y[n + q]) and sd (Y[2n]), det [A; b_0; b_1] = sd det(B Z);
// the member row nearer (relatively, in the sink's first column) to some shared row a_r is
// replaced by its difference b_t - a_r, which leaves the determinant unchanged, and the
// 2 x 2 determinant is formed as in member_det.  The lemma guard is taken again.
static __device__ __noinline__ cd rowdiff2_det(const cd* __restrict__ S, int L, int n, const int32_t* __restrict__ mlab,
                                        const int32_t* __restrict__ arow,
                                        const int32_t* __restrict__ colp, const cd* __restrict__ Y,
                                        int ys, int ey, int kc, bool* fail) {
  const int c0 = colp[0];
  int rt[2];
  double dist[2], nrm[2];
  for (int t = 0; t < 2; t++) {
    const cd b0 = ldS(S + (size_t)mlab[t] * L + c0);
    rt[t] = 0;
    dist[t] = -1.0;
    for (int i = 0; i < n - 2; i++) {
      const cd x = ldS(S + (size_t)arow[i] * L + c0);
      const double v = abs1(make_double2(b0.x - x.x, b0.y - x.y));
      if (dist[t] < 0.0 || v < dist[t]) {
        dist[t] = v;
        rt[t] = i;
      }
    }
    nrm[t] = abs1(b0);
  }
  const int t = (dist[1] * nrm[0] < dist[0] * nrm[1]) ? 1 : 0;  // the relatively nearer row
  const cd* rd = S + (size_t)mlab[t] * L;      // the row that is replaced by a difference
  const cd* ra = S + (size_t)arow[rt[t]] * L;
  const cd* ro = S + (size_t)mlab[1 - t] * L;  // the other member row
  cd dz1 = make_double2(0.0, 0.0), dz2 = dz1, oz1 = dz1, oz2 = dz1;
  int ed = -4096, eo = -4096;
  for (int q = 0; q < n; q++) {
    const int c = colp[q];
    const cd x = ldS(rd + c), z = ldS(ra + c), o = ldS(ro + c);
    const cd del = make_double2(x.x - z.x, x.y - z.y);
    const cd z1 = Y[q * ys], z2 = Y[(n + q) * ys];
    ed = max(ed, expo(del));
    eo = max(eo, expo(o));
    dz1 = cfma(del, z1, dz1);
    dz2 = cfma(del, z2, dz2);
    oz1 = cfma(o, z1, oz1);
    oz2 = cfma(o, z2, oz2);
  }
  // rows in the member's order: [difference; other] for t = 0, [other; difference] for t = 1
  const cd d11 = t == 0 ? dz1 : oz1, d12 = t == 0 ? dz2 : oz2;
  const cd d21 = t == 0 ? oz1 : dz1, d22 = t == 0 ? oz2 : dz2;
  const cd dd = cfms(d12, d21, cmul(d11, d22));
  const cd d = cmul(Y[2 * n * ys], dd);
  *fail = expo(d) < ed + eo + ey - kc;
  return d;
}
__host__ __device__ constexpr int rowdiff2_flops(int n) { return 6 * (n - 2) + 2 * n + 4 * (8 * n - 2) + 20; }

// Scale exponent of a flavour's cached solve as its producers define it: rank 1 the largest
// exponent of y's n entries; rank 2 the exponent of sd plus twice the largest exponent of
// the null vectors' entries (at least 0, their unit entries).
__device__ __forceinline__ int cached_scale(const cd* __restrict__ Y, int ys, int n, int rho) {
  int e = rho == 1 ? -4096 : 0;
  for (int q = 0; q < rho * n; q++) e = max(e, expo(Y[q * ys]));
  return rho == 1 ? e : expo(Y[2 * n * ys]) + 2 * e;
}

// Two-sided update: the sink belongs to a sink family whose members share every column but
// the last, so G = [[B, a], [g^T, alpha]] with B the block of shared rows and shared
// columns.  By the Schur complement det G = alpha det B - g^T adj(B) a, i.e. det G = g' . y
// with g' the member's full row and y = [-det(B) B^{-1} a ; det B].  The block stores the
// LU factors of B once per (family, sink family) block (P B = L U, U's diagonal replaced by
// its reciprocals), the row order P as numbers, -det B and det B; each sink then needs two
// triangular solves.  Writes y like shared_rows (rank 1) and the member-guard scale to *ey.
//   layout: LU[M][M] | perm[M] (real part) | -det B | det B          (M = n - 1)
template <int NC, int NFIX>
__device__ __forceinline__ void kapply(const cd* __restrict__ S, int L, int n_rt,
                                       const int32_t* __restrict__ arow,
                                       const int32_t* __restrict__ colp, const cd* __restrict__ K,
                                       cd* __restrict__ Y, int ys, int* ey) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const int M = n - 1;
  constexpr int MC = NC - 1 > 0 ? NC - 1 : 1;
  const int cj = colp[M];
  cd x[MC];
#pragma unroll UNR
  for (int i = 0; i < M; i++) {  // P a, then L^{-1}
    const int pr = (int)__ldg(&K[M * M + i].x);
    cd w = ldS(S + (size_t)arow[pr] * L + cj);
#pragma unroll UNR
    for (int t = 0; t < i; t++) w = cfms(__ldg(K + i * M + t), x[t], w);
    x[i] = w;
  }
#pragma unroll UNR
  for (int i = M - 1; i >= 0; i--) {  // U^{-1}
    cd w = x[i];
#pragma unroll UNR
    for (int t = i + 1; t < M; t++) w = cfms(__ldg(K + i * M + t), x[t], w);
    x[i] = cmul(w, __ldg(K + i * M + i));
  }
  const cd nd = __ldg(K + M * M + M);
  int ez = -4096;
#pragma unroll UNR
  for (int u = 0; u < M; u++) {
    const cd y = cmul(nd, x[u]);
    Y[u * ys] = y;
    ez = max(ez, expo(y));
  }
  const cd dB = __ldg(K + M * M + M + 1);
  Y[M * ys] = dB;
  *ey = max(ez, expo(dB));
}

// Two-sided update of a two-row family against a one-column sink family.  The shared rows
// A (n-2 of them) restricted to the n-1 shared columns are factorised once per block,
// P A_s = L [U1 | u]; with the free columns ordered last (the last shared column, then the
// sink's changed column) the null vectors of A = [A_s | a(j)] are
//   z1 = [-U1^{-1} u ; 1 ; 0]             (the same for every sink of the family)
//   z2 = [-U1^{-1} L^{-1} P a(j) ; 0 ; 1]
// and det [A ; b1 ; b2] = sd det(B Z) as in shared_rows with RHO = 2.
//   layout: LU[M][M] | perm[M] (real part) | -U1^{-1} u [M] | sd      (M = n - 2)
template <int NC, int NFIX>
__device__ __forceinline__ void kapply2(const cd* __restrict__ S, int L, int n_rt,
                                        const int32_t* __restrict__ arow,
                                        const int32_t* __restrict__ colp, const cd* __restrict__ K,
                                        cd* __restrict__ Y, int ys, int* ey) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const int M = n - 2;
  constexpr int MC = NC - 2 > 0 ? NC - 2 : 1;
  const int cj = colp[n - 1];
  cd x[MC];
#pragma unroll UNR
  for (int i = 0; i < M; i++) {
    const int pr = (int)__ldg(&K[M * M + i].x);
    cd w = ldS(S + (size_t)arow[pr] * L + cj);
#pragma unroll UNR
    for (int t = 0; t < i; t++) w = cfms(__ldg(K + i * M + t), x[t], w);
    x[i] = w;
  }
#pragma unroll UNR
  for (int i = M - 1; i >= 0; i--) {
    cd w = x[i];
#pragma unroll UNR
    for (int t = i + 1; t < M; t++) w = cfms(__ldg(K + i * M + t), x[t], w);
    x[i] = cmul(w, __ldg(K + i * M + i));
  }
  int ez = 0;
#pragma unroll UNR
  for (int u = 0; u < M; u++) {
    const cd v = cneg(x[u]);
    Y[(n + u) * ys] = v;
    const cd nu = __ldg(K + M * M + M + u);
    Y[u * ys] = nu;
    ez = max(ez, max(expo(v), expo(nu)));
  }
  Y[M * ys] = make_double2(1.0, 0.0);
  Y[(M + 1) * ys] = make_double2(0.0, 0.0);
  Y[(n + M) * ys] = make_double2(0.0, 0.0);
  Y[(n + M + 1) * ys] = make_double2(1.0, 0.0);
  const cd sd = __ldg(K + M * M + 2 * M);
  Y[2 * n * ys] = sd;
  *ey = expo(sd) + 2 * ez;
}

// Two-sided update of a two-row family against a two-column sink family: the n-2 shared rows
// and the n-2 shared columns give the square block B, factorised once per block (the layout
// of kapply with n-1 in place of n: LU[M][M] | perm[M] | -det B | det B, M = n - 2).  The
// shared rows are A = [B | a1(j) a2(j)] (the sink's changed columns last), whose null
// vectors are z_t = [-B^{-1} a_t(j) ; e_t], and det [A ; b1 ; b2] = det(B) det(B' Z) as in
// shared_rows with RHO = 2: two triangular solves per sink instead of a factorisation.
template <int NC, int NFIX>
__device__ __forceinline__ void kapply22(const cd* __restrict__ S, int L, int n_rt,
                                         const int32_t* __restrict__ arow,
                                         const int32_t* __restrict__ colp, const cd* __restrict__ K,
                                         cd* __restrict__ Y, int ys, int* ey) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const int M = n - 2;
  constexpr int MC = NC - 2 > 0 ? NC - 2 : 1;
  const int c1 = colp[n - 2], c2 = colp[n - 1];
  cd x1[MC], x2[MC];
#pragma unroll UNR
  for (int i = 0; i < M; i++) {  // P a_t, then L^{-1}
    const int pr = (int)__ldg(&K[M * M + i].x);
    const cd* row = S + (size_t)arow[pr] * L;
    cd w1 = ldS(row + c1), w2 = ldS(row + c2);
#pragma unroll UNR
    for (int t = 0; t < i; t++) {
      const cd l = __ldg(K + i * M + t);
      w1 = cfms(l, x1[t], w1);
      w2 = cfms(l, x2[t], w2);
    }
    x1[i] = w1;
    x2[i] = w2;
  }
#pragma unroll UNR
  for (int i = M - 1; i >= 0; i--) {  // U^{-1}
    cd w1 = x1[i], w2 = x2[i];
#pragma unroll UNR
    for (int t = i + 1; t < M; t++) {
      const cd u = __ldg(K + i * M + t);
      w1 = cfms(u, x1[t], w1);
      w2 = cfms(u, x2[t], w2);
    }
    const cd r = __ldg(K + i * M + i);
    x1[i] = cmul(w1, r);
    x2[i] = cmul(w2, r);
  }
  int ez = 0;
#pragma unroll UNR
  for (int u = 0; u < M; u++) {
    const cd z1 = cneg(x1[u]), z2 = cneg(x2[u]);
    Y[u * ys] = z1;
    Y[(n + u) * ys] = z2;
    ez = max(ez, max(expo(z1), expo(z2)));
  }
  Y[M * ys] = make_double2(1.0, 0.0);
  Y[(M + 1) * ys] = make_double2(0.0, 0.0);
  Y[(n + M) * ys] = make_double2(0.0, 0.0);
  Y[(n + M + 1) * ys] = make_double2(1.0, 0.0);
  const cd sd = __ldg(K + M * M + M + 1);
  Y[2 * n * ys] = sd;
  *ey = expo(sd) + 2 * ez;
}

// Factorisation of one two-sided block (see kapply / kapply2), one thread per block: rows
// S[arow[i]], i < M, columns S[.][scol[u]], u < M (+ the extra column u = M for RHO = 2).
// Partial pivoting with the shared_rows rule.  Returns true when the pivot guard fires.
template <int NC, int NFIX, int RHO>
__device__ __forceinline__ bool kfac_block(const cd* __restrict__ S, int L, int n_rt,
                                           const int32_t* __restrict__ arow,
                                           const int32_t* __restrict__ scol, cd* __restrict__ K,
                                           int kp) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const int M = n - RHO;
  constexpr int MC = NC - RHO > 0 ? NC - RHO : 1;
  const int C = RHO == 2 ? M + 1 : M;  // columns kept
  cd B[MC][MC + 1];
  int perm[MC];
#pragma unroll UNR
  for (int i = 0; i < M; i++) {
    perm[i] = i;
    const cd* row = S + (size_t)arow[i] * L;
#pragma unroll UNR
    for (int u = 0; u < C; u++) B[i][u] = ldS(row + scol[u]);
  }
  int parity = 0, emin = 4096, emax = -4096;
  bool zero = false;
  cd det = make_double2(1.0, 0.0);
#pragma unroll UNR
  for (int k = 0; k < M; k++) {
    double best = abs1(B[k][k]);
#pragma unroll UNR
    for (int i = k + 1; i < M; i++) {
      const double m = abs1(B[i][k]);
      const bool sw = gt_nonneg(m, best);
      best = sw ? m : best;
      parity ^= (int)sw;
      const int pk = perm[k], pi = perm[i];
      perm[k] = sw ? pi : pk;
      perm[i] = sw ? pk : pi;
#pragma unroll UNR
      for (int u = 0; u < C; u++) {
        const cd t = B[k][u];
        B[k][u] = sw ? B[i][u] : t;
        B[i][u] = sw ? t : B[i][u];
      }
    }
    const int e = expo(best);
    zero |= (__double_as_longlong(best) == 0);
    emin = min(emin, e);
    emax = max(emax, e);
    const cd piv = B[k][k];
    det = (k == 0) ? piv : cmul(det, piv);
    const cd rc = crcp(piv);
    B[k][k] = rc;
#pragma unroll UNR
    for (int i = k + 1; i < M; i++) {
      const cd l = cmul(B[i][k], rc);
      B[i][k] = l;
#pragma unroll UNR
      for (int u = k + 1; u < C; u++) B[i][u] = cfms(l, B[k][u], B[i][u]);
    }
  }
  if (M > 0 && (zero || emax - emin > kp)) return true;
  const cd sd = parity ? cneg(det) : det;
#pragma unroll UNR
  for (int i = 0; i < M; i++) {
#pragma unroll UNR
    for (int u = 0; u < M; u++) K[i * M + u] = B[i][u];
    K[M * M + i] = make_double2((double)perm[i], 0.0);
  }
  if (RHO == 1) {
    K[M * M + M] = cneg(sd);
    K[M * M + M + 1] = sd;
  } else {
    cd w[MC];  // -U1^{-1} u, u the transformed extra column
#pragma unroll UNR
    for (int p = M - 1; p >= 0; p--) {
      cd s = B[p][M];
#pragma unroll UNR
      for (int q = p + 1; q < M; q++) s = cfma(B[p][q], w[q], s);
      w[p] = cmul(s, cneg(B[p][p]));
    }
#pragma unroll UNR
    for (int i = 0; i < M; i++) K[M * M + M + i] = w[i];
    K[M * M + 2 * M] = sd;
  }
  return false;
}

// Two-sided update of a one-row family against a two-column sink family: the n-1 shared
// rows A and the n-2 shared columns give B = A[:, shared] ((n-1) x (n-2)), factorised once
// per block, P B = L [U1 ; 0].  For a sink with changed columns a1, a2 let
// at = L^{-1} P a_t = [at_top (n-2) ; at_bot].  The cofactor vector of the member row is
//   y = sd [ -U1^{-1}(a2_top a1_bot - a1_top a2_bot) ; -a2_bot ; a1_bot ],
// sd = sign(P) det(U1), with no division by the last pivot a1_bot.
//   layout: LU[n-1][n-2] (rows < n-2: L below, reciprocal on, U above the diagonal; row
//           n-2: multipliers) | perm[n-1] (real part) | sd
template <int NC, int NFIX>
__device__ __forceinline__ void kapply12(const cd* __restrict__ S, int L, int n_rt,
                                         const int32_t* __restrict__ arow,
                                         const int32_t* __restrict__ colp, const cd* __restrict__ K,
                                         cd* __restrict__ Y, int ys, int* ey) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const int C = n - 2, M = n - 1;
  constexpr int MC = NC - 1 > 0 ? NC - 1 : 1;
  const int c1 = colp[n - 2], c2 = colp[n - 1];
  cd x1[MC], x2[MC];
#pragma unroll UNR
  for (int i = 0; i < M; i++) {  // P a_t, then L^{-1}
    const int pr = (int)__ldg(&K[M * C + i].x);
    const cd* row = S + (size_t)arow[pr] * L;
    cd w1 = ldS(row + c1), w2 = ldS(row + c2);
#pragma unroll UNR
    for (int t = 0; t < i && t < C; t++) {
      const cd l = __ldg(K + i * C + t);
      w1 = cfms(l, x1[t], w1);
      w2 = cfms(l, x2[t], w2);
    }
    x1[i] = w1;
    x2[i] = w2;
  }
  const cd b1 = x1[C], b2 = x2[C];
  cd v[MC];
#pragma unroll UNR
  for (int i = 0; i < C; i++) v[i] = cfms(x1[i], b2, cmul(x2[i], b1));
#pragma unroll UNR
  for (int i = C - 1; i >= 0; i--) {  // U1^{-1}
    cd w = v[i];
#pragma unroll UNR
    for (int t = i + 1; t < C; t++) w = cfms(__ldg(K + i * C + t), v[t], w);
    v[i] = cmul(w, __ldg(K + i * C + i));
  }
  const cd sd = __ldg(K + M * C + M);
  const cd nsd = cneg(sd);
  int ez = -4096;
#pragma unroll UNR
  for (int u = 0; u < C; u++) {
    const cd y = cmul(nsd, v[u]);
    Y[u * ys] = y;
    ez = max(ez, expo(y));
  }
  const cd yc1 = cmul(nsd, b2), yc2 = cmul(sd, b1);
  Y[C * ys] = yc1;
  Y[(C + 1) * ys] = yc2;
  *ey = max(ez, max(expo(yc1), expo(yc2)));
}

// Factorisation of a (one-row family, two-column sink family) block (see kapply12): rows
// S[arow[i]], i < n-1, columns S[.][scol[u]], u < n-2.  Returns true when the pivot guard
// fires.
template <int NC, int NFIX>
__device__ __forceinline__ bool kfac_block12(const cd* __restrict__ S, int L, int n_rt,
                                             const int32_t* __restrict__ arow,
                                             const int32_t* __restrict__ scol, cd* __restrict__ K,
                                             int kp) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const int M = n - 1, C = n - 2;
  constexpr int MC = NC - 1 > 0 ? NC - 1 : 1;
  constexpr int CC = NC - 2 > 0 ? NC - 2 : 1;
  cd B[MC][CC];
  int perm[MC];
#pragma unroll UNR
  for (int i = 0; i < M; i++) {
    perm[i] = i;
    const cd* row = S + (size_t)arow[i] * L;
#pragma unroll UNR
    for (int u = 0; u < C; u++) B[i][u] = ldS(row + scol[u]);
  }
  int parity = 0, emin = 4096, emax = -4096;
  bool zero = false;
  cd det = make_double2(1.0, 0.0);
#pragma unroll UNR
  for (int k = 0; k < C; k++) {
    double best = abs1(B[k][k]);
#pragma unroll UNR
    for (int i = k + 1; i < M; i++) {
      const double m = abs1(B[i][k]);
      const bool sw = gt_nonneg(m, best);
      best = sw ? m : best;
      parity ^= (int)sw;
      const int pk = perm[k], pi = perm[i];
      perm[k] = sw ? pi : pk;
      perm[i] = sw ? pk : pi;
#pragma unroll UNR
      for (int u = 0; u < C; u++) {
        const cd t = B[k][u];
        B[k][u] = sw ? B[i][u] : t;
        B[i][u] = sw ? t : B[i][u];
      }
    }
    const int e = expo(best);
    zero |= (__double_as_longlong(best) == 0);
    emin = min(emin, e);
    emax = max(emax, e);
    const cd piv = B[k][k];
    det = (k == 0) ? piv : cmul(det, piv);
    const cd rc = crcp(piv);
    B[k][k] = rc;
#pragma unroll UNR
    for (int i = k + 1; i < M; i++) {
      const cd l = cmul(B[i][k], rc);
      B[i][k] = l;
#pragma unroll UNR
      for (int u = k + 1; u < C; u++) B[i][u] = cfms(l, B[k][u], B[i][u]);
    }
  }
  if (C > 0 && (zero || emax - emin > kp)) return true;
#pragma unroll UNR
  for (int i = 0; i < M; i++) {
#pragma unroll UNR
    for (int u = 0; u < C; u++) K[i * C + u] = B[i][u];
    K[M * C + i] = make_double2((double)perm[i], 0.0);
  }
  K[M * C + M] = parity ? cneg(det) : det;
  return false;
}

// ------------------------------------------------------------------------------------
// Group-cooperative factorisation of one two-sided block for n > 6.  A per-thread n x n
// complex matrix no longer fits in registers there (17 x 17 at n = 18 is 4.6 KB), and in
// local memory it streams from DRAM.  Instead G consecutive lanes share one block held in
// shared memory: the rows below the pivot are dealt to the G lanes cyclically, so the
// lanes of a warp stay busy with independent eliminations.  Group-local shuffles and
// __syncwarp with the group's lane mask keep groups of one warp independent.
// ------------------------------------------------------------------------------------

// LU with partial pivoting of the R x C matrix B (shared memory, row pitch P), `steps`
// pivot columns.  Pivot: the largest |re| + |im| in the column, ties to the lowest row.
// Rows are exchanged whole (multipliers included); perm[i] = original row at position i.
// On return B holds the multipliers below, U above and the reciprocal pivots on the
// diagonal.  Returns true when the pivot guard fires (a zero pivot, or binary exponents of
// the pivots more than kp apart).
template <int G>
__device__ __forceinline__ bool group_lu(cd* B, int P, int* perm, int R, int C, int steps, int g,
                                         unsigned gm, int kp, cd* det_out, int* par_out) {
  for (int i = g; i < R; i += G) perm[i] = i;
  __syncwarp(gm);
  int parity = 0, emin = 4096, emax = -4096;
  bool zero = false;
  cd det = make_double2(1.0, 0.0);
  for (int k = 0; k < steps; k++) {
    double best = 0.0;
    int idx = -1;
    for (int i = k + g; i < R; i += G) {
      const double m = abs1(B[i * P + k]);
      if (idx < 0 || gt_nonneg(m, best)) {
        best = m;
        idx = i;
      }
    }
#pragma unroll
    for (int off = 1; off < G; off <<= 1) {
      const double ob = __shfl_xor_sync(gm, best, off);
      const int oi = __shfl_xor_sync(gm, idx, off);
      const bool take = oi >= 0 && (idx < 0 || gt_nonneg(ob, best) || (!gt_nonneg(best, ob) && oi < idx));
      best = take ? ob : best;
      idx = take ? oi : idx;
    }
    const int p = idx;
    if (p != k) {
      for (int u = g; u < C; u += G) {
        const cd t = B[k * P + u];
        B[k * P + u] = B[p * P + u];
        B[p * P + u] = t;
      }
      if (g == 0) {
        const int t = perm[k];
        perm[k] = perm[p];
        perm[p] = t;
      }
      parity ^= 1;
    }
    __syncwarp(gm);
    const cd piv = B[k * P + k];
    const int e = expo(best);
    zero |= (__double_as_longlong(best) == 0);
    emin = min(emin, e);
    emax = max(emax, e);
    det = (k == 0) ? piv : cmul(det, piv);
    const cd rc = crcp(piv);
    for (int i = k + 1 + g; i < R; i += G) {
      const cd l = cmul(B[i * P + k], rc);
      B[i * P + k] = l;
      for (int u = k + 1; u < C; u++) B[i * P + u] = cfms(l, B[k * P + u], B[i * P + u]);
    }
    __syncwarp(gm);
    if (g == 0) B[k * P + k] = rc;
  }
  __syncwarp(gm);
  *det_out = det;
  *par_out = parity;
  return steps > 0 && (zero || emax - emin > kp);
}

// Row pitch of a group's block in shared memory: odd, so that the G lanes of a group, which
// work on rows i, i + 1, ..., i + G - 1 at the same column, hit distinct 16-byte bank groups.
__device__ __forceinline__ int group_pitch(int C) { return C | 1; }

// Group version of kfac_block (RHO = 1, 2) for the n > 6 blocks; same factor layout.
// Bs: (NC-1)^2 complex scratch, Ws: NC-1 complex, Ps: NC-1 ints, all in shared memory.
template <int G>
__device__ __forceinline__ bool group_kfac_block(const cd* __restrict__ S, int L, int n, int rho,
                                                 const int32_t* __restrict__ arow,
                                                 const int32_t* __restrict__ scol, cd* __restrict__ K,
                                                 int kp, int g, unsigned gm, cd* Bs, cd* Ws, int* Ps) {
  const int M = n - rho;
  const int C = rho == 2 ? M + 1 : M;
  const int P = group_pitch(C);
  for (int e = g; e < M * C; e += G) {
    const int i = e / C, u = e - i * C;
    Bs[i * P + u] = ldS(S + (size_t)arow[i] * L + scol[u]);
  }
  __syncwarp(gm);
  cd det;
  int parity;
  if (group_lu<G>(Bs, P, Ps, M, C, M, g, gm, kp, &det, &parity)) return true;
  const cd sd = parity ? cneg(det) : det;
  if (rho == 2) {  // w = -U1^{-1} u, u the transformed extra column
    for (int p = M - 1; p >= 0; p--) {
      cd s = make_double2(0.0, 0.0);
      for (int q = p + 1 + g; q < M; q += G) s = cfma(Bs[p * P + q], Ws[q], s);
#pragma unroll
      for (int off = 1; off < G; off <<= 1) {
        s.x += __shfl_xor_sync(gm, s.x, off);
        s.y += __shfl_xor_sync(gm, s.y, off);
      }
      if (g == 0) {
        const cd b = Bs[p * P + M];
        Ws[p] = cmul(make_double2(b.x + s.x, b.y + s.y), cneg(Bs[p * P + p]));
      }
      __syncwarp(gm);
    }
  }
  for (int e = g; e < M * M; e += G) {
    const int i = e / M, u = e - i * M;
    K[e] = Bs[i * P + u];
  }
  for (int i = g; i < M; i += G) K[M * M + i] = make_double2((double)Ps[i], 0.0);
  if (rho == 1) {
    if (g == 0) {
      K[M * M + M] = cneg(sd);
      K[M * M + M + 1] = sd;
    }
  } else {
    for (int i = g; i < M; i += G) K[M * M + M + i] = Ws[i];
    if (g == 0) K[M * M + 2 * M] = sd;
  }
  __syncwarp(gm);
  return false;
}

// Group version of kfac_block12 for the n > 6 blocks; same factor layout.
template <int G>
__device__ __forceinline__ bool group_kfac_block12(const cd* __restrict__ S, int L, int n,
                                                   const int32_t* __restrict__ arow,
                                                   const int32_t* __restrict__ scol, cd* __restrict__ K,
                                                   int kp, int g, unsigned gm, cd* Bs, int* Ps) {
  const int M = n - 1, C = n - 2;
  const int P = group_pitch(C);
  for (int e = g; e < M * C; e += G) {
    const int i = e / C, u = e - i * C;
    Bs[i * P + u] = ldS(S + (size_t)arow[i] * L + scol[u]);
  }
  __syncwarp(gm);
  cd det;
  int parity;
  if (group_lu<G>(Bs, P, Ps, M, C, C, g, gm, kp, &det, &parity)) return true;
  for (int e = g; e < M * C; e += G) {
    const int i = e / C, u = e - i * C;
    K[e] = Bs[i * P + u];
  }
  for (int i = g; i < M; i += G) K[M * C + i] = make_double2((double)Ps[i], 0.0);
  if (g == 0) K[M * C + M] = parity ? cneg(det) : det;
  __syncwarp(gm);
  return false;
}

// Fresh determinant of one n x n block by LU with partial pivoting (the refactor path):
// rows S[rows[m]], columns col[q].
template <int NC, int NFIX>
__device__ __forceinline__ cd fresh_det(const cd* __restrict__ S, int L, int n_rt,
                                        const int32_t* rows, const int32_t* __restrict__ colp) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  cd A[NC][NC];
#pragma unroll UNR
  for (int i = 0; i < n; i++) {
    const cd* row = S + (size_t)rows[i] * L;
#pragma unroll UNR
    for (int q = 0; q < n; q++) A[i][q] = ldS(row + colp[q]);
  }
  int parity = 0;
  bool zero = false;
  cd det = make_double2(1.0, 0.0);
#pragma unroll UNR
  for (int k = 0; k < n; k++) {
    double best = abs1(A[k][k]);
#pragma unroll UNR
    for (int i = k + 1; i < n; i++) {
      const double m = abs1(A[i][k]);
      const bool sw = gt_nonneg(m, best);
      best = sw ? m : best;
      parity ^= (int)sw;
#pragma unroll UNR
      for (int q = k; q < n; q++) {
        const cd t = A[k][q];
        A[k][q] = sw ? A[i][q] : t;
        A[i][q] = sw ? t : A[i][q];
      }
    }
    zero |= (__double_as_longlong(best) == 0);
    const cd piv = A[k][k];
    det = (k == 0) ? piv : cmul(det, piv);
    if (k + 1 < n) {
      const cd rc = crcp(piv);
#pragma unroll UNR
      for (int i = k + 1; i < n; i++) {
        const cd l = cmul(A[i][k], rc);
#pragma unroll UNR
        for (int q = k + 1; q < n; q++) A[i][q] = cfms(l, A[k][q], A[i][q]);
      }
    }
  }
  if (zero) return make_double2(0.0, 0.0);
  return parity ? cneg(det) : det;
}

}  // namespace dev
}  // namespace mhc
