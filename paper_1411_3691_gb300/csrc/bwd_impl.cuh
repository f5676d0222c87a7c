// bwd_impl.cuh -- adjoint of the correlator (templates; instantiated per n class by
// bwd_nc8.cu, bwd_nc18.cu, bwd_nc32.cu).
//
// Jacobi's formula: d det G / d G[m][q] = cof(G)[m][q].  For a work family whose members
// share the rows A of flavour f and differ in the last row g_c, G_c = [A; g_c]:
//   * the cofactors of the last row are y = det(A1) z for every member (they do not
//     depend on g_c), the same cached solve as the forward pass;
//   * the cofactors of the rows of A are linear in g_c, so the whole family contributes
//     cof_A([A; h]) with h = sum_c gamma_c g_c, gamma_c = w_c w_j sign_c prod_{f'!=f} det_f';
//     with A1 = the first n-1 columns of A (LU with partial pivoting, P A1 = L U1),
//     u_m = A1^{-1} e_m, eta_m = h[0..n-1) . u_m:
//       cof_A([A; h])[m] = det(A1) [ (h . z) (u_m ; 0) - eta_m z ]
//     which needs no division by det G (valid for singular members).
// The LU factors are recomputed, not stored.  When the pivot guard fires, y and
// cof_A([A; h]) are taken from their definition (signed minors, fresh LU each).
//
// Scatter: each warp owns a private accumulator D[slot][label] (global memory, L1
// resident) for its sinks (slot s < M: shared row m; slot M + c: member c).  Rank-1
// families deal the (slot, column) cells to the lanes, which add to distinct entries at
// every step (scatter_rows); families of rank 2 and 3 give lane s row s (scatter_rowsk).
// Either way every addition happens in a fixed order, and the per-warp accumulators are
// summed in a fixed order by finalize kernels.
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace mhc {

struct BwdArgs {
  FwdArgs a;
  int tiles_per_cta, n_chunks, warps, kmax, slots_max, Lmax, mn_max, ysl;
  double2* dS_part;     // [cta][warp][F][slots_max][Lmax]
  double2* dwsrc_part;  // [member][n_chunks]
  double2* dwsnk_part;  // [W][n_snk]
  double2* stage;       // [cta][T][mn_max] shared-row cofactors of each sink, per block
  double2* accs;        // [cta][kmax][T] dw_src accumulators of each sink, per block
  double2* r2;          // [cta][kmax][rk2][T] member-row coefficients of rank-2/3 families
  double2* dets;        // [cta][F][kmax][T + 1] member determinants, then gammas, of the block's sinks
  int rk2;              // coefficients per member: (largest rank)^2
  const double2* kinv;  // [W][Q][kistride]: B^{-1} row-major per flavour (two-sided blocks)
  int kistride;
  int kioff[MHC_FMAX];
};

namespace bwd {

using dev::cd;

// Member determinants of the block's sinks in shared memory: [flavour][member][sink] with a
// row pitch of T + 1, so that 8 consecutive members read by the scatter's lanes (one
// 16-byte phase) fall in distinct bank groups.
__device__ __forceinline__ size_t dix(int c, int f, int kmax, int T, int ts) {
  return ((size_t)f * kmax + c) * (T + 1) + ts;
}

// det of an explicit n x n matrix in local memory (LU with partial pivoting; an exactly
// zero pivot column gives 0).  B is destroyed.
template <int NC>
__device__ cd det_local(cd (*B)[NC], int n) {
  cd det = make_double2(1.0, 0.0);
  int parity = 0;
  for (int k = 0; k < n; k++) {
    int p = k;
    double best = dev::abs1(B[k][k]);
    for (int i = k + 1; i < n; i++) {
      const double m = dev::abs1(B[i][k]);
      if (dev::gt_nonneg(m, best)) {
        best = m;
        p = i;
      }
    }
    if (__double_as_longlong(best) == 0) return make_double2(0.0, 0.0);
    if (p != k) {
      for (int q = k; q < n; q++) {
        const cd t = B[k][q];
        B[k][q] = B[p][q];
        B[p][q] = t;
      }
      parity ^= 1;
    }
    det = k == 0 ? B[k][k] : dev::cmul(det, B[k][k]);
    const cd rc = dev::crcp(B[k][k]);
    for (int i = k + 1; i < n; i++) {
      const cd l = dev::cmul(B[i][k], rc);
      for (int q = k + 1; q < n; q++) B[i][q] = dev::cfms(l, B[k][q], B[i][q]);
    }
  }
  return parity ? dev::cneg(det) : det;
}

// (-1)^(r+c) det(G without row r and column c), G n x n explicit
template <int NC>
__device__ cd signed_minor(const cd (*G)[NC], int n, int r, int c) {
  cd B[NC][NC];
  int ii = 0;
  for (int i = 0; i < n; i++) {
    if (i == r) continue;
    int qq = 0;
    for (int q = 0; q < n; q++) {
      if (q == c) continue;
      B[ii][qq++] = G[i][q];
    }
    ii++;
  }
  const cd d = n > 1 ? det_local<NC>(B, n - 1) : make_double2(1.0, 0.0);
  return ((r + c) & 1) ? dev::cneg(d) : d;
}

// Cofactors from their definition for a guarded block: y (cofactors of the member row,
// written to Y with stride ys) and the rows of cof([A; h]) for the shared rows (written
// to Mst, row-major M x n).
template <int NC>
__device__ void minors_block(const cd* __restrict__ S, int L, int n, const int32_t* arow,
                             const int32_t* col, const cd* h, cd* Y, int ys, cd* Mst) {
  const int M = n - 1;
  cd G[NC][NC];
  for (int i = 0; i < M; i++)
    for (int q = 0; q < n; q++) G[i][q] = dev::ldS(S + (size_t)arow[i] * L + col[q]);
  for (int q = 0; q < n; q++) G[M][q] = h[q];
  for (int q = 0; q < n; q++) Y[q * ys] = signed_minor<NC>(G, n, M, q);
  for (int m = 0; m < M; m++)
    for (int q = 0; q < n; q++) Mst[m * n + q] = signed_minor<NC>(G, n, m, q);
}

// Shared-row factorisation kept for the adjoint: writes the rows of cof([A; h]) for the
// shared rows (original row order) to Mst (row-major M x n).  Returns false when the
// pivot guard fires (the caller then takes the minors).
template <int NC, int NFIX>
__device__ __forceinline__ bool lu_block(const cd* __restrict__ S, int L, int n_rt,
                                         const int32_t* __restrict__ arow,
                                         const int32_t* __restrict__ colp, const cd* h,
                                         cd* Mst, int kp) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const int M = n - 1;
  constexpr int MC = NC - 1 > 0 ? NC - 1 : 1;
  cd A[MC][NC];
  int perm[MC];
#pragma unroll UNR
  for (int i = 0; i < M; i++) {
    const cd* row = S + (size_t)arow[i] * L;
    perm[i] = i;
#pragma unroll UNR
    for (int q = 0; q < n; q++) A[i][q] = dev::ldS(row + colp[q]);
  }
  int parity = 0, emin = 4096, emax = -4096;
  bool zero = false;
  cd rc[MC];
  cd det = make_double2(1.0, 0.0);
#pragma unroll UNR
  for (int k = 0; k < M; k++) {
    double best = dev::abs1(A[k][k]);
#pragma unroll UNR
    for (int i = k + 1; i < M; i++) {
      const double m = dev::abs1(A[i][k]);
      const bool sw = dev::gt_nonneg(m, best);
      best = sw ? m : best;
      parity ^= (int)sw;
      const int pk = perm[k], pi = perm[i];
      perm[k] = sw ? pi : pk;
      perm[i] = sw ? pk : pi;
#pragma unroll UNR
      for (int q = 0; q < n; q++) {  // whole rows: the multipliers travel with them
        const cd t = A[k][q];
        A[k][q] = sw ? A[i][q] : t;
        A[i][q] = sw ? t : A[i][q];
      }
    }
    const int e = dev::expo(best);
    zero |= (__double_as_longlong(best) == 0);
    emin = min(emin, e);
    emax = max(emax, e);
    const cd piv = A[k][k];
    det = (k == 0) ? piv : dev::cmul(det, piv);
    rc[k] = dev::crcp(piv);
#pragma unroll UNR
    for (int i = k + 1; i < M; i++) {
      const cd l = dev::cmul(A[i][k], rc[k]);
      A[i][k] = l;
#pragma unroll UNR
      for (int q = k + 1; q < n; q++) A[i][q] = dev::cfms(l, A[k][q], A[i][q]);
    }
  }
  if (M > 0 && (zero || emax - emin > kp)) return false;
  const cd sd = parity ? dev::cneg(det) : det;
  // z = [-U1^{-1} u2 ; 1]
  cd z[NC];
  z[M] = make_double2(1.0, 0.0);
#pragma unroll UNR
  for (int k = M - 1; k >= 0; k--) {
    cd s = A[k][M];
#pragma unroll UNR
    for (int q = k + 1; q < M; q++) s = dev::cfma(A[k][q], z[q], s);
    z[k] = dev::cmul(s, dev::cneg(rc[k]));
  }
  cd hz = dev::cmul(h[0], z[0]);
#pragma unroll UNR
  for (int q = 1; q < n; q++) hz = dev::cfma(h[q], z[q], hz);
  const cd alpha = dev::cmul(sd, hz);
  // one column of A1^{-1} per position i: u = U1^{-1} L^{-1} e_i is column perm[i]
#pragma unroll UNR
  for (int i = 0; i < M; i++) {
    cd w[NC];
#pragma unroll UNR
    for (int p = 0; p < M; p++) {
      if (p < i) {
        w[p] = make_double2(0.0, 0.0);
      } else if (p == i) {
        w[p] = make_double2(1.0, 0.0);
      } else {
        cd s = dev::cneg(A[p][i]);
#pragma unroll UNR
        for (int t = i + 1; t < p; t++) s = dev::cfms(A[p][t], w[t], s);
        w[p] = s;
      }
    }
    cd u[NC];
#pragma unroll UNR
    for (int p = M - 1; p >= 0; p--) {
      cd s = w[p];
#pragma unroll UNR
      for (int t = p + 1; t < M; t++) s = dev::cfms(A[p][t], u[t], s);
      u[p] = dev::cmul(s, rc[p]);
    }
    cd eta = make_double2(0.0, 0.0);
#pragma unroll UNR
    for (int q = 0; q < M; q++) eta = dev::cfma(h[q], u[q], eta);
    const cd beta = dev::cmul(sd, eta);
    cd* row = Mst + perm[i] * n;
#pragma unroll UNR
    for (int q = 0; q < M; q++) row[q] = dev::cfms(beta, z[q], dev::cmul(alpha, u[q]));
    row[M] = dev::cneg(beta);
  }
  return true;
}

// B^{-1} of every (one-row family, one-column sink family) block, from the LU factors the
// forward stores (see kapply): column perm[i] of B^{-1} is U^{-1} L^{-1} e_i.  One thread
// per block; blocks that are not two-sided, or whose pivot guard fired, are skipped.
template <int NCMAX>
__global__ void __launch_bounds__(128) kinv_kernel(const BwdArgs B, int64_t n_fam) {
  const FwdArgs& a = B.a;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_fam * a.n_q * a.F) return;
  // flavour slowest across threads (a warp shares n_f); t indexes the [W][Q][f] layout
  const int64_t nwq = n_fam * a.n_q;
  const int f = (int)(u / nwq);
  const int64_t wq = u % nwq;
  const int64_t t = wq * a.F + f;
  const int Q = (int)(wq % a.n_q);
  const int W = (int)(wq / a.n_q);
  const int n = a.n_f[f];
  if (n < 2 || !a.q_two[Q] || a.fam_rank[(int64_t)W * a.F + f] != 1 ||
      a.q_rank[(int64_t)Q * a.F + f] != 1 || a.kguard[t])
    return;
  const int M = n - 1;
  const cd* K = a.kbuf + wq * a.kstride + a.koff[f];
  cd* X = const_cast<cd*>(B.kinv) + wq * B.kistride + B.kioff[f];
  cd w[NCMAX];
  for (int i = 0; i < M; i++) {
    for (int p = 0; p < M; p++) {
      if (p < i) {
        w[p] = make_double2(0.0, 0.0);
      } else if (p == i) {
        w[p] = make_double2(1.0, 0.0);
      } else {
        cd s = dev::cneg(K[p * M + i]);
        for (int q = i + 1; q < p; q++) s = dev::cfms(K[p * M + q], w[q], s);
        w[p] = s;
      }
    }
    for (int p = M - 1; p >= 0; p--) {
      cd s = w[p];
      for (int q = p + 1; q < M; q++) s = dev::cfms(K[p * M + q], w[q], s);
      w[p] = dev::cmul(s, K[p * M + p]);
    }
    const int col = (int)K[M * M + i].x;
    for (int u = 0; u < M; u++) X[u * M + col] = w[u];
  }
}

// Shared-row cofactors of [A; h] for a two-sided block: with B^{-1} shared by the block,
// y = det(B) [-B^{-1} a ; 1] the cached vector and eta = h[0..M) B^{-1},
//   cof[m][q] = (h . y) B^{-1}[q][m] - eta_m y_q  (q < M),   cof[m][M] = -det(B) eta_m,
// i.e. det(A1) [ (h . z)(u_m ; 0) - eta_m z ] with A1 = B; no division.
template <int NC, int NFIX>
__device__ __forceinline__ void two_cof(int n_rt, const cd* __restrict__ Binv, cd detB, const cd* h,
                                        const cd* __restrict__ Y, int ys, cd* Mst) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const int M = n - 1;
  cd y[NC];
#pragma unroll UNR
  for (int q = 0; q < n; q++) y[q] = Y[q * ys];
  cd alpha = dev::cmul(h[0], y[0]);
#pragma unroll UNR
  for (int q = 1; q < n; q++) alpha = dev::cfma(h[q], y[q], alpha);
#pragma unroll UNR
  for (int m = 0; m < M; m++) {
    cd eta = make_double2(0.0, 0.0);
#pragma unroll UNR
    for (int q = 0; q < M; q++) eta = dev::cfma(h[q], __ldg(Binv + q * M + m), eta);
    cd* row = Mst + m * n;
#pragma unroll UNR
    for (int q = 0; q < M; q++) row[q] = dev::cfms(eta, y[q], dev::cmul(alpha, __ldg(Binv + q * M + m)));
    row[M] = dev::cneg(dev::cmul(detB, eta));
  }
}

// Pass 2 of one (sink, flavour): the aggregated member row h = sum_c gamma_c g_c and the
// shared-row cofactors of [A; h] into Mst (row-major M x n) -- from B^{-1} for a two-sided
// block, from the recomputed shared-row LU otherwise, from signed minors where the pivot
// guard fired.  With NFIX the row h stays in registers.
template <int NC, int NFIX>
__device__ __forceinline__ void cof_pass(const FwdArgs& a, const BwdArgs& B, int f, int n_rt, int W,
                                         int mem0, int kW, double wj, int tid, int T,
                                         const int32_t* __restrict__ col, const int32_t* __restrict__ arow,
                                         const cd* Dets, const cd* Y, bool guarded, const cd* Binv,
                                         cd detB, cd* Mst) {
  constexpr int UNR = NFIX ? NC : 1;
  const int n = NFIX ? NFIX : n_rt;
  const cd* S = a.S[f];
  const int L = a.L_f[f];
  cd h[NC];
#pragma unroll UNR
  for (int q = 0; q < n; q++) h[q] = make_double2(0.0, 0.0);
  for (int c = 0; c < kW; c++) {
    const int m = mem0 + c;
    const cd g = Dets[dix(c, f, B.kmax, T, tid)];  // gamma_c of this flavour
    const cd* brow = S + (size_t)a.mem_lab[((int64_t)m * a.F + f) * MHC_MAX_RANK] * L;
#pragma unroll UNR
    for (int q = 0; q < n; q++) h[q] = dev::cfma(g, dev::ldS(brow + col[q]), h[q]);
  }
  bool ok = false;
  if (!guarded) {
    if (Binv) {
      two_cof<NC, NFIX>(n, Binv, detB, h, Y, T, Mst);
      ok = true;
    } else {
      ok = lu_block<NC, NFIX>(S, L, n, arow, col, h, Mst, a.kp);
    }
  }
  if (!ok) {
    cd hl[NC];
#pragma unroll UNR
    for (int q = 0; q < n; q++) hl[q] = h[q];
    minors_block<NC>(S, L, n, arow, col, hl, const_cast<cd*>(Y), T, Mst);
  }
}

// Family of rank k (k = 2, 3 changed rows), shared rows A ((n-k) x n), member rows
// b_0..b_{k-1}: G = [A; B].  With the null vectors z_v of A (last k coordinates the
// identity), sd = sign(P) det(A1) and D = B Z (k x k), det G = sd det(D), and from
// cof(G) = det(G) G^{-T} (G^{-1}'s A-columns X = X0 - Z D^{-1} B X0 with the right inverse
// X0 = [A1^{-1}; 0], det(D) D^{-1} = adj D):
//   cof(G)[b_a] = sd Z adj(D) e_a,
//   sum_c gamma_c cof(G_c)[A] = sd X0^T (s I - E Z^T),
// s = sum_c gamma_c det(D_c), E = sum_c gamma_c B_c^T adj(D_c)^T (n x k): row m of the
// shared block is sd [ s (u_m; 0) - sum_v (u_m . E_v) z_v ],  u_m = A1^{-1} e_m, O(n) per
// member and no division by det G.  Writes the shared block to Mst (row-major
// (n-k) x n) and member row a's coefficients on z_v, gamma sd adj(D)[v][a], to
// R[c][a k + v][T].  When the shared rows fail the pivot guard the same outputs come from
// cof_passk_guarded (complete pivoting, or signed minors for rank-deficient shared rows).
template <int RK>
__device__ __forceinline__ void adjugate(const cd (&D)[RK][RK], cd (&adj)[RK][RK], cd* det) {
  if constexpr (RK == 2) {
    adj[0][0] = D[1][1];
    adj[0][1] = dev::cneg(D[0][1]);
    adj[1][0] = dev::cneg(D[1][0]);
    adj[1][1] = D[0][0];
    *det = dev::cfms(D[0][1], D[1][0], dev::cmul(D[0][0], D[1][1]));
  } else if constexpr (RK == 3) {
    // adj[j][i] = (-1)^(i+j) minor(i, j)
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++) {
        const int r0 = i == 0 ? 1 : 0, r1 = i == 2 ? 1 : 2;
        const int c0 = j == 0 ? 1 : 0, c1 = j == 2 ? 1 : 2;
        const cd m = dev::cfms(D[r0][c1], D[r1][c0], dev::cmul(D[r0][c0], D[r1][c1]));
        adj[j][i] = ((i + j) & 1) ? dev::cneg(m) : m;
      }
    *det = dev::cfma(D[0][2], adj[2][0], dev::cfma(D[0][1], adj[1][0], dev::cmul(D[0][0], adj[0][0])));
  } else {
    // RK >= 4: adj[j][i] = (-1)^(i+j) det(D without row i and column j), each by a small LU
    // (no division by det D, so a singular D is exact); det D along the first row
#pragma unroll
    for (int i = 0; i < RK; i++)
#pragma unroll
      for (int j = 0; j < RK; j++) {
        cd mn[RK - 1][RK - 1];
#pragma unroll
        for (int r = 0; r < RK - 1; r++)
#pragma unroll
          for (int c = 0; c < RK - 1; c++) mn[r][c] = D[r < i ? r : r + 1][c < j ? c : c + 1];
        const cd m = dev::small_det<RK - 1>(mn);
        adj[j][i] = ((i + j) & 1) ? dev::cneg(m) : m;
      }
    cd d = dev::cmul(D[0][0], adj[0][0]);
#pragma unroll
    for (int j = 1; j < RK; j++) d = dev::cfma(D[0][j], adj[j][0], d);
    *det = d;
  }
}

// The rank-k block of one sink when the shared rows' factorisation fails the pivot guard
// (the first n - k columns of A nearly singular, or A itself rank-deficient, e.g. a repeated
// shared label).  The member rows' cofactors always lie in the null space of A: every shared
// row is orthogonal (bilinearly) to them.
//   * A of full rank: an LU of A with complete pivoting, P A Pi = L [U1 | U2], picks the n - k
//     pivot columns; the null vectors z'_v (unit entry at the v-th free column, -U1^{-1}U2 e_v
//     at the pivot columns) and sd' = sign(P) sign(Pi) det(U1) satisfy det [A; B] =
//     sd' det(B Z'), and X0 = Pi [A1'^{-1}; 0] is a right inverse of A, so the formulas of
//     cof_passk hold with (Z', sd', X0) -- the derivation only uses A X0 = I and A Z' = 0.
//     Z' and sd' replace the sink's cached solves, which the scatter reads.
//   * A rank-deficient (an exactly zero pivot): every member's [A; B] is singular and every
//     member-row cofactor is a minor of rank below its size, so exactly 0; the shared rows'
//     block sum_c gamma_c cof(G_c)[A] is taken from signed minors (fresh LU each).
template <int NC, int RK>
__device__ __noinline__ void cof_passk_guarded(const FwdArgs& a, int f, int n, int mem0, int kW, int tid,
                                               int T, int kmax, const int32_t* __restrict__ col,
                                               const int32_t* __restrict__ arow, const cd* Dets, cd* Y,
                                               cd* Mst, cd* R) {
  constexpr int MC = NC - RK > 0 ? NC - RK : 1;
  const int M = n - RK;
  const cd* S = a.S[f];
  const int L = a.L_f[f];
  cd A[NC][NC];  // the shared rows (complete-pivoting LU), or [A; B_c] for the minors
  int rp[MC], cp[NC];
  for (int i = 0; i < M; i++) {
    rp[i] = i;
    const cd* row = S + (size_t)arow[i] * L;
    for (int q = 0; q < n; q++) A[i][q] = dev::ldS(row + col[q]);
  }
  for (int q = 0; q < n; q++) cp[q] = q;
  int parity = 0;
  bool degenerate = false;
  cd det = make_double2(1.0, 0.0);
  cd rc[MC];
  for (int t = 0; t < M; t++) {
    // complete pivoting: the largest |re| + |im| of the remaining block, first in row-major order
    int pi = t, pq = t;
    double best = -1.0;
    for (int i = t; i < M; i++)
      for (int q = t; q < n; q++) {
        const double v = dev::abs1(A[i][q]);
        if (best < 0.0 || dev::gt_nonneg(v, best)) {
          best = v;
          pi = i;
          pq = q;
        }
      }
    if (__double_as_longlong(best) == 0) {
      degenerate = true;
      break;
    }
    if (pi != t) {
      for (int q = 0; q < n; q++) {
        const cd x = A[t][q];
        A[t][q] = A[pi][q];
        A[pi][q] = x;
      }
      const int x = rp[t];
      rp[t] = rp[pi];
      rp[pi] = x;
      parity ^= 1;
    }
    if (pq != t) {
      for (int i = 0; i < M; i++) {
        const cd x = A[i][t];
        A[i][t] = A[i][pq];
        A[i][pq] = x;
      }
      const int x = cp[t];
      cp[t] = cp[pq];
      cp[pq] = x;
      parity ^= 1;
    }
    det = t == 0 ? A[t][t] : dev::cmul(det, A[t][t]);
    rc[t] = dev::crcp(A[t][t]);
    for (int i = t + 1; i < M; i++) {
      const cd l = dev::cmul(A[i][t], rc[t]);
      A[i][t] = l;
      for (int q = t + 1; q < n; q++) A[i][q] = dev::cfms(l, A[t][q], A[i][q]);
    }
  }
  if (degenerate) {
    for (int v = 0; v < RK; v++)
      for (int q = 0; q < n; q++) Y[(size_t)(v * n + q) * T] = make_double2(0.0, 0.0);
    Y[(size_t)RK * n * T] = make_double2(0.0, 0.0);
    for (int c = 0; c < kW; c++)
      for (int t = 0; t < RK * RK; t++) R[((size_t)c * RK * RK + t) * T + tid] = make_double2(0.0, 0.0);
    for (int e = 0; e < M * n; e++) Mst[e] = make_double2(0.0, 0.0);
    for (int i = 0; i < M; i++)
      for (int q = 0; q < n; q++) A[i][q] = dev::ldS(S + (size_t)arow[i] * L + col[q]);
    for (int c = 0; c < kW; c++) {
      const int m = mem0 + c;
      const cd g = Dets[dix(c, f, kmax, T, tid)];  // gamma_c of this flavour
      for (int u = 0; u < RK; u++) {
        const cd* br = S + (size_t)a.mem_lab[((int64_t)m * a.F + f) * MHC_MAX_RANK + u] * L;
        for (int q = 0; q < n; q++) A[M + u][q] = dev::ldS(br + col[q]);
      }
      for (int i = 0; i < M; i++)
        for (int q = 0; q < n; q++) Mst[i * n + q] = dev::cfma(g, signed_minor<NC>(A, n, i, q), Mst[i * n + q]);
    }
    return;
  }
  const cd sd = parity ? dev::cneg(det) : det;
  // null vectors in the original column order, written over the sink's cached solves
  for (int v = 0; v < RK; v++) {
    cd w[MC];
    for (int p = M - 1; p >= 0; p--) {
      cd x = A[p][M + v];
      for (int q = p + 1; q < M; q++) x = dev::cfma(A[p][q], w[q], x);
      w[p] = dev::cmul(x, dev::cneg(rc[p]));
    }
    for (int q = 0; q < M; q++) Y[(size_t)(v * n + cp[q]) * T] = w[q];
    for (int u = 0; u < RK; u++) Y[(size_t)(v * n + cp[M + u]) * T] = make_double2(u == v ? 1.0 : 0.0, 0.0);
  }
  Y[(size_t)RK * n * T] = sd;
  // members: D = B Z', adj(D), s, E, the member rows' coefficients (as in cof_passk)
  cd E[RK][NC];
  for (int q = 0; q < n; q++)
    for (int v = 0; v < RK; v++) E[v][q] = make_double2(0.0, 0.0);
  cd s = make_double2(0.0, 0.0);
  for (int c = 0; c < kW; c++) {
    const int m = mem0 + c;
    const cd g = Dets[dix(c, f, kmax, T, tid)];
    const cd* r[RK];
    for (int u = 0; u < RK; u++) r[u] = S + (size_t)a.mem_lab[((int64_t)m * a.F + f) * MHC_MAX_RANK + u] * L;
    cd D[RK][RK];
    for (int u = 0; u < RK; u++)
      for (int v = 0; v < RK; v++) D[u][v] = make_double2(0.0, 0.0);
    for (int q = 0; q < n; q++)
      for (int u = 0; u < RK; u++) {
        const cd b = dev::ldS(r[u] + col[q]);
        for (int v = 0; v < RK; v++) D[u][v] = dev::cfma(b, Y[(size_t)(v * n + q) * T], D[u][v]);
      }
    cd adj[RK][RK], dd;
    adjugate<RK>(D, adj, &dd);
    s = dev::cfma(g, dd, s);
    cd ga[RK][RK];
    for (int u = 0; u < RK; u++)
      for (int v = 0; v < RK; v++) ga[u][v] = dev::cmul(g, adj[u][v]);
    for (int q = 0; q < n; q++)
      for (int u = 0; u < RK; u++) {
        const cd b = dev::ldS(r[u] + col[q]);
        for (int v = 0; v < RK; v++) E[v][q] = dev::cfma(b, ga[v][u], E[v][q]);
      }
    cd* Rc = R + (size_t)c * RK * RK * T + tid;
    for (int u = 0; u < RK; u++)
      for (int v = 0; v < RK; v++) Rc[(size_t)(u * RK + v) * T] = dev::cmul(sd, ga[v][u]);
  }
  // shared rows: row rp[i] = sd [ s u~ - sum_v (u~ . E_v) z'_v ], u~ = A1'^{-1} e_{rp[i]} at
  // the pivot columns
  const cd ss = dev::cmul(sd, s);
  for (int i = 0; i < M; i++) {
    cd u[MC];
    for (int p = 0; p < M; p++) {
      if (p < i) {
        u[p] = make_double2(0.0, 0.0);
      } else if (p == i) {
        u[p] = make_double2(1.0, 0.0);
      } else {
        cd w = dev::cneg(A[p][i]);
        for (int t = i + 1; t < p; t++) w = dev::cfms(A[p][t], u[t], w);
        u[p] = w;
      }
    }
    for (int p = M - 1; p >= 0; p--) {
      cd w = u[p];
      for (int t = p + 1; t < M; t++) w = dev::cfms(A[p][t], u[t], w);
      u[p] = dev::cmul(w, rc[p]);
    }
    cd se[RK];
    for (int v = 0; v < RK; v++) {
      cd e = make_double2(0.0, 0.0);
      for (int t = 0; t < M; t++) e = dev::cfma(u[t], E[v][cp[t]], e);
      se[v] = dev::cmul(sd, e);
    }
    cd* row = Mst + (size_t)rp[i] * n;
    for (int q = 0; q < n; q++) {
      cd x = make_double2(0.0, 0.0);
      for (int v = 0; v < RK; v++) x = dev::cfms(se[v], Y[(size_t)(v * n + q) * T], x);
      row[q] = x;
    }
    for (int t = 0; t < M; t++) row[cp[t]] = dev::cfma(ss, u[t], row[cp[t]]);
  }
}

template <int NC, int RK>
__device__ __noinline__ bool cof_passk(const FwdArgs& a, int f, int n, int mem0, int kW, int tid,
                                       int T, int kmax, const int32_t* __restrict__ col,
                                       const int32_t* __restrict__ arow, const cd* Dets, const cd* Y,
                                       bool guarded, cd* Mst, cd* R) {
  const int M = n - RK;
  const cd* S = a.S[f];
  const int L = a.L_f[f];
  if (guarded) return false;  // the forward's shared-row factorisation failed its pivot guard
  const cd sd = Y[(size_t)RK * n * T];
  cd E[RK][NC];
  for (int q = 0; q < n; q++)
#pragma unroll
    for (int v = 0; v < RK; v++) E[v][q] = make_double2(0.0, 0.0);
  cd s = make_double2(0.0, 0.0);
  for (int c = 0; c < kW; c++) {
    const int m = mem0 + c;
    const cd g = Dets[dix(c, f, kmax, T, tid)];  // gamma_c of this flavour
    const cd* r[RK];
#pragma unroll
    for (int u = 0; u < RK; u++) r[u] = S + (size_t)a.mem_lab[((int64_t)m * a.F + f) * MHC_MAX_RANK + u] * L;
    cd D[RK][RK];
#pragma unroll
    for (int u = 0; u < RK; u++)
#pragma unroll
      for (int v = 0; v < RK; v++) D[u][v] = make_double2(0.0, 0.0);
    for (int q = 0; q < n; q++) {
#pragma unroll
      for (int u = 0; u < RK; u++) {
        const cd b = dev::ldS(r[u] + col[q]);
#pragma unroll
        for (int v = 0; v < RK; v++) D[u][v] = dev::cfma(b, Y[(size_t)(v * n + q) * T], D[u][v]);
      }
    }
    cd adj[RK][RK], det;
    adjugate<RK>(D, adj, &det);
    s = dev::cfma(g, det, s);
    cd ga[RK][RK];  // gamma adj(D)
#pragma unroll
    for (int u = 0; u < RK; u++)
#pragma unroll
      for (int v = 0; v < RK; v++) ga[u][v] = dev::cmul(g, adj[u][v]);
    for (int q = 0; q < n; q++) {  // E_v += gamma sum_a b_a adj(D)[v][a]
#pragma unroll
      for (int u = 0; u < RK; u++) {
        const cd b = dev::ldS(r[u] + col[q]);
#pragma unroll
        for (int v = 0; v < RK; v++) E[v][q] = dev::cfma(b, ga[v][u], E[v][q]);
      }
    }
    cd* Rc = R + (size_t)c * RK * RK * T + tid;
#pragma unroll
    for (int u = 0; u < RK; u++)
#pragma unroll
      for (int v = 0; v < RK; v++)
        Rc[(size_t)(u * RK + v) * T] = dev::cmul(sd, ga[v][u]);
  }
  // LU of A1 (the shared rows on the first n - k columns), partial pivoting
  constexpr int MC = NC - RK > 0 ? NC - RK : 1;
  cd A[MC][MC];
  int perm[MC];
  for (int i = 0; i < M; i++) {
    perm[i] = i;
    const cd* row = S + (size_t)arow[i] * L;
    for (int q = 0; q < M; q++) A[i][q] = dev::ldS(row + col[q]);
  }
  int emin = 4096, emax = -4096;
  bool zero = false;
  cd rc[MC];
  for (int k = 0; k < M; k++) {
    double best = dev::abs1(A[k][k]);
    int p = k;
    for (int i = k + 1; i < M; i++) {
      const double v = dev::abs1(A[i][k]);
      if (dev::gt_nonneg(v, best)) {
        best = v;
        p = i;
      }
    }
    if (p != k) {
      for (int q = 0; q < M; q++) {
        const cd t = A[k][q];
        A[k][q] = A[p][q];
        A[p][q] = t;
      }
      const int t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
    const int e = dev::expo(best);
    zero |= (__double_as_longlong(best) == 0);
    emin = min(emin, e);
    emax = max(emax, e);
    rc[k] = dev::crcp(A[k][k]);
    for (int i = k + 1; i < M; i++) {
      const cd l = dev::cmul(A[i][k], rc[k]);
      A[i][k] = l;
      for (int q = k + 1; q < M; q++) A[i][q] = dev::cfms(l, A[k][q], A[i][q]);
    }
  }
  if (M > 0 && (zero || emax - emin > a.kp)) return false;  // A1 fails the guard: cof_passk_guarded
  const cd ss = dev::cmul(sd, s);
  for (int i = 0; i < M; i++) {  // u = column perm[i] of A1^{-1} = U^{-1} L^{-1} e_i
    cd u[MC];
    for (int p = 0; p < M; p++) {
      if (p < i) {
        u[p] = make_double2(0.0, 0.0);
      } else if (p == i) {
        u[p] = make_double2(1.0, 0.0);
      } else {
        cd w = dev::cneg(A[p][i]);
        for (int t = i + 1; t < p; t++) w = dev::cfms(A[p][t], u[t], w);
        u[p] = w;
      }
    }
    for (int p = M - 1; p >= 0; p--) {
      cd w = u[p];
      for (int t = p + 1; t < M; t++) w = dev::cfms(A[p][t], u[t], w);
      u[p] = dev::cmul(w, rc[p]);
    }
    cd se[RK];
#pragma unroll
    for (int v = 0; v < RK; v++) {
      cd e = make_double2(0.0, 0.0);
      for (int q = 0; q < M; q++) e = dev::cfma(u[q], E[v][q], e);
      se[v] = dev::cmul(sd, e);
    }
    cd* row = Mst + (size_t)perm[i] * n;
    for (int q = 0; q < M; q++) {
      cd x = dev::cmul(ss, u[q]);
#pragma unroll
      for (int v = 0; v < RK; v++) x = dev::cfms(se[v], Y[(size_t)(v * n + q) * T], x);
      row[q] = x;
    }
#pragma unroll
    for (int v = 0; v < RK; v++) row[M + v] = dev::cneg(se[v]);  // z_v's unit coordinates
  }
  return true;
}

// Scatter of one warp's sinks for a family of rank k (flavour f): lane s owns row s -- a
// shared row (s < n - k, from the staged block) or row a of member c (s = n - k + k c + a),
// whose values are the coefficient combination sum_v R[c][a k + v] z_v.  Same fixed order
// and shared-column sums as scatter_rows.
template <int NC, int RK>
__device__ __noinline__ void scatter_rowsk(const FwdArgs& a, const BwdArgs& B, int f, int n, int kW,
                                           int nlive, int T, int warp, int lane,
                                           const int32_t* __restrict__ mycol, int myQ, int mynsh,
                                           const cd* Stage, const cd* Ysm, const cd* R, cd* Df) {
  constexpr unsigned FULL = 0xffffffffu;
  const int M = n - RK;
  const int nslots = M + RK * kW;
  int cl[NC];
#pragma unroll
  for (int q = 0; q < NC; q++) cl[q] = q < n ? mycol[q] : 0;
  for (int s = lane; s < ((nslots + 31) & ~31); s += 32) {
    const bool act = s < nslots;
    const bool mem = s >= M;
    const int c = act && mem ? (s - M) / RK : 0;
    const int t = act && mem ? (s - M) - RK * c : 0;
    cd* Drow = Df + (size_t)(act ? s : 0) * B.Lmax;
    cd acc[NC];
    int curlab[NC];
    int curQ = -2, nsh = 0;
#pragma unroll
    for (int q = 0; q < NC; q++) {
      acc[q] = make_double2(0.0, 0.0);
      curlab[q] = 0;
    }
    for (int jl = 0; jl <= nlive; jl++) {
      const bool live = jl < nlive;
      const int src = jl & 31;
      const int Qj = __shfl_sync(FULL, myQ, src);
      const int nsj = __shfl_sync(FULL, mynsh, src);
      int cj[NC];
#pragma unroll
      for (int q = 0; q < NC; q++) cj[q] = __shfl_sync(FULL, cl[q], src);
      if (!live || Qj != curQ || Qj < 0) {
        if (act) {
#pragma unroll
          for (int q = 0; q < NC; q++)
            if (q < nsh) {
              cd& d = Drow[curlab[q]];
              d.x += acc[q].x;
              d.y += acc[q].y;
            }
        }
        if (!live) break;
        curQ = Qj;
        nsh = nsj;
#pragma unroll
        for (int q = 0; q < NC; q++) {
          acc[q] = make_double2(0.0, 0.0);
          curlab[q] = cj[q];
        }
      }
      const int ts = warp * 32 + jl;
      cd k[RK];
#pragma unroll
      for (int v = 0; v < RK; v++)
        k[v] = mem ? R[((size_t)c * RK * RK + t * RK + v) * T + ts] : make_double2(0.0, 0.0);
      const cd* st = Stage + (size_t)ts * B.mn_max + (mem ? 0 : s * n);
#pragma unroll
      for (int q = 0; q < NC; q++) {
        if (q >= n) break;
        cd v = make_double2(0.0, 0.0);
        if (mem) {
#pragma unroll
          for (int u = 0; u < RK; u++) v = dev::cfma(k[u], Ysm[(size_t)(a.yoff[f] + u * n + q) * T + ts], v);
        } else {
          v = st[q];
        }
        if (q < nsh) {
          acc[q] = dev::cadd(acc[q], v);
        } else if (act) {
          cd& d = Drow[cj[q]];
          d = dev::cadd(d, v);
        }
      }
    }
  }
}

// One (sink, flavour) block of a family of rank RK >= 2: the cofactor pass (redone with
// complete pivoting or signed minors where the shared rows fail the pivot guard) and the
// warp's scatter.  Called by the whole warp.
template <int NCMAX, int RK>
__device__ __forceinline__ void rank_block(const FwdArgs& a, const BwdArgs& B, int f, int n, int mem0, int kW,
                                           int tid, int T, int warp, int lane, int nlive,
                                           const int32_t* col, const int32_t* arow, const cd* Dets,
                                           const cd* Ysm, bool gd, cd* myStage, const cd* Stage, cd* Rk,
                                           int myQ, int mynsh, cd* Df) {
  const cd* Yf = Ysm + (size_t)a.yoff[f] * T + tid;
  if (!cof_passk<NCMAX, RK>(a, f, n, mem0, kW, tid, T, B.kmax, col, arow, Dets, Yf, gd, myStage, Rk))
    cof_passk_guarded<NCMAX, RK>(a, f, n, mem0, kW, tid, T, B.kmax, col, arow, Dets, const_cast<cd*>(Yf), myStage,
                                 Rk);
  __syncwarp();
  scatter_rowsk<NCMAX, RK>(a, B, f, n, kW, nlive, T, warp, lane, col, myQ, mynsh, Stage, Ysm, Rk, Df);
  __syncwarp();
}

template <int NCMAX>
__device__ __forceinline__ void dispatch_cof_pass(const FwdArgs& a, const BwdArgs& B, int f, int n, int W,
                                                  int mem0, int kW, double wj, int tid, int T,
                                                  const int32_t* col, const int32_t* arow, const cd* Dets,
                                                  const cd* Y, bool guarded, const cd* Binv, cd detB,
                                                  cd* Mst) {
#define MHC_COF(NN) cof_pass<NN, NN>(a, B, f, NN, W, mem0, kW, wj, tid, T, col, arow, Dets, Y, guarded, \
                                     Binv, detB, Mst)
  switch (n) {
    case 1: MHC_COF(1); return;
    case 2: MHC_COF(2); return;
    case 3: MHC_COF(3); return;
    case 4: MHC_COF(4); return;
    case 5: MHC_COF(5); return;
    case 6: MHC_COF(6); return;
    default:
      cof_pass<NCMAX, 0>(a, B, f, n, W, mem0, kW, wj, tid, T, col, arow, Dets, Y, guarded, Binv, detB, Mst);
  }
#undef MHC_COF
}

// Scatter of one warp's 32 sinks into its accumulator rows (flavour f).  The cells of the
// block -- row s (a shared row, s < n - 1, values from the staged cofactor block, or member
// s - n + 1, gamma times the cached y) by column q -- are dealt to the lanes 32 at a time,
// the members' cells column by column, then the shared rows' cells, cell e to lane e mod
// 32, so that the lanes stay busy whatever the number of rows, the lanes of one step
// mostly read one column of y, and a step of shared rows only adds (gamma = 1).  Within a two-sided sink family the shared columns carry the same labels for every
// sink, so their contributions are summed in registers and added to the row once per
// family; the changed columns are added per sink.  Lanes that hold cells of one row add to
// distinct labels (the columns of a sink carry distinct labels), except for a sink that
// repeats a label, whose cells are added one column at a time; a __syncwarp after every
// sink orders the additions to one accumulator entry by sink, so the order is fixed.  Each
// sink's metadata (sink family, number of shared columns, column labels, weight) sits in
// the registers of the sink's own lane and reaches the other lanes by shuffles.
template <int NC, int NFIX>
__device__ __forceinline__ void scatter_rows(const FwdArgs& a, const BwdArgs& B, int f, int n_rt,
                                             int kW, int mem0, int nlive, int T, int warp, int lane,
                                             const int32_t* __restrict__ mycol, int myQ, int mynsh,
                                             const cd* Stage, const cd* Ysm,
                                             const cd* Dets, cd* Df) {
  constexpr int UNR = NFIX ? NC : 1;
  constexpr unsigned FULL = 0xffffffffu;
  const int n = NFIX ? NFIX : n_rt;
  const int M = n - 1;
  const int nslots = M + kW;
  const int ncells = nslots * n;
  int cl[NC];
#pragma unroll UNR
  for (int q = 0; q < n; q++) cl[q] = mycol[q];
  // does this lane's sink repeat a label in flavour f
  int myrep = 0;
#pragma unroll UNR
  for (int q = 1; q < n; q++)
#pragma unroll UNR
    for (int p = 0; p < q; p++) myrep |= cl[q] == cl[p];
  for (int e0 = 0; e0 < ncells; e0 += 32) {
    const int e = e0 + lane;
    const bool act = e < ncells;
    // member cells first (column by column), then the shared rows' cells
    const int nmc = kW * n;
    const bool shround = e0 >= nmc;  // every cell of this step is a shared row's: g = 1
    const int e1 = e - nmc;
    const int q = !act ? 0 : (e < nmc ? e / kW : e1 / M);
    const int s = !act ? 0 : (e < nmc ? M + (e - q * kW) : e1 - q * M);
    const bool mem = s >= M;
    const int c = mem ? s - M : 0;
    cd* Drow = Df + (size_t)s * B.Lmax;
    const cd* Ycol = Ysm + (size_t)(a.yoff[f] + q) * T;
    // the sweep over the sinks, compiled apart for the steps of shared rows only
    auto sweep = [&](auto sh) {
      cd acc = make_double2(0.0, 0.0);
      int curlab = 0, curQ = -2, nsh = 0;
      for (int jl = 0; jl <= nlive; jl++) {
        const bool live = jl < nlive;
        const int src = jl & 31;
        const int Qj = __shfl_sync(FULL, myQ, src);
        const int nsj = __shfl_sync(FULL, mynsh, src);
        const int rep = __shfl_sync(FULL, myrep, src);
        int lab = 0;  // the label of this cell's column in sink jl
#pragma unroll UNR
        for (int p = 0; p < n; p++) {
          const int t = __shfl_sync(FULL, cl[p], src);
          lab = p == q ? t : lab;
        }
        if (!live || Qj != curQ || Qj < 0) {  // flush the summed shared columns of the previous family
          // one column at a time: the family's shared labels may repeat
          for (int p = 0; p < nsh; p++) {
            if (act && q == p) {
              cd& d = Drow[curlab];
              d.x += acc.x;
              d.y += acc.y;
            }
            __syncwarp();
          }
          if (!live) break;
          curQ = Qj;
          nsh = nsj;
          acc = make_double2(0.0, 0.0);
          curlab = lab;
        }
        const int ts = warp * 32 + jl;
        const cd g = (mem && !decltype(sh)::value) ? Dets[dix(c, f, B.kmax, T, ts)] : make_double2(1.0, 0.0);
        const cd v = mem ? Ycol[ts] : Stage[(size_t)ts * B.mn_max + s * n + q];
        const bool shcol = q < nsh;
        if (!rep) {
          // one complex FMA (an addition in a step of shared rows) per lane, on the register
          // sum or on the accumulator entry
          const cd base = shcol ? acc : (act ? Drow[lab] : make_double2(0.0, 0.0));
          cd r;
        if constexpr (decltype(sh)::value)
          r = dev::cadd(base, v);
        else
          r = dev::cfma(g, v, base);
          if (shcol)
            acc = r;
          else if (act)
            Drow[lab] = r;
        } else {
          if (shcol) acc = dev::cfma(g, v, acc);
          for (int p = nsh; p < n; p++) {
            if (act && q == p) Drow[lab] = dev::cfma(g, v, Drow[lab]);
            __syncwarp();
          }
        }
        __syncwarp();
      }
    };
    if (shround)
      sweep(std::true_type{});
    else
      sweep(std::false_type{});
  }
}

template <int NCMAX>
__device__ __forceinline__ void dispatch_scatter(const FwdArgs& a, const BwdArgs& B, int f, int n,
                                                 int kW, int mem0, int nlive, int T, int warp, int lane,
                                                 const int32_t* mycol, int myQ, int mynsh,
                                                 const cd* Stage, const cd* Ysm, const cd* Dets, cd* Df) {
#define MHC_SC(NN) scatter_rows<NN, NN>(a, B, f, NN, kW, mem0, nlive, T, warp, lane, mycol, myQ, mynsh, \
                                        Stage, Ysm, Dets, Df)
  switch (n) {
    case 1: MHC_SC(1); return;
    case 2: MHC_SC(2); return;
    case 3: MHC_SC(3); return;
    case 4: MHC_SC(4); return;
    case 5: MHC_SC(5); return;
    case 6: MHC_SC(6); return;
    default:
      scatter_rows<NCMAX, 0>(a, B, f, n, kW, mem0, nlive, T, warp, lane, mycol, myQ, mynsh, Stage, Ysm,
                             Dets, Df);
  }
#undef MHC_SC
}

// Blocks per SM: the n <= 8 class asks for 14 one-warp blocks (it compiles to 128 registers,
// with spills): measured 7.88 ms per He-4-like call against 8.00 ms when asking for 16 and
// 8.38 ms at the 12 blocks that 168 registers allowed.
template <int NCMAX>
__global__ void __launch_bounds__(32, NCMAX <= 8 ? 14 : 9) bwd_kernel(const BwdArgs B) {
  const FwdArgs& a = B.a;
  extern __shared__ double2 smem[];
  const int T = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cta = blockIdx.x;
  const int W = cta / B.n_chunks, chunk = cta % B.n_chunks;
  const int mem0 = a.fam_info[4 * W], kW = a.fam_info[4 * W + 1];
  // shared memory: the y cache [ysl][T]; the member determinants [F][kmax][T + 1] live in
  // global scratch of the block (L1-resident), which leaves the shared memory small enough
  // for the registers to set the occupancy
  cd* Ysm = smem;
  cd* Dets = B.dets + (size_t)cta * a.F * B.kmax * (T + 1);
  // dw_src accumulators: global scratch of this block (L1/L2-resident), which leaves the
  // shared memory to the data the scatter shares across lanes
  cd* AccS = B.accs + (size_t)cta * B.kmax * T;
  // staging of the shared-row cofactors: global scratch of this block (L1 resident)
  cd* Stage = B.stage + (size_t)cta * T * B.mn_max;
  cd* myStage = Stage + (size_t)(warp * 32 + lane) * B.mn_max;
  cd* Dw = B.dS_part + ((size_t)(cta * B.warps + warp) * a.F) * B.slots_max * B.Lmax;

  for (int c = 0; c < kW; c++) AccS[c * T + tid] = make_double2(0.0, 0.0);
  for (size_t e = lane; e < (size_t)a.F * B.slots_max * B.Lmax; e += 32) Dw[e] = make_double2(0.0, 0.0);
  __syncwarp();

  const int t0 = chunk * B.tiles_per_cta;
  const int t1 = min(a.n_tiles, t0 + B.tiles_per_cta);
  int32_t rows[NCMAX];
  for (int tile = t0; tile < t1; tile++) {
    const int64_t jraw = (int64_t)tile * T + tid;
    const bool valid = jraw < a.n_snk;
    const int64_t j = valid ? jraw : a.n_snk - 1;  // sink position
    const int32_t* cols = dev::sink_cols(a, j);
    const int64_t jo = a.snk_orig ? a.snk_orig[j] : j;
    const bool jpar = a.snk_orig && (__popc(a.snk_par[j]) & 1);
    const double wj = valid ? (jpar ? -a.w_snk[jo] : a.w_snk[jo]) : 0.0;
    const int Q = a.snk_orig ? a.snk_q[j] : -1;
    const bool qtwo = Q >= 0 && a.q_two[Q];

    // ---- pass 1: cached solves, member dets (fresh where guarded), dw partials --------
    unsigned pguard = 0;
    dev::ScalesFor<NCMAX> eys;
    for (int f = 0; f < a.F; f++) {
      const int n = a.n_f[f];
      int ey = 0;
      if (n == 0) continue;
      const int32_t* arow = a.fam_arow + (int64_t)W * a.Tn + a.off_f[f];
      const int rho = a.fam_rank[(int64_t)W * a.F + f];
      const int sig = qtwo ? a.q_rank[(int64_t)Q * a.F + f] : 0;
      if (qtwo && (rho == 1 || sig == 1 || (rho == 2 && sig == 2)) &&
          !a.kguard[((int64_t)W * a.n_q + Q) * a.F + f]) {
        // two-sided block: y (z1, z2 for two-row families) from the stored factors
        const double2* K = a.kbuf + ((int64_t)W * a.n_q + Q) * a.kstride + a.koff[f];
        if (rho == 2 && sig == 2)
          dev::dispatch_kapply22<NCMAX>(n, a.S[f], a.L_f[f], arow, cols + a.off_f[f], K,
                                        Ysm + (size_t)a.yoff[f] * T + tid, T, &ey);
        else if (rho == 2)
          dev::dispatch_kapply2<NCMAX>(n, a.S[f], a.L_f[f], arow, cols + a.off_f[f], K,
                                       Ysm + (size_t)a.yoff[f] * T + tid, T, &ey);
        else if (sig == 2)
          dev::dispatch_kapply12<NCMAX>(n, a.S[f], a.L_f[f], arow, cols + a.off_f[f], K,
                                        Ysm + (size_t)a.yoff[f] * T + tid, T, &ey);
        else
          dev::dispatch_kapply<NCMAX>(n, a.S[f], a.L_f[f], arow, cols + a.off_f[f], K,
                                      Ysm + (size_t)a.yoff[f] * T + tid, T, &ey);
      } else {
        const bool g = dev::dispatch_shared<NCMAX>(n, rho, a.S[f], a.L_f[f], arow, cols + a.off_f[f],
                                                   Ysm + (size_t)a.yoff[f] * T + tid, T, &ey, a.kp);
        pguard |= (unsigned)g << f;
      }
      eys.set(f, ey);
    }
    double2 accj = make_double2(0.0, 0.0);
    for (int c = 0; c < kW; c++) {
      const int m = mem0 + c;
      double2 prod = make_double2(1.0, 0.0);
      for (int f = 0; f < a.F; f++) {
        const int n = a.n_f[f];
        cd d = make_double2(1.0, 0.0);
        if (n > 0) {
          bool fail = (pguard >> f) & 1;
          const int32_t* col = cols + a.off_f[f];
          const int rho = a.fam_rank[(int64_t)W * a.F + f];
          const bool lemma = !fail;  // the member's own guard decides (not the pivot guard)
          if (!fail)
            d = dev::dispatch_member<NCMAX>(n, rho, a.S[f], a.L_f[f], a.mem_lab + ((int64_t)m * a.F + f) * MHC_MAX_RANK,
                                            col, Ysm + (size_t)a.yoff[f] * T + tid, T, eys.get(f), a.kc, &fail);
          if (fail && lemma && rho <= 2 && n >= rho + 1 && a.rowdiff) {  // as in the forward
            bool f2 = true;
            const int32_t* mlab = a.mem_lab + ((int64_t)m * a.F + f) * MHC_MAX_RANK;
            const int32_t* arow = a.fam_arow + (int64_t)W * a.Tn + a.off_f[f];
            const cd* Yf = Ysm + (size_t)a.yoff[f] * T + tid;
            cd d2;
            if constexpr (NCMAX >= 10)  // two-row families need n_f >= 10
              d2 = rho == 1 ? dev::rowdiff_det(a.S[f], a.L_f[f], n, mlab[0], arow, col, Yf, T, eys.get(f), a.kc, &f2)
                            : dev::rowdiff2_det(a.S[f], a.L_f[f], n, mlab, arow, col, Yf, T, eys.get(f), a.kc, &f2);
            else
              d2 = dev::rowdiff_det(a.S[f], a.L_f[f], n, mlab[0], arow, col, Yf, T, eys.get(f), a.kc, &f2);
            if (!f2) {
              d = d2;
              fail = false;
            }
          }
          if (fail) {
            dev::member_rows(a, W, m, f, rho, rows);
            d = dev::dispatch_fresh<NCMAX>(n, a.S[f], a.L_f[f], rows, col);
          }
        }
        Dets[dix(c, f, B.kmax, T, tid)] = d;
        prod = f == 0 ? d : dev::cmul(prod, d);
      }
      double wc = a.w_src[a.mem_term[m]];
      if (__popc(a.mem_par[m]) & 1) wc = -wc;
      accj.x = fma(wc, prod.x, accj.x);
      accj.y = fma(wc, prod.y, accj.y);
      cd& s = AccS[c * T + tid];
      s.x = fma(wj, prod.x, s.x);
      s.y = fma(wj, prod.y, s.y);
      // gamma_{c,f} = w_c w_j sign prod_{f' != f} det_{f'}, the weight of member c's
      // cofactors in flavour f; it replaces the member's dets, which are not read again
      const double wcj = wc * wj;
      if (a.F == 2) {
        const cd d0 = Dets[dix(c, 0, B.kmax, T, tid)], d1 = Dets[dix(c, 1, B.kmax, T, tid)];
        Dets[dix(c, 0, B.kmax, T, tid)] = make_double2(wcj * d1.x, wcj * d1.y);
        Dets[dix(c, 1, B.kmax, T, tid)] = make_double2(wcj * d0.x, wcj * d0.y);
      } else {
        cd dd[MHC_FMAX];
        for (int f = 0; f < a.F; f++) dd[f] = Dets[dix(c, f, B.kmax, T, tid)];
        for (int f = 0; f < a.F; f++) {
          cd g = make_double2(wcj, 0.0);
          for (int f2 = 0; f2 < a.F; f2++)
            if (f2 != f) g = dev::cmul(g, dd[f2]);
          Dets[dix(c, f, B.kmax, T, tid)] = g;
        }
      }
    }
    if (jpar) accj = dev::cneg(accj);  // back to the sink's own column order
    if (valid) B.dwsnk_part[(int64_t)W * a.n_snk + jo] = accj;

    // ---- pass 2 per flavour: h, shared-row cofactors, scatter -------------------------
    for (int f = 0; f < a.F; f++) {
      const int n = a.n_f[f];
      if (n == 0) continue;
      const int M = n - 1;
      const int32_t* col = cols + a.off_f[f];
      const int32_t* arow = a.fam_arow + (int64_t)W * a.Tn + a.off_f[f];
      if constexpr (NCMAX >= 10) {
        const int rho = a.fam_rank[(int64_t)W * a.F + f];
        if (rho >= 2) {  // rank-k families (k = 2 .. MHC_MAX_RANK; rank k needs n_f >= 4k + 2)
          cd* Rk = B.r2 + (size_t)cta * B.kmax * B.rk2 * T;
          const bool gd = (pguard >> f) & 1;
          const int64_t rem = a.n_snk - ((int64_t)tile * T + warp * 32);
          const int nlive = rem < 32 ? (int)rem : 32;
          const int mynsh = qtwo ? n - a.q_rank[(int64_t)Q * a.F + f] : 0;
          cd* Df = Dw + (size_t)f * B.slots_max * B.Lmax;
#define MHC_RB(K) rank_block<NCMAX, K>(a, B, f, n, mem0, kW, tid, T, warp, lane, nlive, col, arow, Dets, Ysm, gd, \
                                       myStage, Stage, Rk, qtwo ? Q : -1, mynsh, Df)
          if (rho == 2) {
            MHC_RB(2);
          } else if constexpr (NCMAX >= 14) {
            if (rho == 3) {
              MHC_RB(3);
            } else if constexpr (NCMAX >= 18) {
              if (rho == 4) {
                MHC_RB(4);
              } else if constexpr (NCMAX >= 32) {
                if (rho == 5) MHC_RB(5);
                if (rho == 6) MHC_RB(6);
              }
            }
          }
#undef MHC_RB
          continue;
        }
      }
      const int64_t blk = ((int64_t)W * a.n_q + Q) * a.F + f;
      const bool twoc = B.kinv && qtwo && n >= 2 && a.q_rank[(int64_t)Q * a.F + f] == 1 && !a.kguard[blk];
      const int64_t wq = (int64_t)W * a.n_q + Q;
      // B^{-1} shared by the (family, sink family) block
      const cd* Binv = twoc ? B.kinv + wq * B.kistride + B.kioff[f] : nullptr;
      const cd detB = twoc ? a.kbuf[wq * a.kstride + a.koff[f] + M * M + M + 1] : make_double2(0.0, 0.0);
      dispatch_cof_pass<NCMAX>(a, B, f, n, W, mem0, kW, wj, tid, T, col, arow, Dets,
                               Ysm + (size_t)a.yoff[f] * T + tid, (pguard >> f) & 1, Binv, detB, myStage);
      __syncwarp();

      // warp scatter: the block's (row, column) cells dealt to the lanes (rows s < M: shared
      // rows; else member s - M)
      const int mynsh = qtwo ? n - a.q_rank[(int64_t)Q * a.F + f] : 0;
      const int64_t rem = a.n_snk - ((int64_t)tile * T + warp * 32);
      const int nlive = rem < 32 ? (int)rem : 32;
      dispatch_scatter<NCMAX>(a, B, f, n, kW, mem0, nlive, T, warp, lane, col, qtwo ? Q : -1, mynsh,
                              Stage, Ysm, Dets, Dw + (size_t)f * B.slots_max * B.Lmax);
      __syncwarp();
    }
  }
  __syncthreads();
  // dw_src partials of this chunk: fixed-order sum over the block's threads
  for (int c = tid; c < kW; c += T) {
    cd s = AccS[c * T];
    for (int t = 1; t < T; t++) {
      s.x += AccS[c * T + t].x;
      s.y += AccS[c * T + t].y;
    }
    if (__popc(a.mem_par[mem0 + c]) & 1) s = dev::cneg(s);  // member sign
    B.dwsrc_part[(int64_t)(mem0 + c) * B.n_chunks + chunk] = s;
  }
}

}  // namespace bwd

template <int NCMAX>
cudaError_t launch_kinv_nc(const BwdArgs& b, int64_t n_fam, cudaStream_t s) {
  const int64_t threads = n_fam * b.a.n_q * b.a.F;
  if (threads == 0) return cudaSuccess;
  bwd::kinv_kernel<NCMAX><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(b, n_fam);
  return cudaGetLastError();
}

template <int NCMAX>
cudaError_t launch_bwd_nc(const BwdArgs& b, int T, int64_t ctas, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(bwd::bwd_kernel<NCMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  bwd::bwd_kernel<NCMAX><<<(unsigned)ctas, T, smem, s>>>(b);
  return cudaGetLastError();
}

}  // namespace mhc
