// fwd_impl.cuh -- forward correlator kernel and per-pair probe (templates; instantiated
// once per n class by fwd_nc8.cu, fwd_nc18.cu and fwd_nc32.cu).
//
// One thread block per work item (work family W, tile of `tile` sinks); one thread per
// sink.  Per flavour a thread factorises the family's shared rows against its sink's
// columns (shared_rows) and caches y = det(G) G^{-1} e_r in shared memory; then every
// member of the family costs one O(n) dot product per flavour (member_det), Sec. 2.1.
// Two-sided blocks (a family against a sink family) take y from factors stored once per
// block (kapply*).  Members whose lemma factor or whose family pivots fail the guards go
// to a per-warp queue and are refactored from scratch 32 at a time -- pairs that share the
// member and the sink family's columns as one group (group_fresh), so the FP64 pipe stays
// occupied.  Thread sums are reduced in a fixed order into one partial per work item (and
// by reduce_kernel into C): bitwise reproducible.
#pragma once

#include "kernels.cuh"

namespace mhc {

namespace fwd {

struct QEntry {
  int32_t member;  // member slot
  int32_t lane;    // lane (sink) of the warp that produced it
  int32_t fail;    // flavours to refactor (bit f)
  int32_t pguard;  // of those, the flavours whose shared rows failed the pivot guard
  double2 prod;    // product of the flavours that did not fail
  double w;        // signed w_i w_j of the pair
  double pad2;
};

// Algorithmic flops of the refactor path, counted with the planner's rule (real add/mul 1,
// FMA 2, complex multiply 6, complex FMA 8, complex reciprocal 6, pivot measure 1):
// a fresh partial-pivot LU determinant of one n x n block, ...
__device__ __forceinline__ unsigned long long fresh_flops(int n) {
  const long long m = n;
  return (unsigned long long)(m * (m + 1) / 2 + 6 * (m - 1) + 3 * m * (m - 1) +
                              8 * (m - 1) * m * (2 * m - 1) / 6 + 6 * (m - 1));
}
// ... and a grouped refactor (group_fresh) of pairs whose matrices share their first
// n - rc columns: the group's elimination of those columns and the rows of L^{-1} P of the
// rc remaining rows (one complex multiply-add per unused row and step) ...
__device__ __forceinline__ unsigned long long group_shared_flops(int n, int rc) {
  long long f = 0;
  const int M = n - rc;
  for (int k = 0; k < M; k++)
    f += (n - k) + 6 + 6 * (n - k - 1) + 8 * (n - k - 1) * (M - 1 - k) + 8 * rc * (n - k - 1);
  return (unsigned long long)(f + 6 * (M > 1 ? M - 1 : 0));
}
// ... and each pair's share: rc x rc dot products of length n, the last rc x rc step (for
// rc = 2: two pivot measures, a reciprocal, a multiplier, one update, two products) and
// the product with the shared pivots.
__device__ __forceinline__ unsigned long long group_pair_flops(int n, int rc) {
  return (unsigned long long)(rc * rc * (8LL * n - 2) + (rc == 2 ? 2 + 6 + 6 + 8 + 12 : 6));
}

// Pivot search of one step of group_fresh: the largest |re| + |im| in column k (rk: this
// lane's entry) among the unused rows, by one warp-wide maximum of a key made of the
// measure's sign, exponent and leading 15 mantissa bits with (31 - lane) below them: a pivot
// within 2^-15 of the largest, the lowest row of those -- partial pivoting up to that tie
// tolerance; a zero measure keeps key bits 5..31 zero, which is how an exactly zero pivot
// column shows.  Updates the used rows, the permutation's parity, the determinant and the
// pivot's reciprocal.  Called by the whole warp.
struct PivotState {
  unsigned piv;  // rows already used as pivots
  int mystep;    // the step at which this lane's row became the pivot (NC: never)
  int parity;
  bool zero;
  dev::cd det;
  int p;         // this step's pivot row
  dev::cd rc;    // its reciprocal
};
__device__ __forceinline__ void select_pivot(PivotState& s, dev::cd rk, int k, int n, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  const bool cand = lane < n && !((s.piv >> lane) & 1);
  const unsigned mkey = cand ? (((unsigned)__double2hiint(dev::abs1(rk)) & ~31u) | (unsigned)(31 - lane)) : 0u;
  const unsigned top = __reduce_max_sync(FULL, mkey);
  const int p = 31 - (int)(top & 31u);
  // the permutation's parity: p moves ahead of the unused rows that precede it
  s.parity ^= __popc(~s.piv & ((1u << p) - 1u) & ((1u << n) - 1u)) & 1;
  s.piv |= 1u << p;
  s.mystep = lane == p ? k : s.mystep;
  s.zero |= (top >> 5) == 0u;
  const dev::cd pk = make_double2(__shfl_sync(FULL, rk.x, p), __shfl_sync(FULL, rk.y, p));
  s.det = (k == 0) ? pk : dev::cmul(s.det, pk);
  s.rc = dev::crcp(pk);
  s.p = p;
}

// Fresh determinants of a group of queued pairs that share member m and a two-sided sink
// family Q whose members change RC columns of flavour f (RC = 1 or 2; family of rank rho):
// their matrices G = [R | A_j] agree in the first n - RC columns R (the family's n - rho
// shared rows and the member's rho rows, in member_rows order, against the sink family's
// shared columns) and differ in the last RC columns A_j.  Partial-pivot LU eliminates
// column by column, so the first n - RC steps are those of R for every pair: P R = L [U; 0],
// and the last RC rows of L^{-1} P A_j form the RC x RC block that the last steps factorise,
// det G = sign(P) det(U) det(V A_j) with V the rows of L^{-1} P that belong to the RC rows
// left after the shared steps.  The warp factorises R once (lane i holds row i and keeps
// its multiplier of every step), forms V by walking the steps backwards (the coefficient of
// a step's pivot row is minus the warp sum, over the rows still unused at that step, of
// multiplier times coefficient), and each lane of the group then needs RC x RC dot products
// of length n with its own sink's columns and the last RC x RC step with the same pivot
// rule.  Called by the whole warp; returns the determinant on the lanes in grp.
template <int NC, int RC>
__device__ __forceinline__ dev::cd group_fresh(const FwdArgs& a, int W, int f, int rho, int m, int Q,
                                               int64_t j, unsigned grp, dev::cd* wk) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int NR = NC - RC > 0 ? NC - RC : 1;
  const int lane = threadIdx.x & 31;
  const int n = a.n_f[f];
  const int M = n - RC;  // shared columns: the common elimination steps
  const int L = a.L_f[f];
  const dev::cd* S = a.S[f];
  const int32_t* arow = a.fam_arow + (int64_t)W * a.Tn + a.off_f[f];
  const int32_t* mlab = a.mem_lab + ((int64_t)m * a.F + f) * MHC_MAX_RANK;
  const int32_t* scol = a.snk_pos + (int64_t)a.q_off[Q] * a.Tn + a.off_f[f];
  // label of row i: the family's shared rows, then the member's changed rows
  auto row_label = [&](int i) { return i < n - rho ? arow[i] : mlab[min(i - (n - rho), rho - 1)]; };
  const int rlab = row_label(min(lane, n - 1));
  dev::cd R[NR];
#pragma unroll
  for (int u = 0; u < NR; u++)
    R[u] = (lane < n && u < M) ? dev::ldS(S + (size_t)rlab * L + scol[u]) : make_double2(0.0, 0.0);
  PivotState ps;
  ps.piv = 0;
  ps.mystep = NC;
  ps.parity = 0;
  ps.zero = false;
  ps.det = make_double2(1.0, 0.0);
  if (M > 0) select_pivot(ps, R[0], 0, n, lane);
  // Step k: the multipliers of column k, then column k + 1 updated first and the pivot of
  // step k + 1 chosen (with its reciprocal) before the other columns of step k, so that the
  // chain of the next pivot (maximum, broadcast, reciprocal) overlaps independent updates.
  // The values are those of the plain order: each entry sees the same operations.
#pragma unroll
  for (int k = 0; k < NR; k++) {
    if (k >= M) break;
    const int p = ps.p;
    const bool act = lane < n && !((ps.piv >> lane) & 1);
    const dev::cd l = dev::cmul(R[k], ps.rc);
    if (k + 1 < NR && k + 1 < M) {
      const dev::cd pu = make_double2(__shfl_sync(FULL, R[k + 1].x, p), __shfl_sync(FULL, R[k + 1].y, p));
      if (act) R[k + 1] = dev::cfms(l, pu, R[k + 1]);
      select_pivot(ps, R[k + 1], k + 1, n, lane);
    }
#pragma unroll
    for (int u = k + 2; u < NR; u++) {
      if (u >= M) break;
      const dev::cd pu = make_double2(__shfl_sync(FULL, R[u].x, p), __shfl_sync(FULL, R[u].y, p));
      if (act) R[u] = dev::cfms(l, pu, R[u]);
    }
    if (act) R[k] = l;  // this row's multiplier of step k
  }
  const unsigned piv = ps.piv;
  const int mystep = ps.mystep;
  int parity = ps.parity;
  bool zero = ps.zero;
  dev::cd det = ps.det;
  // the RC rows left after the shared steps, ascending
  const unsigned rest = ~piv & ((1u << n) - 1u);
  int left[RC];
  left[0] = __ffs(rest) - 1;
  if (RC == 2) left[RC - 1] = __ffs(rest & ~(1u << left[0])) - 1;
  // V: lane i holds the coefficient of row i in each remaining row's functional.  In the
  // order of the steps (position s < M: the pivot row of step s; M + t: the t-th remaining
  // row), the functional's coefficient at position s is minus the sum, over the later
  // positions s', of the multiplier of row s' at step s times the coefficient at s' -- a
  // back substitution with the unit lower factor.  The multipliers are staged by step in
  // the warp's shared scratch wk (column s: positions s + 1 .. n - 1, packed), and the
  // substitution runs as pushes: once position s' is final it is broadcast and every
  // earlier position adds its term, so the dependency chain per position is one shuffle and
  // one complex multiply-add.
  const int pos = mystep < NC ? mystep : (lane == left[0] ? M : M + RC - 1);
  auto woff = [&](int c) { return c * (n - 1) - c * (c - 1) / 2; };  // column c of the packed store
  __syncwarp();
#pragma unroll
  for (int k = 0; k < NR; k++) {
    if (k >= M) break;
    if (lane < n && k < pos) wk[woff(k) + pos - k - 1] = R[k];  // this row's multiplier at step k
  }
  __syncwarp();
  dev::cd acc[RC];
#pragma unroll
  for (int t = 0; t < RC; t++)  // the remaining rows: coefficient 1 in their own functional
    acc[t] = lane < M ? wk[woff(lane) + M + t - lane - 1] : make_double2(0.0, 0.0);
#pragma unroll
  for (int sp = NR - 1; sp >= 1; sp--) {
    if (sp >= M) continue;
    dev::cd v[RC];
#pragma unroll
    for (int t = 0; t < RC; t++)
      v[t] = dev::cneg(make_double2(__shfl_sync(FULL, acc[t].x, sp), __shfl_sync(FULL, acc[t].y, sp)));
    if (lane < sp) {
      const dev::cd w = wk[woff(lane) + sp - lane - 1];
#pragma unroll
      for (int t = 0; t < RC; t++) acc[t] = dev::cfma(w, v[t], acc[t]);
    }
  }
  // back to row order: row i takes the coefficient of its position
  const int src = pos < M ? pos : 0;
  dev::cd V[RC];
#pragma unroll
  for (int t = 0; t < RC; t++) {
    const dev::cd x = make_double2(-__shfl_sync(FULL, acc[t].x, src), -__shfl_sync(FULL, acc[t].y, src));
    V[t] = lane >= n ? make_double2(0.0, 0.0) : pos < M ? x : make_double2(pos == M + t ? 1.0 : 0.0, 0.0);
  }
  // each lane: its sink's last RC columns against the RC functionals
  const bool mine = (grp >> lane) & 1;
  const int32_t* cj = dev::sink_cols(a, j) + a.off_f[f];
  dev::cd D[RC][RC];
#pragma unroll
  for (int t = 0; t < RC; t++)
#pragma unroll
    for (int u = 0; u < RC; u++) D[t][u] = make_double2(0.0, 0.0);
  int lc[RC];
#pragma unroll
  for (int u = 0; u < RC; u++) lc[u] = mine ? cj[n - RC + u] : 0;
#pragma unroll
  for (int i = 0; i < NC; i++) {
    if (i >= n) break;
    const int li = row_label(i);
    dev::cd vi[RC];
#pragma unroll
    for (int t = 0; t < RC; t++) vi[t] = make_double2(__shfl_sync(FULL, V[t].x, i), __shfl_sync(FULL, V[t].y, i));
#pragma unroll
    for (int u = 0; u < RC; u++) {
      const dev::cd x = mine ? dev::ldS(S + (size_t)li * L + lc[u]) : make_double2(0.0, 0.0);
#pragma unroll
      for (int t = 0; t < RC; t++) D[t][u] = dev::cfma(vi[t], x, D[t][u]);
    }
  }
  if (RC == 1) {
    zero |= __double_as_longlong(dev::abs1(D[0][0])) == 0;
    det = M == 0 ? D[0][0] : dev::cmul(det, D[0][0]);
  } else {
    // last 2 x 2 step: pivot the larger |re| + |im| of the first column, ties to the lower row
    const double b0 = dev::abs1(D[0][0]), b1 = dev::abs1(D[RC - 1][0]);
    const bool swp = dev::gt_nonneg(b1, b0);
    parity ^= (int)swp;
    const dev::cd pv = swp ? D[RC - 1][0] : D[0][0], ov = swp ? D[0][0] : D[RC - 1][0];
    const dev::cd pw = swp ? D[RC - 1][RC - 1] : D[0][RC - 1], ow = swp ? D[0][RC - 1] : D[RC - 1][RC - 1];
    zero |= __double_as_longlong(swp ? b1 : b0) == 0;
    const dev::cd l = dev::cmul(ov, dev::crcp(pv));
    const dev::cd last = dev::cfms(l, pw, ow);
    zero |= __double_as_longlong(dev::abs1(last)) == 0;
    det = M == 0 ? dev::cmul(pv, last) : dev::cmul(dev::cmul(det, pv), last);
  }
  if (zero) return make_double2(0.0, 0.0);
  return parity ? dev::cneg(det) : det;
}

// Refactor one pair per lane (the lanes with have; e: the pair, j: its sink position):
// the product of the flavours that passed, times fresh determinants of the flavours that
// failed, accumulated into acc.  With a.rowdiff the row-difference update is tried first
// for members of one- and two-row families.  Pairs that share a member and a two-sided sink
// family with one or two changed columns (n <= 18) are factorised together (group_fresh);
// the others one per lane.  Yw: the warp's cached solves (lane l at Yw + l, stride
// blockDim.x); wk: the warp's scratch for group_fresh.  Called by the whole warp.
template <int NCMAX>
__device__ void process_pairs(const FwdArgs& a, int W, bool have, const QEntry& e, int64_t j,
                              const double2* Yw, double2* wk, double2& acc, unsigned long long& rflops,
                              unsigned long long& nrd) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int T = blockDim.x;
  const int32_t* cols = dev::sink_cols(a, j);
  double2 prod = have ? e.prod : make_double2(1.0, 0.0);
  int32_t fail = have ? e.fail : 0;
  const int Q = a.snk_orig ? a.snk_q[j] : -1;
  if (a.rowdiff && have) {
    // members of one- and two-row families that failed the lemma guard (not the pivot
    // guard): the row-difference update with the cached solve of the pair's sink (lane
    // e.lane of this warp) and its scale exponent as the solve's producer defines it
    const unsigned cand = (unsigned)(e.fail & ~e.pguard);
    for (int f = 0; f < a.F; f++) {
      const int n = a.n_f[f];
      const int rho = a.fam_rank[(int64_t)W * a.F + f];
      if (!((cand >> f) & 1) || rho > 2 || n < rho + 1) continue;
      const double2* Yf = Yw + (size_t)a.yoff[f] * T + e.lane;
      const int ey = dev::cached_scale(Yf, T, n, rho);
      bool f2 = true;
      const int32_t* mlab = a.mem_lab + ((int64_t)e.member * a.F + f) * MHC_MAX_RANK;
      const int32_t* arow = a.fam_arow + (int64_t)W * a.Tn + a.off_f[f];
      double2 d;
      if constexpr (NCMAX >= 10)  // two-row families need n_f >= 10
        d = rho == 1 ? dev::rowdiff_det(a.S[f], a.L_f[f], n, mlab[0], arow, cols + a.off_f[f], Yf, T, ey, a.kc, &f2)
                     : dev::rowdiff2_det(a.S[f], a.L_f[f], n, mlab, arow, cols + a.off_f[f], Yf, T, ey, a.kc, &f2);
      else
        d = dev::rowdiff_det(a.S[f], a.L_f[f], n, mlab[0], arow, cols + a.off_f[f], Yf, T, ey, a.kc, &f2);
      rflops += rho == 1 ? dev::rowdiff_flops(n) : dev::rowdiff2_flops(n);
      if (!f2) {
        prod = dev::cmul(prod, d);
        fail &= ~(1 << f);
        nrd++;
      }
    }
  }
  int32_t rows[NCMAX];
  for (int f = 0; f < a.F; f++) {
    const bool need = have && ((fail >> f) & 1);
    const int n = a.n_f[f];
    const int rho = a.fam_rank[(int64_t)W * a.F + f];
    const int sig = (Q >= 0 && a.q_two[Q]) ? a.q_rank[(int64_t)Q * a.F + f] : 0;
    const bool grouped = need && NCMAX <= 18 && n >= 2 && sig == 1;
    const bool grouped2 = need && NCMAX <= 18 && n >= 3 && sig == 2;
    unsigned todo = __ballot_sync(FULL, grouped || grouped2);
    while (todo) {
      const int leader = __ffs(todo) - 1;
      const int lm = __shfl_sync(FULL, have ? e.member : 0, leader);
      const int lq = __shfl_sync(FULL, Q, leader);
      const int lsig = __shfl_sync(FULL, sig, leader);
      const unsigned grp = __ballot_sync(FULL, ((todo >> lane) & 1) && e.member == lm && Q == lq);
      const double2 d = lsig == 1 ? group_fresh<NCMAX <= 18 ? NCMAX : 18, 1>(a, W, f, rho, lm, lq, j, grp, wk)
                                  : group_fresh<NCMAX <= 18 ? NCMAX : 18, 2>(a, W, f, rho, lm, lq, j, grp, wk);
      if ((grp >> lane) & 1) {
        prod = dev::cmul(prod, d);
        rflops += group_pair_flops(n, lsig) + (lane == leader ? group_shared_flops(n, lsig) : 0ull);
      }
      todo &= ~grp;
    }
    if (need && !grouped && !grouped2) {
      dev::member_rows(a, W, e.member, f, rho, rows);
      const double2 d = dev::dispatch_fresh<NCMAX>(n, a.S[f], a.L_f[f], rows, cols + a.off_f[f]);
      prod = dev::cmul(prod, d);
      rflops += fresh_flops(n);
    }
  }
  if (have) {
    acc.x = fma(e.w, prod.x, acc.x);
    acc.y = fma(e.w, prod.y, acc.y);
  }
}

// Refactor the first count queued pairs (one per lane).  Called by the whole warp.
template <int NCMAX>
__device__ void process_queue(const FwdArgs& a, int W, QEntry* q, int count, int64_t jbase,
                              const double2* Yw, double2* wk, double2& acc, unsigned long long& rflops,
                              unsigned long long& nrd) {
  const int lane = threadIdx.x & 31;
  const bool have = lane < count;
  QEntry e = {};
  if (have) e = q[lane];
  process_pairs<NCMAX>(a, W, have, e, jbase + (have ? e.lane : 0), Yw, wk, acc, rflops, nrd);
}

// One work item (family W x sink tile) by the whole thread block; the block's sum goes
// to *partial.  Shared by the per-plan launch and the persistent batched launch.
template <int NCMAX>
__device__ __forceinline__ void fwd_item(const FwdArgs& a, int W, int tile, double2* smem,
                                         double2* partial) {
  const int T = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t jraw = (int64_t)tile * T + tid;
  const bool valid = jraw < a.n_snk;
  const int64_t j = valid ? jraw : a.n_snk - 1;  // sink position
  const int32_t* cols = dev::sink_cols(a, j);
  const int Q = a.snk_orig ? a.snk_q[j] : -1;
  const bool qtwo = Q >= 0 && a.q_two[Q];
  const int mem0 = a.fam_info[4 * W], kW = a.fam_info[4 * W + 1];
  QEntry* queue = reinterpret_cast<QEntry*>(smem + (size_t)a.slots * T) + warp * kQueueCap;
  double2* Y = smem + tid;
  const double2* Yw = smem + (tid & ~31);  // the warp's cached solves (lane l: Yw + l)

  // ---- per flavour: factorise the shared rows against this sink ----------------------
  unsigned pguard = 0;
  dev::ScalesFor<NCMAX> eys;
  for (int f = 0; f < a.F; f++) {
    const int n = a.n_f[f];
    int ey = 0;
    if (n == 0) continue;
    const int rho = a.fam_rank[(int64_t)W * a.F + f];
    const int32_t* arow = a.fam_arow + (int64_t)W * a.Tn + a.off_f[f];
    const int sig = qtwo ? a.q_rank[(int64_t)Q * a.F + f] : 0;
    if (qtwo && (rho == 1 || sig == 1 || (rho == 2 && sig == 2)) &&
        !a.kguard[((int64_t)W * a.n_q + Q) * a.F + f]) {
      const double2* K = a.kbuf + ((int64_t)W * a.n_q + Q) * a.kstride + a.koff[f];
      if (rho == 2 && sig == 2)
        dev::dispatch_kapply22<NCMAX>(n, a.S[f], a.L_f[f], arow, cols + a.off_f[f], K,
                                      Y + (size_t)a.yoff[f] * T, T, &ey);
      else if (rho == 2)
        dev::dispatch_kapply2<NCMAX>(n, a.S[f], a.L_f[f], arow, cols + a.off_f[f], K,
                                     Y + (size_t)a.yoff[f] * T, T, &ey);
      else if (sig == 2)
        dev::dispatch_kapply12<NCMAX>(n, a.S[f], a.L_f[f], arow, cols + a.off_f[f], K,
                                      Y + (size_t)a.yoff[f] * T, T, &ey);
      else
        dev::dispatch_kapply<NCMAX>(n, a.S[f], a.L_f[f], arow, cols + a.off_f[f], K,
                                    Y + (size_t)a.yoff[f] * T, T, &ey);
    } else {
      const bool g = dev::dispatch_shared<NCMAX>(n, rho, a.S[f], a.L_f[f], arow, cols + a.off_f[f],
                                                 Y + (size_t)a.yoff[f] * T, T, &ey, a.kp);
      pguard |= (unsigned)g << f;
    }
    eys.set(f, ey);
  }

  // ---- rank-2 flavours against a one-column sink family shared by the warp's sinks: the
  // members' dots with the block's first null vector, once per warp (lane t: member t) -----
  // (two-row families need n_f >= 10: the classes below compile none of this)
  constexpr bool kZ1 = NCMAX >= 10;
  int zf0 = -1, zf1 = -1;
  double2* z1d = reinterpret_cast<double2*>(reinterpret_cast<char*>(smem + (size_t)a.slots * T) +
                                            (size_t)(T >> 5) * kQueueCap * kQueueEntryBytes +
                                            (size_t)warp * kZ1Bytes);
  // the warp's scratch for the grouped refactors' multipliers (group_fresh)
  double2* wk = reinterpret_cast<double2*>(reinterpret_cast<char*>(smem + (size_t)a.slots * T) +
                                           (size_t)(T >> 5) * (kQueueCap * kQueueEntryBytes + kZ1Bytes) +
                                           (size_t)warp * kWalkBytes);
  // (the shuffle and the vote run on every lane: qtwo differs between lanes whose sinks
  // belong to a two-sided family and lanes whose sinks stand alone)
  const int Q0 = kZ1 ? __shfl_sync(0xffffffffu, Q, 0) : 0;
  const bool z1_warp = kZ1 && __all_sync(0xffffffffu, qtwo && Q == Q0);
  if (kZ1 && z1_warp && kW <= 32) {
    // the flavours are chosen from warp-uniform data only (W, Q), so every lane assigns the
    // same slots; such a flavour took kapply2 on every lane
    for (int f = 0; f < a.F && zf1 < 0; f++) {
      const int n = a.n_f[f];
      if (n == 0 || a.fam_rank[(int64_t)W * a.F + f] != 2 || a.q_rank[(int64_t)Q * a.F + f] != 1 ||
          a.kguard[((int64_t)W * a.n_q + Q) * a.F + f])
        continue;
      const int slot = zf0 < 0 ? 0 : 1;
      if (lane < kW) {
        double2 d11, d21;
        dev::dispatch_dots_z1<NCMAX>(n, a.S[f], a.L_f[f],
                                     a.mem_lab + ((int64_t)(mem0 + lane) * a.F + f) * MHC_MAX_RANK,
                                     cols + a.off_f[f], Y + (size_t)a.yoff[f] * T, T, &d11, &d21);
        z1d[(slot * 32 + lane) * 2] = d11;
        z1d[(slot * 32 + lane) * 2 + 1] = d21;
      }
      if (slot == 0) zf0 = f; else zf1 = f;
    }
    __syncwarp();
  }

  // ---- per member: one dot product per flavour --------------------------------------
  double wj = valid ? a.w_snk[a.snk_orig ? a.snk_orig[j] : j] : 0.0;
  if (a.snk_orig && (__popc(a.snk_par[j]) & 1)) wj = -wj;
  // acc: sum over the members of w_i prod_f det (this lane's sink; times w_j once, at the
  // end); accq: the refactored pairs, w_i w_j included (a queue lane holds other sinks' pairs)
  double2 acc = make_double2(0.0, 0.0), accq = make_double2(0.0, 0.0);
  int qn = 0;
  unsigned long long n_parent = 0, n_child = 0, n_rowdiff = 0, rflops = 0;
  for (int c = 0; c < kW; c++) {
    const int m = mem0 + c;
    unsigned fail = pguard;
    double2 prod = make_double2(1.0, 0.0);
    bool first = true;
    for (int f = 0; f < a.F; f++) {
      const int n = a.n_f[f];
      if (n == 0 || ((pguard >> f) & 1)) continue;
      const int rho = a.fam_rank[(int64_t)W * a.F + f];
      bool cf = false;
      const int32_t* mlab = a.mem_lab + ((int64_t)m * a.F + f) * MHC_MAX_RANK;
      const double2* Yf = Y + (size_t)a.yoff[f] * T;
      double2 d;
      if (kZ1 && (f == zf0 || f == zf1)) {
        const double2* zd = z1d + ((f == zf0 ? 0 : 32) + c) * 2;
        d = dev::dispatch_member_z1<NCMAX>(n, a.S[f], a.L_f[f], mlab, cols + a.off_f[f], Yf, T, eys.get(f),
                                           a.kc, &cf, zd[0], zd[1]);
      } else {
        d = dev::dispatch_member<NCMAX>(n, rho, a.S[f], a.L_f[f], mlab, cols + a.off_f[f], Yf, T, eys.get(f),
                                        a.kc, &cf);
      }
      if (cf) {
        fail |= 1u << f;
      } else {
        prod = first ? d : dev::cmul(prod, d);
        first = false;
      }
    }
    const bool need = valid && fail != 0;
    double wi = a.w_src[a.mem_term[m]];
    if (__popc(a.mem_par[m]) & 1) wi = -wi;
    if (!fail) {
      acc.x = fma(wi, prod.x, acc.x);
      acc.y = fma(wi, prod.y, acc.y);
    }
    const unsigned ball = __ballot_sync(0xffffffffu, need);
    if (ball == 0xffffffffu) {
      // every lane refactors this member (a member near-singular against its family): the
      // pairs go straight to the refactor as one group, past the queue, so that a queue
      // flush never splits the group that group_fresh factorises once
      QEntry e;
      e.member = m;
      e.lane = lane;
      e.fail = (int32_t)fail;
      e.pguard = (int32_t)pguard;
      e.prod = prod;
      e.w = wi * wj;
      e.pad2 = 0.0;
      process_pairs<NCMAX>(a, W, true, e, j, Yw, wk, accq, rflops, n_rowdiff);
      n_parent += __popc(fail & pguard);
      n_child += __popc(fail & ~pguard);
    } else if (ball) {
      if (need) {
        const int pos = qn + __popc(ball & ((1u << lane) - 1u));
        QEntry e;
        e.member = m;
        e.lane = lane;
        e.fail = (int32_t)fail;
        e.pguard = (int32_t)pguard;
        e.prod = prod;
        e.w = wi * wj;
        e.pad2 = 0.0;
        queue[pos] = e;
        n_parent += __popc(fail & pguard);
        n_child += __popc(fail & ~pguard);
      }
      qn += __popc(ball);
      __syncwarp();
      if (qn >= 32) {
        process_queue<NCMAX>(a, W, queue, 32, (int64_t)tile * T + warp * 32, Yw, wk, accq, rflops, n_rowdiff);
        __syncwarp();
        if (lane < qn - 32) queue[lane] = queue[32 + lane];
        __syncwarp();
        qn -= 32;
      }
    }
  }
  if (qn > 0) process_queue<NCMAX>(a, W, queue, qn, (int64_t)tile * T + warp * 32, Yw, wk, accq, rflops, n_rowdiff);
  acc.x = fma(wj, acc.x, accq.x);
  acc.y = fma(wj, acc.y, accq.y);

  // ---- fixed-order reduction: lanes, then warps --------------------------------------
  acc = dev::warp_sum(acc);
  for (int o = 16; o > 0; o >>= 1) {
    n_parent += __shfl_xor_sync(0xffffffffu, n_parent, o);
    n_child += __shfl_xor_sync(0xffffffffu, n_child, o);
    n_rowdiff += __shfl_xor_sync(0xffffffffu, n_rowdiff, o);
    rflops += __shfl_xor_sync(0xffffffffu, rflops, o);
  }
  __syncthreads();
  double2* red = smem;  // reuse: the factor cache is no longer needed
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double2 s = red[0];
    for (int w = 1; w < (T >> 5); w++) {
      s.x += red[w].x;
      s.y += red[w].y;
    }
    *partial = s;
    if (!dev::finite2(s)) atomicOr(&a.counters[0], kStatusNonFinite);
  }
  if (lane == 0 && (n_parent | n_child | n_rowdiff)) {
    atomicAdd(&a.counters[1], n_parent);
    atomicAdd(&a.counters[2], n_child - n_rowdiff);  // queued for the lemma guard, less those the
    atomicAdd(&a.counters[3], rflops);               // row-difference update resolved
    atomicAdd(&a.counters[4], n_rowdiff);
  }
}

// Registers: the n <= 8 class keeps 168 (12 one-warp blocks per SM, or 3 blocks of its
// 128-thread tile); the larger classes may use all 255, measured fastest for n = 18 (8 blocks
// per SM against 9 at 216 and 10 at 200, whose spills cost more than the warps gain).
template <int NCMAX>
__global__ void __maxnreg__(NCMAX <= 8 ? 168 : 255) fwd_kernel(const FwdArgs a) {
  extern __shared__ double2 smem[];
  const int64_t item = a.item0 + blockIdx.x;
  const int64_t pos = item / a.n_tiles;
  const int W = a.fam_order ? a.fam_order[pos] : (int)pos;
  fwd_item<NCMAX>(a, W, (int)(item % a.n_tiles), smem, &a.partials[item]);
}

// Per-pair determinants through the same update path (one thread per pair).
template <int NCMAX>
__global__ void __launch_bounds__(64) pair_kernel(const FwdArgs a, int64_t n_pairs, int64_t n_src,
                                                  const int64_t* __restrict__ ii,
                                                  const int64_t* __restrict__ jj,
                                                  const int32_t* __restrict__ src_member,
                                                  const int32_t* __restrict__ mem_family,
                                                  double2* __restrict__ dets, int32_t* path) {
  extern __shared__ double2 smem[];
  const int T = blockDim.x;
  const int64_t p = (int64_t)blockIdx.x * T + threadIdx.x;
  if (p >= n_pairs) return;
  const int64_t i = ii[p], j = jj[p];
  if (i < 0 || i >= n_src || j < 0 || j >= a.n_snk) {
    atomicOr(&a.counters[0], kStatusBadIndex);
    return;
  }
  const int m = src_member[i];
  const int W = mem_family[m];
  double2* Y = smem + threadIdx.x;
  int32_t rows[NCMAX];
  int32_t bits = 0;
  for (int f = 0; f < a.F; f++) {
    const int n = a.n_f[f];
    double2 d = make_double2(1.0, 0.0);
    if (n > 0) {
      const int rho = a.fam_rank[(int64_t)W * a.F + f];
      const int32_t* col = a.snk_lab + j * a.Tn + a.off_f[f];
      int ey = 0;
      bool fail = dev::dispatch_shared<NCMAX>(n, rho, a.S[f], a.L_f[f],
                                              a.fam_arow + (int64_t)W * a.Tn + a.off_f[f], col,
                                              Y, T, &ey, a.kp);
      if (!fail) {
        const int32_t* mlab = a.mem_lab + ((int64_t)m * a.F + f) * MHC_MAX_RANK;
        d = dev::dispatch_member<NCMAX>(n, rho, a.S[f], a.L_f[f], mlab, col, Y, T, ey, a.kc, &fail);
        if (fail && rho <= 2 && n >= rho + 1 && a.rowdiff) {
          bool f2 = true;
          const int32_t* arow = a.fam_arow + (int64_t)W * a.Tn + a.off_f[f];
          double2 d2;
          if constexpr (NCMAX >= 10)  // two-row families need n_f >= 10
            d2 = rho == 1 ? dev::rowdiff_det(a.S[f], a.L_f[f], n, mlab[0], arow, col, Y, T, ey, a.kc, &f2)
                          : dev::rowdiff2_det(a.S[f], a.L_f[f], n, mlab, arow, col, Y, T, ey, a.kc, &f2);
          else
            d2 = dev::rowdiff_det(a.S[f], a.L_f[f], n, mlab[0], arow, col, Y, T, ey, a.kc, &f2);
          if (!f2) {
            d = d2;
            fail = false;
            bits |= 1 << (8 + f);
          }
        }
      }
      if (fail) {
        dev::member_rows(a, W, m, f, rho, rows);
        d = dev::dispatch_fresh<NCMAX>(n, a.S[f], a.L_f[f], rows, col);
        bits |= 1 << f;
      }
      if ((a.mem_par[m] >> f) & 1) d = dev::cneg(d);
    }
    dets[p * a.F + f] = d;
  }
  if (path) path[p] = bits;
}

// One two-sided block (family W, sink family Q, flavour f) of plan a: factorise B
// (rank-1 family) or the two-row family's shared rows (see kapply2), or nothing.
template <int NCMAX>
__device__ __forceinline__ void kfac_one(const FwdArgs& a, int64_t t, int64_t n_fam) {
  const int f = (int)(t % a.F);
  const int64_t wq = t / a.F;
  const int Q = (int)(wq % a.n_q);
  const int W = (int)(wq / a.n_q);
  const int n = a.n_f[f];
  if (n == 0 || n > 6 || !a.q_two[Q]) return;  // n > 6: kfac_group_kernel
  const int rho = a.fam_rank[(int64_t)W * a.F + f];
  const int sig = a.q_rank[(int64_t)Q * a.F + f];
  const dev::cd* S = a.S[f];
  const int L = a.L_f[f];
  const int32_t* arow = a.fam_arow + (int64_t)W * a.Tn + a.off_f[f];
  const int32_t* scol = a.snk_pos + (int64_t)a.q_off[Q] * a.Tn + a.off_f[f];
  dev::cd* K = const_cast<dev::cd*>(a.kbuf) + wq * a.kstride + a.koff[f];
  if ((rho == 2 && sig == 2) || rho >= 3) {  // one-sided update for these blocks
    a.kguard[t] = 1;
    return;
  }
  bool g;
  if (sig == 2) {
#define MHC_K12(N) \
  case N:          \
    g = dev::kfac_block12<N, N>(S, L, N, arow, scol, K, a.kp); \
    break;
    switch (n) {
      MHC_K12(2)
      MHC_K12(3)
      MHC_K12(4)
      MHC_K12(5)
      MHC_K12(6)
      default:
        return;
    }
#undef MHC_K12
    a.kguard[t] = g ? 1 : 0;
    return;
  }
#define MHC_KF(N)                                                                         \
  case N:                                                                                 \
    g = rho == 1 ? dev::kfac_block<N, N, 1>(S, L, N, arow, scol, K, a.kp)                 \
                 : dev::kfac_block<N, N, (N >= 2 ? 2 : 1)>(S, L, N, arow, scol, K, a.kp); \
    break;
  switch (n) {
    MHC_KF(1)
    MHC_KF(2)
    MHC_KF(3)
    MHC_KF(4)
    MHC_KF(5)
    MHC_KF(6)
    default:
      return;
  }
#undef MHC_KF
  a.kguard[t] = g ? 1 : 0;
}

// Thread u of a plan's block grid takes flavour u / (n_fam n_q) and block u mod (n_fam n_q):
// the flavour varies slowest, so a warp's threads share n_f (flavours of different sizes
// would otherwise alternate across the lanes and run both code paths).  Returns the index
// of the block in the [W][Q][f] layout of the factor buffer.
__device__ __forceinline__ int64_t kfac_index(const FwdArgs& a, int64_t u, int64_t n_fam) {
  const int64_t nwq = n_fam * a.n_q;
  return (u % nwq) * a.F + u / nwq;
}

// two-sided blocks of one plan: one thread per (W, Q, f)
template <int NCMAX>
__global__ void __launch_bounds__(128) kfac_kernel(const FwdArgs a, int64_t n_fam) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_fam * a.n_q * a.F) return;
  kfac_one<NCMAX>(a, kfac_index(a, u, n_fam), n_fam);
}

// two-sided blocks of every plan of a batch in one launch: kpref[k] is the first thread of
// correlator k (prefix sums of n_fam * n_q * F; kpref[count] = total)
template <int NCMAX>
__global__ void __launch_bounds__(128) kfac_batch_kernel(const FwdArgs* __restrict__ desc,
                                                         const int64_t* __restrict__ kpref,
                                                         const int64_t* __restrict__ nfam, int count) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kpref[count]) return;
  int lo = 0, hi = count - 1;
  while (lo < hi) {  // last k with kpref[k] <= t
    const int mid = (lo + hi + 1) >> 1;
    if (kpref[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const FwdArgs& a = desc[lo];
  if (!a.snk_orig) return;
  kfac_one<NCMAX>(a, kfac_index(a, t - kpref[lo], nfam[lo]), nfam[lo]);
}

// Two-sided blocks with n > 6: G lanes per block, the block in shared memory (see
// dev::group_lu).  One warp per thread block; GPW blocks per warp.
template <int NCMAX>
struct KGroup {
  static constexpr int G = NCMAX <= 8 ? 4 : (NCMAX <= 18 ? 8 : 16);  // lanes per block
  static constexpr int GPW = 32 / G;                           // blocks per warp
  // complex per block (matrix + back-substitution vector), padded to 4 mod 8 16-byte units
  // so that two groups sharing an 8-lane shared-memory phase use disjoint bank groups
  static constexpr int RAW = (NCMAX - 1) * (NCMAX - 1) + (NCMAX - 1);
  static constexpr int BS = RAW + ((4 - RAW % 8) + 8) % 8;
  static constexpr int PS = NCMAX;                             // ints per block
  static constexpr size_t smem() { return (size_t)GPW * (BS * sizeof(double2) + PS * sizeof(int)); }
};

template <int NCMAX>
__device__ __forceinline__ void kfac_group_one(const FwdArgs& a, int64_t t) {
  using KG = KGroup<NCMAX>;
  extern __shared__ double2 ksm[];
  const int lane = threadIdx.x & 31;
  const int j = lane / KG::G, g = lane % KG::G;
  const unsigned gm = KG::G == 32 ? 0xffffffffu : (((1u << KG::G) - 1u) << (j * KG::G));
  dev::cd* Bs = ksm + (size_t)j * KG::BS;
  dev::cd* Ws = Bs + (NCMAX - 1) * (NCMAX - 1);
  int* Ps = reinterpret_cast<int*>(ksm + (size_t)KG::GPW * KG::BS) + j * KG::PS;
  const int f = (int)(t % a.F);
  const int64_t wq = t / a.F;
  const int Q = (int)(wq % a.n_q);
  const int W = (int)(wq / a.n_q);
  const int n = a.n_f[f];
  if (n <= 6 || !a.q_two[Q]) return;
  const int rho = a.fam_rank[(int64_t)W * a.F + f];
  const int sig = a.q_rank[(int64_t)Q * a.F + f];
  const dev::cd* S = a.S[f];
  const int L = a.L_f[f];
  const int32_t* arow = a.fam_arow + (int64_t)W * a.Tn + a.off_f[f];
  const int32_t* scol = a.snk_pos + (int64_t)a.q_off[Q] * a.Tn + a.off_f[f];
  dev::cd* K = const_cast<dev::cd*>(a.kbuf) + wq * a.kstride + a.koff[f];
  bool gd;
  if (rho >= 3)  // one-sided update for these blocks
    gd = true;
  else if (rho == 2 && sig == 2)  // the (n-2) x (n-2) shared block, kapply's layout (kapply22)
    gd = dev::group_kfac_block<KG::G>(S, L, n - 1, 1, arow, scol, K, a.kp, g, gm, Bs, Ws, Ps);
  else if (sig == 2)
    gd = dev::group_kfac_block12<KG::G>(S, L, n, arow, scol, K, a.kp, g, gm, Bs, Ps);
  else
    gd = dev::group_kfac_block<KG::G>(S, L, n, rho, arow, scol, K, a.kp, g, gm, Bs, Ws, Ps);
  if (g == 0) a.kguard[t] = gd ? 1 : 0;
}

template <int NCMAX>
__global__ void __launch_bounds__(32) kfac_group_kernel(const FwdArgs a, int64_t n_fam) {
  const int64_t u = (int64_t)blockIdx.x * KGroup<NCMAX>::GPW + (threadIdx.x / KGroup<NCMAX>::G);
  if (u >= n_fam * a.n_q * a.F) return;
  kfac_group_one<NCMAX>(a, kfac_index(a, u, n_fam));
}

template <int NCMAX>
__global__ void __launch_bounds__(32) kfac_group_batch_kernel(const FwdArgs* __restrict__ desc,
                                                              const int64_t* __restrict__ kpref,
                                                              const int64_t* __restrict__ nfam, int count) {
  const int64_t t = (int64_t)blockIdx.x * KGroup<NCMAX>::GPW + (threadIdx.x / KGroup<NCMAX>::G);
  if (t >= kpref[count]) return;
  int lo = 0, hi = count - 1;
  while (lo < hi) {  // last k with kpref[k] <= t
    const int mid = (lo + hi + 1) >> 1;
    if (kpref[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const FwdArgs& a = desc[lo];
  if (!a.snk_orig) return;
  kfac_group_one<NCMAX>(a, kfac_index(a, t - kpref[lo], nfam[lo]));
}

}  // namespace fwd

// Block factors of every plan of a batch: blocks with n <= 6 one per thread, blocks with
// n > 6 (present when big != 0) by lane groups.
template <int NCMAX>
cudaError_t launch_kfac_batch_nc(const FwdArgs* desc, const int64_t* kpref, const int64_t* nfam,
                                 int count, int64_t total, int big, cudaStream_t s) {
  if (total == 0) return cudaSuccess;
  fwd::kfac_batch_kernel<NCMAX><<<(unsigned)((total + 127) / 128), 128, 0, s>>>(desc, kpref, nfam, count);
  if (big) {
    using KG = fwd::KGroup<NCMAX>;
    fwd::kfac_group_batch_kernel<NCMAX><<<(unsigned)((total + KG::GPW - 1) / KG::GPW), 32, KG::smem(), s>>>(
        desc, kpref, nfam, count);
  }
  return cudaGetLastError();
}

template <int NCMAX>
cudaError_t launch_kfac_nc(const FwdArgs& a, int64_t n_fam, cudaStream_t s) {
  const int64_t threads = n_fam * a.n_q * a.F;
  if (threads == 0) return cudaSuccess;
  fwd::kfac_kernel<NCMAX><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(a, n_fam);
  bool big = false;
  for (int f = 0; f < a.F; f++) big |= a.n_f[f] > 6;
  if (big) {
    using KG = fwd::KGroup<NCMAX>;
    fwd::kfac_group_kernel<NCMAX><<<(unsigned)((threads + KG::GPW - 1) / KG::GPW), 32, KG::smem(), s>>>(a, n_fam);
  }
  return cudaGetLastError();
}

// Persistent batched launch: blocks pull (correlator, family, tile) items from a list
// ordered by decreasing cost through one atomic counter; each item's partial goes to its
// own slot (see batch.cu).  Registers as fwd_kernel's (at most 128 threads per block).
template <int NCMAX>
__global__ void __maxnreg__(NCMAX <= 8 ? 168 : 255) batch_kernel(const FwdArgs* __restrict__ desc,
                                                    const BatchItem* __restrict__ items,
                                                    int64_t n_items, unsigned long long* head,
                                                    const int64_t* __restrict__ part_off,
                                                    double2* __restrict__ partials) {
  extern __shared__ double2 smem[];
  __shared__ int64_t s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(head, 1ull);
    __syncthreads();
    const int64_t it = s_item;
    if (it >= n_items) break;
    const BatchItem bi = items[it];
    const FwdArgs& a = desc[bi.corr];
    fwd::fwd_item<NCMAX>(a, bi.W, bi.tile, smem,
                    &partials[part_off[bi.corr] + (int64_t)bi.W * a.n_tiles + bi.tile]);
    __syncthreads();
  }
}

template <int NCMAX>
cudaError_t launch_batch_nc(int grid, int T, size_t smem, cudaStream_t s, const FwdArgs* desc,
                            const BatchItem* items, int64_t n_items, unsigned long long* head,
                            const int64_t* part_off, double2* partials) {
  // the shared-memory limit was raised by batch_occupancy_nc, outside any stream capture
  batch_kernel<NCMAX><<<grid, T, smem, s>>>(desc, items, n_items, head, part_off, partials);
  return cudaGetLastError();
}

template <int NCMAX>
int batch_occupancy_nc(int T, size_t smem) {
  int nb = 0, dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, batch_kernel<NCMAX>) == cudaSuccess) optin -= (int)fa.sharedSizeBytes;
  cudaFuncSetAttribute(batch_kernel<NCMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<NCMAX>, T, smem) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

template <int NCMAX>
cudaError_t launch_fwd_nc(const FwdArgs& a, int tile, int64_t items, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(fwd::fwd_kernel<NCMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fwd::fwd_kernel<NCMAX><<<(unsigned)items, tile, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NCMAX>
cudaError_t launch_pairs_nc(const FwdArgs& a, int64_t n_pairs, int64_t n_src, const int64_t* ii,
                            const int64_t* jj, const int32_t* src_member, const int32_t* mem_family,
                            double* dets, int32_t* path, cudaStream_t s) {
  const int T = 64;
  const size_t smem = (size_t)a.slots * T * sizeof(double2);
  if (n_pairs == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fwd::pair_kernel<NCMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((n_pairs + T - 1) / T);
  fwd::pair_kernel<NCMAX><<<grid, T, smem, s>>>(a, n_pairs, n_src, ii, jj, src_member, mem_family,
                                                reinterpret_cast<double2*>(dets), path);
  return cudaGetLastError();
}

}  // namespace mhc
