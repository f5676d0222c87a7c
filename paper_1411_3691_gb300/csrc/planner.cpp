// planner.cpp -- host planner: validation, source-term graph, greedy dominating set,
// member alignment and work families (Sec. 3 of the paper: execution order).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "plan.h"
#include "trace.h"

namespace mhc {

namespace {

thread_local std::string g_last_error;

// Largest bucket of the candidate-pair hash scan that is compared exhaustively; pairs of
// a longer bucket are compared only within a sliding window of this many terms.
constexpr size_t kBucketWindow = 2048;
// Rank-2 adjacency is used for a flavour only when n_f is at least this large: below it
// a rank-2 update (4 dot products per member over n - 2 shared rows) saves too little over
// splitting the family.
constexpr int kRank2MinN = 10;
// rank k (k changed rows per flavour) only for n_f >= 4k + 2: rank 2 from 10, rank 3 from 14
int rank_min_n(int k) { return 4 * k + 2; }
// Largest number of leave-d-out keys per build of the candidate list: above it the keys
// leave out at most two labels (pairs that differ in more labels in the key flavour are
// then not adjacent in the graph).
constexpr double kMaxKeys = 5e7;

uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ULL;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebULL;
  x ^= x >> 31;
  return x;
}

// number of labels two sorted multisets share
int common_sorted(const int32_t* a, const int32_t* b, int n) {
  int i = 0, j = 0, c = 0;
  while (i < n && j < n) {
    if (a[i] == b[j]) {
      c++;
      i++;
      j++;
    } else if (a[i] < b[j]) {
      i++;
    } else {
      j++;
    }
  }
  return c;
}

int perm_parity(const std::vector<int>& p) {
  int inv = 0;
  for (size_t a = 0; a < p.size(); a++)
    for (size_t b = a + 1; b < p.size(); b++)
      if (p[a] > p[b]) inv++;
  return inv & 1;
}

// Alignment of one member tuple t to the reference tuple ref (both n labels, given order).
struct Align {
  std::vector<int> changed;  // reference positions not matched (ascending)
  std::vector<int> aligned;  // member labels placed at the reference positions
  int parity = 0;            // parity of the row permutation: det(t) = (-1)^parity det(aligned)
};

Align align(const int32_t* ref, const int32_t* t, int n) {
  Align a;
  std::vector<int> match(n, -1);  // ref position -> member position
  std::vector<char> used(n, 0);
  for (int m = 0; m < n; m++)
    for (int p = 0; p < n; p++)
      if (!used[p] && t[p] == ref[m]) {
        match[m] = p;
        used[p] = 1;
        break;
      }
  std::vector<int> extras;  // member positions not matched (ascending)
  for (int p = 0; p < n; p++)
    if (!used[p]) extras.push_back(p);
  a.aligned.assign(ref, ref + n);
  std::vector<int> pi(n, -1);  // member position -> aligned position
  int k = 0;
  for (int m = 0; m < n; m++) {
    if (match[m] >= 0) {
      pi[match[m]] = m;
    } else {
      a.changed.push_back(m);
      a.aligned[m] = t[extras[k]];
      pi[extras[k]] = m;
      k++;
    }
  }
  a.parity = perm_parity(pi);
  return a;
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

double flops_shared_rows(int n, int rho) {
  const double M = n - rho;
  if (n <= 0) return 0.0;
  double f = 0.0;
  f += M * (M + 1) / 2;                        // pivot measures |re|+|im|
  f += 6.0 * M;                                // pivot reciprocals
  f += 6.0 * M * (M - 1) / 2;                  // multipliers
  double upd = 0.0;
  for (int k = 0; k < (int)M; k++) upd += (M - 1 - k) * (n - 1 - k);
  f += 8.0 * upd;                              // trailing updates
  if (M >= 1) f += 6.0 * (M - 1);              // det of the shared-row factor
  f += rho * (8.0 * M * (M - 1) / 2 + 6.0 * M);  // back substitutions
  f += rho * 6.0 * M;                          // scaling by the determinant
  return f;
}

double flops_member(int n, int rho) {
  if (n <= 0) return 0.0;
  const double dot = 6.0 + 8.0 * (n - 1);
  if (rho >= 4) return rho * rho * dot + flops_fresh_lu(rho) + 6.0;  // k x k LU det, times sd
  if (rho == 3) return 9.0 * dot + 3.0 * 14.0 + 22.0 + 6.0;  // 3x3 det by cofactors, times sd
  return rho == 2 ? 4.0 * dot + 2.0 * 6.0 + 2.0 : dot;
}

// two-sided update, per sink: P a, forward and backward triangular solves with the stored
// LU factors of B (M = n - 1), scaling by -det B
double flops_kapply(int n) {
  if (n <= 1) return 0.0;
  const double M = n - 1;
  return 8.0 * M * (M - 1) + 6.0 * M + 6.0 * M;
}

// LU factors of one M x M block B with partial pivoting (two-sided update, per block)
double flops_adjugate(int m) {
  if (m <= 0) return 0.0;
  double f = m * (m + 1) / 2.0;  // pivot measures
  f += 6.0 * m;                  // reciprocals (kept for the solves)
  f += 6.0 * m * (m - 1) / 2.0;  // multipliers
  for (int k = 0; k < m; k++) f += 8.0 * (m - 1 - k) * (m - 1 - k);  // updates
  f += 6.0 * (m - 1);            // det(B)
  return f;
}

// two-row family, per sink: z2 = -U1^{-1} L^{-1} P a (M = n - 2)
double flops_kapply2(int n) {
  if (n < 3) return 0.0;
  const double M = n - 2;
  return 8.0 * M * (M - 1) + 6.0 * M;
}

// two-row family x two-column sink family, per sink: two forward and two backward solves
// with the stored factors of the (n-2) x (n-2) shared block (M = n - 2)
double flops_kapply22(int n) {
  if (n < 3) return 0.0;
  const double M = n - 2;
  return 2.0 * (8.0 * M * (M - 1) + 6.0 * M);
}

// two-row family, per block: LU of the M shared rows over M + 1 shared columns, -U1^{-1} u
double flops_rank2_block(int n) {
  if (n < 2) return 0.0;
  const int m = n - 2;
  double f = m * (m + 1) / 2.0 + 6.0 * m + 6.0 * m * (m - 1) / 2.0;
  for (int k = 0; k < m; k++) f += 8.0 * (m - 1 - k) * (m - k);
  f += 6.0 * std::max(m - 1, 0);
  f += 8.0 * m * (m - 1) / 2.0 + 6.0 * m;
  return f;
}

// one-row family x two-column sink family, per block: LU of the n-1 shared rows over the
// n-2 shared columns
double flops_block12(int n) {
  if (n < 2) return 0.0;
  const int m = n - 2, r = n - 1;  // columns, rows
  double f = 0.0;
  for (int k = 0; k < m; k++) {
    f += (r - k);                     // pivot measures
    f += 6.0;                         // reciprocal
    f += 6.0 * (r - 1 - k);           // multipliers
    f += 8.0 * (r - 1 - k) * (m - 1 - k);  // updates
  }
  f += 6.0 * std::max(m - 1, 0);      // det(U1)
  return f;
}

// one-row family x two-column sink family, per sink: two forward solves over the n-1 rows,
// the 2 x 2 combination, one backward solve and the scaling (see kapply12)
double flops_kapply12(int n) {
  if (n < 2) return 0.0;
  const double m = n - 2;
  return 2.0 * 8.0 * (m * (m - 1) / 2.0 + m) + m * (6.0 + 8.0) + 8.0 * m * (m - 1) / 2.0 + 6.0 * m +
         6.0 * m + 12.0;
}

double flops_fresh_lu(int n) {
  if (n <= 0) return 0.0;
  double f = n * (n + 1) / 2.0;                  // pivot measures
  f += 6.0 * (n - 1);                            // reciprocals
  f += 6.0 * n * (n - 1) / 2.0;                  // multipliers
  f += 8.0 * (n - 1) * n * (2.0 * n - 1) / 6.0;  // trailing updates
  f += 6.0 * (n - 1);                            // product of the pivots
  return f;
}

// Greedy dominating set of a term graph (Sec. 3): two terms are adjacent when, in every
// flavour f, their label multisets differ in at most dmax[f] labels.  Candidate pairs come
// from shared leave-d-out keys of one flavour, then every flavour is checked exactly.
// Returns the dominated sets (dominator first, then its neighbours ascending).
std::vector<std::vector<int32_t>> dominated_sets(const std::vector<int32_t>& labels, int64_t N,
                                                 int F, const std::vector<int32_t>& n_f,
                                                 const std::vector<int32_t>& off_f, int Tn,
                                                 const std::vector<int>& dmax, int64_t* n_edges) {
  // ---- per term, per flavour sorted label multisets -------------------------------
  std::vector<int32_t> sorted(labels);
  for (int64_t i = 0; i < N; i++)
    for (int f = 0; f < F; f++)
      std::sort(sorted.begin() + i * Tn + off_f[f], sorted.begin() + i * Tn + off_f[f] + n_f[f]);

  // key flavour: the smallest allowed difference, then the largest n
  int f0 = -1;
  for (int f = 0; f < F; f++) {
    if (n_f[f] == 0) continue;
    if (f0 < 0 || dmax[f] < dmax[f0] || (dmax[f] == dmax[f0] && n_f[f] > n_f[f0])) f0 = f;
  }

  // ---- candidate pairs: shared leave-d-out keys of the key flavour ------------------
  std::vector<std::pair<uint64_t, int32_t>> keys;
  if (f0 >= 0) {
    const int n = n_f[f0];
    int d = std::min(dmax[f0], n);
    auto choose = [](int a, int b) {
      double c = 1.0;
      for (int t = 0; t < b; t++) c = c * (a - t) / (t + 1);
      return c;
    };
    while (d > 2 && (double)N * choose(n, d) > kMaxKeys) d--;
    keys.reserve((size_t)((double)N * (d == 1 ? n : choose(n, d))));
    std::vector<int> skip(d);
    for (int64_t i = 0; i < N; i++) {
      const int32_t* s = &sorted[i * Tn + off_f[f0]];
      // one key per d-subset of positions left out: the hash of the remaining labels
      auto emit = [&]() {
        uint64_t h = 0x9e3779b97f4a7c15ULL;
        int t = 0;
        for (int m = 0; m < n; m++) {
          if (t < d && skip[t] == m) {
            t++;
            continue;
          }
          h = mix64(h ^ (uint64_t)(uint32_t)s[m]);
        }
        keys.emplace_back(h, (int32_t)i);
      };
      if (d == 1) {
        for (int m = 0; m < n; m++)
          if (m == 0 || s[m] != s[m - 1]) {
            skip[0] = m;
            emit();
          }
      } else {
        for (int t = 0; t < d; t++) skip[t] = t;
        for (;;) {  // every d-subset of [0, n) in lexicographic order
          emit();
          int t = d - 1;
          while (t >= 0 && skip[t] == n - d + t) t--;
          if (t < 0) break;
          skip[t]++;
          for (int u = t + 1; u < d; u++) skip[u] = skip[u - 1] + 1;
        }
      }
    }
  } else {
    for (int64_t i = 0; i < N; i++) keys.emplace_back(0, (int32_t)i);
  }
  std::sort(keys.begin(), keys.end());
  std::vector<std::pair<int32_t, int32_t>> cand;
  for (size_t a = 0; a < keys.size();) {
    size_t b = a;
    while (b < keys.size() && keys[b].first == keys[a].first) b++;
    for (size_t x = a; x < b; x++)
      for (size_t y = x + 1; y < b && y - x < kBucketWindow; y++)
        if (keys[x].second != keys[y].second) cand.emplace_back(keys[x].second, keys[y].second);
    a = b;
  }
  keys.clear();
  keys.shrink_to_fit();
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());

  // ---- exact adjacency check: every flavour differs in at most dmax[f] labels ---------
  std::vector<std::vector<int32_t>> adj(N);
  int64_t edges = 0;
  for (auto& e : cand) {
    const int64_t i = e.first, j = e.second;
    bool ok = true;
    for (int f = 0; f < F && ok; f++) {
      const int n = n_f[f];
      if (n == 0) continue;
      const int c = common_sorted(&sorted[i * Tn + off_f[f]], &sorted[j * Tn + off_f[f]], n);
      ok = (n - c) <= dmax[f];
    }
    if (ok) {
      adj[i].push_back((int32_t)j);
      adj[j].push_back((int32_t)i);
      edges++;
    }
  }
  cand.clear();
  cand.shrink_to_fit();
  for (auto& a : adj) std::sort(a.begin(), a.end());

  // ---- greedy dominating set (Sec. 3): highest remaining degree, ties to lowest index -
  std::vector<int32_t> deg(N);
  std::vector<char> alive(N, 1);
  std::set<std::pair<int32_t, int32_t>> pq;  // (-degree, index)
  for (int64_t i = 0; i < N; i++) {
    deg[i] = (int32_t)adj[i].size();
    pq.emplace(-deg[i], (int32_t)i);
  }
  std::vector<std::vector<int32_t>> dom_sets;  // dominator first, then its neighbours
  while (!pq.empty()) {
    const int32_t v = pq.begin()->second;
    std::vector<int32_t> fam{v};
    for (int32_t u : adj[v])
      if (alive[u]) fam.push_back(u);
    for (int32_t x : fam) {
      pq.erase({-deg[x], x});
      alive[x] = 0;
    }
    for (int32_t x : fam)
      for (int32_t w : adj[x])
        if (alive[w]) {
          pq.erase({-deg[w], w});
          deg[w]--;
          pq.emplace(-deg[w], w);
        }
    std::sort(fam.begin() + 1, fam.end());
    dom_sets.push_back(std::move(fam));
  }
  adj.clear();

  *n_edges = edges;
  return dom_sets;
}

mhc_status build_plan(Plan& p) {
  auto t0 = std::chrono::steady_clock::now();
  const int F = p.F;
  const int64_t N = p.n_src;
  const int Tn = p.Tn;
  const int rank2 = p.opts.rank2 ? 1 : 0;
  const int kmax = p.opts.max_family;

  // changed labels allowed per flavour: sources up to the largest rank the options allow
  // for n_f (opts.max_rank, or 3 with opts.rank3, else 2), sinks up to 2
  const int rmax = !rank2 ? 1 : (p.opts.max_rank > 0 ? p.opts.max_rank : (p.opts.rank3 ? 3 : 2));
  std::vector<int> dmax(F), dmax_snk(F);
  for (int f = 0; f < F; f++) {
    dmax[f] = 1;
    for (int k = 2; k <= rmax; k++)
      if (p.n_f[f] >= rank_min_n(k)) dmax[f] = k;
    dmax_snk[f] = std::min(dmax[f], 2);
  }
  int64_t edges = 0;
  std::vector<std::vector<int32_t>> dom_sets =
      dominated_sets(p.labels_src, N, F, p.n_f, p.off_f, Tn, dmax, &edges);

  // ---- sink families for the two-sided update (Sec. 2: a sink term that differs in one
  // label changes one column; the same greedy dominating set on the sink side, with two
  // changed columns allowed where two changed rows are) ---------------------------------
  {
    int64_t sedges = 0;
    std::vector<std::vector<int32_t>> sink_sets =
        p.opts.one_sided ? std::vector<std::vector<int32_t>>()
                         : dominated_sets(p.labels_snk, p.n_snk, F, p.n_f, p.off_f, Tn, dmax_snk, &sedges);
    if (p.opts.one_sided)
      for (int64_t j = 0; j < p.n_snk; j++) sink_sets.push_back({(int32_t)j});
    struct SGroup {
      std::vector<std::vector<int>> R;  // per flavour: changed columns (ascending)
      std::vector<int32_t> members;
      int32_t ref;
    };
    std::vector<SGroup> groups;
    for (auto& ds : sink_sets) {
      const int32_t v = ds[0];
      const int32_t* ref = &p.labels_snk[(int64_t)v * Tn];
      std::vector<SGroup> local;
      for (int32_t t : ds) {
        std::vector<std::vector<int>> ch(F);
        for (int f = 0; f < F; f++)
          ch[f] = align(ref + p.off_f[f], &p.labels_snk[(int64_t)t * Tn + p.off_f[f]], p.n_f[f]).changed;
        bool placed = false;
        for (auto& g : local) {
          if ((int)g.members.size() >= 32) continue;
          bool ok = true;
          std::vector<std::vector<int>> U(F);
          for (int f = 0; f < F && ok; f++) {
            std::set<int> u(g.R[f].begin(), g.R[f].end());
            u.insert(ch[f].begin(), ch[f].end());
            U[f].assign(u.begin(), u.end());
            ok = (int)U[f].size() <= dmax_snk[f];
          }
          if (!ok) continue;
          g.R = U;
          g.members.push_back(t);
          placed = true;
          break;
        }
        if (!placed) local.push_back(SGroup{ch, {t}, v});
      }
      for (auto& g : local) groups.push_back(std::move(g));
    }
    // families with at least two sinks use the two-sided update and come first
    std::stable_partition(groups.begin(), groups.end(), [](const SGroup& g) { return g.members.size() >= 2; });
    p.snk_order.clear();
    p.snk_lab2.clear();
    p.snk_par2.clear();
    p.snk_q.clear();
    p.q_off.assign(1, 0);
    p.q_two.clear();
    p.q_rank.clear();
    for (auto& g : groups) {
      const int32_t Q = (int32_t)p.q_two.size();
      const int32_t* ref = &p.labels_snk[(int64_t)g.ref * Tn];
      std::vector<std::vector<int>> R(F);
      for (int f = 0; f < F; f++) {
        R[f] = g.R[f];
        if (R[f].empty() && p.n_f[f] > 0) R[f].push_back(p.n_f[f] - 1);
        p.q_rank.push_back((int32_t)R[f].size());
      }
      for (int32_t t : g.members) {
        int bits = 0;
        std::vector<int32_t> lab(Tn);
        for (int f = 0; f < F; f++) {
          const int n = p.n_f[f];
          if (n == 0) continue;
          Align al = align(ref + p.off_f[f], &p.labels_snk[(int64_t)t * Tn + p.off_f[f]], n);
          // columns: the shared ones (ascending positions), then the changed ones
          std::vector<int> order;
          for (int m = 0; m < n; m++)
            if (std::find(R[f].begin(), R[f].end(), m) == R[f].end()) order.push_back(m);
          for (int r : R[f]) order.push_back(r);
          for (int m = 0; m < n; m++) lab[p.off_f[f] + m] = al.aligned[order[m]];
          bits |= (al.parity ^ perm_parity(order)) << f;
        }
        p.snk_order.push_back(t);
        p.snk_lab2.insert(p.snk_lab2.end(), lab.begin(), lab.end());
        p.snk_par2.push_back(bits);
        p.snk_q.push_back(Q);
      }
      p.q_off.push_back((int32_t)p.snk_order.size());
      p.q_two.push_back(g.members.size() >= 2 ? 1 : 0);
    }
    p.n_qfam = (int64_t)p.q_two.size();
  }

  // ---- sink-side cost of one source family, per flavour and rank (the flop model below):
  // every two-sided sink family contributes its block factors once and its solves per
  // sink, every other sink a shared-row factorisation -----------------------------------
  std::vector<int64_t> gq1(F, 0), gs1(F, 0), gq2(F, 0), gs2(F, 0);
  int64_t g_one = 0;
  for (int64_t Q = 0; Q < p.n_qfam; Q++) {
    const int64_t sz = p.q_off[Q + 1] - p.q_off[Q];
    if (!p.q_two[Q]) {
      g_one += sz;
      continue;
    }
    for (int f = 0; f < F; f++) {
      if (p.q_rank[Q * F + f] == 2) {
        gq2[f]++;
        gs2[f] += sz;
      } else {
        gq1[f]++;
        gs1[f] += sz;
      }
    }
  }
  auto fam_cost = [&](int f, int rho, int64_t k) {
    const int n = p.n_f[f];
    if (n == 0) return 0.0;
    double c = (double)p.n_snk * (double)k * flops_member(n, rho) + (double)g_one * flops_shared_rows(n, rho);
    if (rho == 1) {
      c += (double)gq1[f] * flops_adjugate(n - 1) + (double)gs1[f] * flops_kapply(n);
      c += (double)gq2[f] * flops_block12(n) + (double)gs2[f] * flops_kapply12(n);
    } else if (rho == 2) {
      c += (double)gq1[f] * flops_rank2_block(n) + (double)gs1[f] * flops_kapply2(n);
      c += (double)gq2[f] * flops_adjugate(n - 2) + (double)gs2[f] * flops_kapply22(n);
    } else {
      c += (double)(gs1[f] + gs2[f]) * flops_shared_rows(n, rho);
    }
    return c;
  };

  // ---- work families: align members, group by compatible changed rows ---------------
  p.fam_off.assign(1, 0);
  p.fam_rank.clear();
  p.fam_rows.clear();
  p.fam_ref.clear();
  p.fam_arow.clear();
  p.mem_term.clear();
  p.mem_sign.clear();
  p.mem_par.clear();
  p.mem_lab.clear();
  p.src_member.assign(N, -1);
  p.mem_family.clear();
  int64_t rank2_blocks = 0, rank3_blocks = 0, rank4p_blocks = 0;
  p.max_members = 0;

  struct Member {
    int32_t term;
    std::vector<Align> al;  // per flavour
  };
  struct Group {
    std::vector<std::vector<int>> R;  // per flavour, ascending changed rows
    std::vector<int> members;         // indices into the member list
  };
  for (auto& ds : dom_sets) {
    const int32_t v = ds[0];
    const int32_t* ref = &p.labels_src[(int64_t)v * Tn];
    std::vector<Member> mems;
    for (int32_t t : ds) {
      Member m;
      m.term = t;
      for (int f = 0; f < F; f++)
        m.al.push_back(align(ref + p.off_f[f], &p.labels_src[(int64_t)t * Tn + p.off_f[f]], p.n_f[f]));
      mems.push_back(std::move(m));
    }
    std::vector<Group> groups;
    if (p.opts.first_fit) {
      // members in order, each into the first group that stays within dmax changed rows
      for (int mi = 0; mi < (int)mems.size(); mi++) {
        bool placed = false;
        for (auto& g : groups) {
          if ((int)g.members.size() >= kmax) continue;
          bool ok = true;
          std::vector<std::vector<int>> U(F);
          for (int f = 0; f < F && ok; f++) {
            std::set<int> u(g.R[f].begin(), g.R[f].end());
            u.insert(mems[mi].al[f].changed.begin(), mems[mi].al[f].changed.end());
            U[f].assign(u.begin(), u.end());
            ok = (int)U[f].size() <= dmax[f];
          }
          if (ok) {
            g.R = U;
            g.members.push_back(mi);
            placed = true;
            break;
          }
        }
        if (!placed) {
          Group g;
          g.R.resize(F);
          for (int f = 0; f < F; f++) g.R[f] = mems[mi].al[f].changed;
          g.members.push_back(mi);
          groups.push_back(std::move(g));
        }
      }
    } else {
      // cost-driven: start from the groups of members with the same changed rows (at most
      // kmax each), then merge the pair of groups whose merge lowers the plan's flop count
      // most (a merged family shares one factorisation per sink but may need a higher rank
      // for all its members), until no merge lowers it
      std::map<std::vector<std::vector<int>>, std::vector<int>> bysig;
      for (int mi = 0; mi < (int)mems.size(); mi++) {
        std::vector<std::vector<int>> sig(F);
        for (int f = 0; f < F; f++) sig[f] = mems[mi].al[f].changed;
        bysig[sig].push_back(mi);
      }
      for (auto& kv : bysig)
        for (size_t a = 0; a < kv.second.size(); a += (size_t)kmax) {
          Group g;
          g.R = kv.first;
          g.members.assign(kv.second.begin() + a, kv.second.begin() + std::min(kv.second.size(), a + (size_t)kmax));
          groups.push_back(std::move(g));
        }
      auto gcost = [&](const std::vector<std::vector<int>>& R, int64_t k) {
        double c = 0.0;
        for (int f = 0; f < F; f++) c += fam_cost(f, std::max<int>(1, (int)R[f].size()), k);
        return c;
      };
      for (;;) {
        double best = 0.0;
        int ba = -1, bb = -1;
        std::vector<std::vector<int>> bestU;
        for (int x = 0; x < (int)groups.size(); x++)
          for (int y = x + 1; y < (int)groups.size(); y++) {
            const int64_t k = (int64_t)(groups[x].members.size() + groups[y].members.size());
            if (k > kmax) continue;
            std::vector<std::vector<int>> U(F);
            bool ok = true;
            for (int f = 0; f < F && ok; f++) {
              std::set<int> u(groups[x].R[f].begin(), groups[x].R[f].end());
              u.insert(groups[y].R[f].begin(), groups[y].R[f].end());
              U[f].assign(u.begin(), u.end());
              ok = (int)U[f].size() <= dmax[f];
            }
            if (!ok) continue;
            const double gain = gcost(groups[x].R, (int64_t)groups[x].members.size()) +
                                gcost(groups[y].R, (int64_t)groups[y].members.size()) - gcost(U, k);
            if (gain > best) {
              best = gain;
              ba = x;
              bb = y;
              bestU = U;
            }
          }
        if (ba < 0) break;
        groups[ba].R = bestU;
        groups[ba].members.insert(groups[ba].members.end(), groups[bb].members.begin(), groups[bb].members.end());
        std::sort(groups[ba].members.begin(), groups[ba].members.end());
        groups.erase(groups.begin() + bb);
      }
      // the dominator's group first, then by first member: a deterministic order
      std::sort(groups.begin(), groups.end(),
                [](const Group& x, const Group& y) { return x.members[0] < y.members[0]; });
    }
    for (auto& g : groups) {
      const int64_t W = p.n_fam++;
      std::vector<int32_t> ranks(F), rows(MHC_MAX_RANK * F, -1), arow(Tn, -1);
      std::vector<int> eps(F, 0);
      for (int f = 0; f < F; f++) {
        const int n = p.n_f[f];
        std::vector<int> R = g.R[f];
        if (n == 0) {
          ranks[f] = 0;
          continue;
        }
        if (R.empty()) R.push_back(n - 1);
        ranks[f] = (int32_t)R.size();
        if (R.size() == 2) rank2_blocks++;
        if (R.size() == 3) rank3_blocks++;
        if (R.size() >= 4) rank4p_blocks++;
        for (size_t k = 0; k < R.size(); k++) rows[MHC_MAX_RANK * f + k] = R[k];
        // [shared rows ascending; changed rows ascending] and the sign of that reordering
        std::vector<int> order;
        int a = 0;
        for (int m = 0; m < n; m++)
          if (std::find(R.begin(), R.end(), m) == R.end()) {
            order.push_back(m);
            arow[p.off_f[f] + a++] = ref[p.off_f[f] + m];
          }
        for (int r : R) order.push_back(r);
        eps[f] = perm_parity(order);
        g.R[f] = R;
      }
      for (int f = 0; f < F; f++) p.fam_rank.push_back(ranks[f]);
      p.fam_rows.insert(p.fam_rows.end(), rows.begin(), rows.end());
      p.fam_ref.insert(p.fam_ref.end(), ref, ref + Tn);
      p.fam_arow.insert(p.fam_arow.end(), arow.begin(), arow.end());
      for (int mi : g.members) {
        const Member& m = mems[mi];
        int parity = 0, bits = 0;
        std::vector<int32_t> lab(MHC_MAX_RANK * F, -1);
        for (int f = 0; f < F; f++) {
          if (p.n_f[f] == 0) continue;
          const int pf = m.al[f].parity ^ eps[f];
          parity ^= pf;
          bits |= pf << f;
          for (int k = 0; k < ranks[f]; k++) lab[MHC_MAX_RANK * f + k] = m.al[f].aligned[g.R[f][k]];
        }
        p.mem_lab.insert(p.mem_lab.end(), lab.begin(), lab.end());
        p.src_member[m.term] = (int32_t)p.mem_term.size();
        p.mem_term.push_back(m.term);
        p.mem_sign.push_back(parity ? -1 : 1);
        p.mem_par.push_back(bits);
        p.mem_family.push_back((int32_t)W);
      }
      p.fam_off.push_back((int64_t)p.mem_term.size());
      p.max_members = std::max(p.max_members, (int)g.members.size());
    }
  }

  // ---- statistics -------------------------------------------------------------------
  mhc_stats& s = p.stats;
  std::memset(&s, 0, sizeof(s));
  s.n_src = p.n_src;
  s.n_snk = p.n_snk;
  s.n_flavours = F;
  s.max_n = p.max_n;
  s.dominators = (int64_t)dom_sets.size();
  s.families = p.n_fam;
  s.rank2_family_flavours = rank2_blocks;
  s.rank3_family_flavours = rank3_blocks;
  s.rank4plus_family_flavours = rank4p_blocks;
  s.members = (int64_t)p.mem_term.size();
  s.graph_edges = edges;
  s.sink_families = p.n_qfam;
  double fl = 0.0;
  // per flavour: two-sided sink families by column rank (count, sinks), one-sided sinks
  std::vector<int64_t> qc1(F, 0), qs1(F, 0), qc2(F, 0), qs2(F, 0);
  int64_t one_sinks = 0;
  for (int64_t Q = 0; Q < p.n_qfam; Q++) {
    const int64_t sz = p.q_off[Q + 1] - p.q_off[Q];
    if (!p.q_two[Q]) {
      one_sinks += sz;
      continue;
    }
    for (int f = 0; f < F; f++) {
      if (p.q_rank[Q * F + f] == 2) {
        qc2[f]++;
        qs2[f] += sz;
      } else {
        qc1[f]++;
        qs1[f] += sz;
      }
    }
  }
  int64_t two_blocks = 0;
  for (int64_t W = 0; W < p.n_fam; W++) {
    const double k = (double)(p.fam_off[W + 1] - p.fam_off[W]);
    for (int f = 0; f < F; f++) {
      const int n = p.n_f[f], rho = p.fam_rank[W * F + f];
      if (n == 0) continue;
      fl += (double)p.n_snk * k * flops_member(n, rho);
      fl += (double)one_sinks * flops_shared_rows(n, rho);
      if (rho == 1) {
        fl += (double)qc1[f] * flops_adjugate(n - 1) + (double)qs1[f] * flops_kapply(n);
        fl += (double)qc2[f] * flops_block12(n) + (double)qs2[f] * flops_kapply12(n);
        two_blocks += qc1[f] + qc2[f];
      } else if (rho == 2) {
        fl += (double)qc1[f] * flops_rank2_block(n) + (double)qs1[f] * flops_kapply2(n);
        // two changed rows and columns: the (n-2) x (n-2) shared block once, two solves per sink
        fl += (double)qc2[f] * flops_adjugate(n - 2) + (double)qs2[f] * flops_kapply22(n);
        two_blocks += qc1[f] + qc2[f];
      } else {  // three changed rows: every sink one-sided
        fl += (double)(qs1[f] + qs2[f]) * flops_shared_rows(n, rho);
      }
    }
  }
  // adjoint: the forward's block factors, solves and member dets
  // again; per (family, sink, flavour) the aggregated row h and the shared-row cofactor
  // block -- from B^{-1} (computed once per two-sided block) for one-column sink families,
  // from the recomputed shared-row LU with the columns of A1^{-1} otherwise; per pair the
  // scatter and the weight gradients
  double bfl = fl;  // the forward part (without the final combine, added below)
  // The forward's two-row members against one-column sink families: a warp whose 32 sinks
  // all belong to one such family forms each member's dots with the block's first null
  // vector once (they do not depend on the sink), for the first two such flavours of the
  // family; per sink the member then needs the two dots with the second null vector.  The
  // adjoint forms every dot per sink, so only the forward's count changes.
  if (!p.snk_q.empty() && p.n_qfam > 0) {
    std::vector<int64_t> zw(p.n_qfam, 0), zs(p.n_qfam, 0);  // such warps per sink family, their sinks
    for (int64_t w0 = 0; w0 < p.n_snk; w0 += 32) {
      const int64_t w1 = std::min<int64_t>(w0 + 32, p.n_snk);
      const int32_t Q = p.snk_q[w0];
      if (Q < 0 || !p.q_two[Q] || p.snk_q[w1 - 1] != Q) continue;
      zw[Q]++;
      zs[Q] += w1 - w0;
    }
    double save = 0.0;
    for (int64_t W = 0; W < p.n_fam; W++) {
      bool any2 = false;
      for (int f = 0; f < F; f++) any2 |= p.fam_rank[W * F + f] == 2 && p.n_f[f] > 0;
      if (!any2) continue;
      const double k = (double)(p.fam_off[W + 1] - p.fam_off[W]);
      if (k > 32) continue;
      for (int64_t Q = 0; Q < p.n_qfam; Q++) {
        if (zw[Q] == 0) continue;
        int used = 0;
        for (int f = 0; f < F && used < 2; f++) {
          const int n = p.n_f[f];
          if (n == 0 || p.fam_rank[W * F + f] != 2 || p.q_rank[Q * F + f] != 1) continue;
          const double dot = 6.0 + 8.0 * (n - 1);
          save += k * (2.0 * dot * (double)zs[Q] - 2.0 * dot * (double)zw[Q]);
          used++;
        }
      }
    }
    fl -= save;
  }
  for (int64_t W = 0; W < p.n_fam; W++) {
    const double k = (double)(p.fam_off[W + 1] - p.fam_off[W]);
    for (int f = 0; f < F; f++) {
      const int n = p.n_f[f];
      if (n == 0) continue;
      const double M = n - 1;
      const double gh = k * (6.0 * std::max(F - 1, 0) + 1.0 + 8.0 * n);       // gamma_c, h
      double one = flops_shared_rows(n, 1) - 6.0 * M + 8.0 * n + 6.0;           // LU, z, h.z, alpha
      double inv = 0.0;                                                         // columns of A1^{-1}
      for (int i = 0; i < (int)M; i++)
        inv += 8.0 * (M - i - 1) * (M - i - 2) / 2.0 + 8.0 * M * (M - 1) / 2.0 + 6.0 * M;
      one += inv + M * (8.0 * M + 6.0) + M * M * 14.0;                          // eta, beta, cofactor rows
      const double two = 8.0 * n - 2.0 + M * (22.0 * M + 6.0);                  // h.y, eta, cofactor rows
      const double scat = M * n * 2.0 + k * n * 8.0;  // the members' gamma comes with h (gh)
      const int rk = p.fam_rank[W * F + f];
      if (rk >= 2) {
        // rank k = 2, 3: per member D = B Z (k^2 dots), adj(D) and det D, s, E, the member
        // rows' coefficients; per sink the LU of A1 ((n-k) x (n-k)), the columns of A1^{-1},
        // the shared block rows; the scatter of k per member rows and n-k shared rows
        const double K = rk, Mk = n - rk;
        const double adj = rk == 2 ? 6.0 + 8.0
                           : rk == 3 ? 9.0 * 14.0 + 22.0
                                     : K * K * flops_fresh_lu(rk - 1) + 8.0 * K;  // minors by small LUs
        double rr = k * (2.0 * K * K * 8.0 * n + adj + 8.0 + 2.0 * K * K * 6.0);
        rr += flops_adjugate((int)Mk);
        for (int i = 0; i < (int)Mk; i++)
          rr += 8.0 * (Mk - i - 1) * (Mk - i - 2) / 2.0 + 8.0 * Mk * (Mk - 1) / 2.0 + 6.0 * Mk;
        rr += Mk * (K * (8.0 * Mk + 6.0) + 6.0 + Mk * (6.0 + 8.0 * K));
        rr += K * k * n * 8.0 * K + 2.0 * Mk * n;
        bfl += (double)p.n_snk * rr;
        continue;
      }
      bfl += (double)p.n_snk * (gh + scat);
      if (p.fam_rank[W * F + f] == 1 && n >= 2) {
        bfl += (double)(one_sinks + qs2[f]) * one + (double)qs1[f] * two + (double)qc1[f] * inv;
      } else {
        bfl += (double)p.n_snk * one;
      }
    }
  }
  p.two_sided_pairs = two_blocks;
  s.two_sided_blocks = two_blocks;
  int Fa = 0;
  for (int f = 0; f < F; f++) Fa += p.n_f[f] > 0;
  // forward, per pair: the flavour product and w_i times it accumulated; per (family,
  // sink): the sum times w_j, added to the refactored pairs' sum
  const double combine = 6.0 * std::max(Fa - 1, 0) + 4.0;
  fl += combine * (double)p.n_src * (double)p.n_snk + 4.0 * (double)p.n_fam * (double)p.n_snk;
  s.flops_per_call = fl;
  // adjoint, per pair: the flavour product, w_i w_j, accumulate, and the combine of the
  // weight gradients
  const double bcombine = 6.0 * std::max(Fa - 1, 0) + 1.0 + 4.0 + 8.0;
  s.backward_flops_per_call = bfl + bcombine * (double)p.n_src * (double)p.n_snk;
  double fresh = 0.0;
  for (int f = 0; f < F; f++) fresh += flops_fresh_lu(p.n_f[f]);
  s.fresh_lu_flops_per_pair = fresh + combine;
  double bytes = 16.0;
  for (int f = 0; f < F; f++) bytes += 16.0 * p.L_f[f] * p.L_f[f];
  bytes += 4.0 * Tn * (double)(p.n_src + p.n_snk) + 8.0 * (double)(p.n_src + p.n_snk);
  s.bytes_per_call = bytes;
  s.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return MHC_OK;
}

}  // namespace mhc

using namespace mhc;

extern "C" {

const char* mhc_last_error(void) { return g_last_error.c_str(); }

void mhc_plan_opts_default(mhc_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tau_parent = 1e-4;
  o->tau_child = 1e-3;
  o->sink_tile = 0;
  o->rank2 = 1;
  o->max_family = 32;
}

mhc_status mhc_plan(mhc_plan_t* out, int32_t F, const int32_t* n_f, const int32_t* L_f, int64_t n_src,
                    const int32_t* labels_src, const double* w_src, int64_t n_snk,
                    const int32_t* labels_snk, const double* w_snk, const mhc_plan_opts* opts) {
  TraceRange trace("mhc_plan");
  if (!out) {
    set_error("mhc_plan: out is NULL");
    return MHC_EINVAL;
  }
  *out = nullptr;
  if (F <= 0 || F > MHC_FMAX) {
    set_error("mhc_plan: n_flavours must be in [1, " + std::to_string(MHC_FMAX) + "]");
    return MHC_EINVAL;
  }
  if (!n_f || !L_f || !labels_src || !labels_snk || !w_src || !w_snk) {
    set_error("mhc_plan: NULL input pointer");
    return MHC_EINVAL;
  }
  if (n_src <= 0 || n_snk <= 0 || n_src > (int64_t)INT32_MAX || n_snk > (int64_t)INT32_MAX) {
    set_error("mhc_plan: term counts must be in [1, 2^31)");
    return MHC_EINVAL;
  }
  Plan* p = nullptr;
  try {
    p = new Plan();
    p->F = F;
    p->n_f.assign(n_f, n_f + F);
    p->L_f.assign(L_f, L_f + F);
    p->off_f.resize(F);
    int Tn = 0;
    for (int f = 0; f < F; f++) {
      if (n_f[f] < 0 || n_f[f] > MHC_NMAX) {
        set_error("mhc_plan: n_f[" + std::to_string(f) + "] = " + std::to_string(n_f[f]) +
                  " outside [0, " + std::to_string(MHC_NMAX) + "]");
        delete p;
        return MHC_EINVAL;
      }
      if (L_f[f] < 1 || L_f[f] > 4096) {
        set_error("mhc_plan: L_f[" + std::to_string(f) + "] outside [1, 4096]");
        delete p;
        return MHC_EINVAL;
      }
      p->off_f[f] = Tn;
      Tn += n_f[f];
      p->max_n = std::max(p->max_n, (int)n_f[f]);
    }
    p->Tn = Tn;
    p->n_src = n_src;
    p->n_snk = n_snk;
    p->labels_src.assign(labels_src, labels_src + n_src * Tn);
    p->labels_snk.assign(labels_snk, labels_snk + n_snk * Tn);
    p->w_src.assign(w_src, w_src + n_src);
    p->w_snk.assign(w_snk, w_snk + n_snk);
    for (int side = 0; side < 2; side++) {
      const std::vector<int32_t>& lab = side ? p->labels_snk : p->labels_src;
      const int64_t Nn = side ? n_snk : n_src;
      for (int64_t i = 0; i < Nn; i++)
        for (int f = 0; f < F; f++)
          for (int m = 0; m < n_f[f]; m++) {
            const int32_t x = lab[i * Tn + p->off_f[f] + m];
            if (x < 0 || x >= L_f[f]) {
              set_error(std::string("mhc_plan: ") + (side ? "sink" : "source") + " term " +
                        std::to_string(i) + " flavour " + std::to_string(f) + " label " +
                        std::to_string(x) + " outside [0, L_f)");
              delete p;
              return MHC_EINVAL;
            }
          }
    }
    if (opts) {
      p->opts = *opts;
    } else {
      mhc_plan_opts_default(&p->opts);
    }
    if (p->opts.max_family <= 0) p->opts.max_family = 32;
    if (p->opts.max_family > 64) {
      set_error("mhc_plan: max_family must be in [1, 64]");
      delete p;
      return MHC_EINVAL;
    }
    if (!(p->opts.tau_parent >= 0.0 && p->opts.tau_parent < 1.0) ||
        !(p->opts.tau_child >= 0.0 && p->opts.tau_child < 1.0)) {
      set_error("mhc_plan: tau_parent and tau_child must be in [0, 1)");
      delete p;
      return MHC_EINVAL;
    }
    if (p->opts.max_rank < 0 || p->opts.max_rank > MHC_MAX_RANK) {
      set_error("mhc_plan: max_rank must be in [0, MHC_MAX_RANK]");
      delete p;
      return MHC_EINVAL;
    }
    if (p->opts.sink_tile != 0 && p->opts.sink_tile != 32 && p->opts.sink_tile != 64 &&
        p->opts.sink_tile != 128) {
      set_error("mhc_plan: sink_tile must be 0, 32, 64 or 128");
      delete p;
      return MHC_EINVAL;
    }
    mhc_status st = build_plan(*p);
    if (st != MHC_OK) {
      delete p;
      return st;
    }
  } catch (const std::bad_alloc&) {
    delete p;
    set_error("mhc_plan: out of host memory");
    return MHC_ENOMEM;
  }
  *out = reinterpret_cast<mhc_plan_t>(p);
  return MHC_OK;
}

mhc_status mhc_plan_families(mhc_plan_t plan, int64_t* n_families, int64_t* fam_member_offset,
                             int32_t* fam_rank, int32_t* fam_rows, int32_t* fam_ref,
                             int64_t* member_term, int32_t* member_sign, int32_t* member_labels) {
  if (!plan || !n_families) {
    set_error("mhc_plan_families: NULL argument");
    return MHC_EINVAL;
  }
  const Plan& p = *reinterpret_cast<const Plan*>(plan);
  *n_families = p.n_fam;
  if (fam_member_offset) std::copy(p.fam_off.begin(), p.fam_off.end(), fam_member_offset);
  if (fam_rank) std::copy(p.fam_rank.begin(), p.fam_rank.end(), fam_rank);
  if (fam_rows) std::copy(p.fam_rows.begin(), p.fam_rows.end(), fam_rows);
  if (fam_ref) std::copy(p.fam_ref.begin(), p.fam_ref.end(), fam_ref);
  if (member_term) std::copy(p.mem_term.begin(), p.mem_term.end(), member_term);
  if (member_sign) std::copy(p.mem_sign.begin(), p.mem_sign.end(), member_sign);
  if (member_labels) std::copy(p.mem_lab.begin(), p.mem_lab.end(), member_labels);
  return MHC_OK;
}

mhc_status mhc_plan_sinks(mhc_plan_t plan, int64_t* n_sink_families, int32_t* order,
                          int32_t* labels, int32_t* parity, int32_t* family, int32_t* two_sided) {
  if (!plan || !n_sink_families) {
    set_error("mhc_plan_sinks: NULL argument");
    return MHC_EINVAL;
  }
  const Plan& p = *reinterpret_cast<const Plan*>(plan);
  *n_sink_families = p.n_qfam;
  if (order) std::copy(p.snk_order.begin(), p.snk_order.end(), order);
  if (labels) std::copy(p.snk_lab2.begin(), p.snk_lab2.end(), labels);
  if (parity) std::copy(p.snk_par2.begin(), p.snk_par2.end(), parity);
  if (family) std::copy(p.snk_q.begin(), p.snk_q.end(), family);
  if (two_sided) std::copy(p.q_two.begin(), p.q_two.end(), two_sided);
  return MHC_OK;
}

mhc_status mhc_plan_stats(mhc_plan_t plan, mhc_stats* out) {
  if (!plan || !out) {
    set_error("mhc_plan_stats: NULL argument");
    return MHC_EINVAL;
  }
  *out = reinterpret_cast<const Plan*>(plan)->stats;
  return MHC_OK;
}

}  // extern "C"
