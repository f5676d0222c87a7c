// plan.h -- host-side plan of the correlator library (internal header).
//
// A plan is the output of the execution-order step of the method (Sec. 3): the source
// terms grouped into work families.  A work family has, per flavour f, a reference label
// tuple (the dominator's, Sec. 3 greedy dominating set) and a set R_f of one or two
// "changed rows": every member agrees with the reference on the other rows (after
// alignment) and differs only at R_f.  Per (family, sink, flavour) the device factorises
// the shared rows once and evaluates every member with an O(n) dot product (Sec. 2.1).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mhc.h"
#include "layout.h"

namespace mhc {

void set_error(const std::string& msg);

// device counters of a plan: status bits, refactor parent, refactor child, refactor flops,
// row-difference updates
constexpr int kNumCounters = 5;

// Device-side tables of one plan (owned by the plan, allocated on first use).
struct DevicePlan {
  int device = -1;
  int32_t* fam_info = nullptr;   // [W][4]: member offset, member count, pad, pad
  int32_t* fam_rank = nullptr;   // [W][F]
  int32_t* fam_arow = nullptr;   // [W][Tn]: shared-row labels first, then unused
  int32_t* fam_order = nullptr;  // [W] families grouped by y-cache layout (FwdArgs::fam_order), or nullptr
  int n_ranges = 0;              // layout ranges of fam_order (FwdArgs::ranges)
  FwdRange ranges[kMaxFwdRanges] = {};
  int32_t* mem_term = nullptr;   // [n_src] source term index of each member
  int32_t* mem_par = nullptr;    // [n_src] bit f: sign parity of flavour f
  int32_t* mem_lab = nullptr;    // [n_src][F][MHC_MAX_RANK]
  int32_t* snk_lab = nullptr;    // [n_snk][Tn]
  int32_t* src_member = nullptr; // [n_src] member slot of each source term
  int32_t* mem_family = nullptr; // [n_src] family of each member slot
  int32_t* snk_order = nullptr;  // two-sided tables (see Plan)
  int32_t* snk_lab2 = nullptr;
  int32_t* snk_par2 = nullptr;
  int32_t* snk_q = nullptr;
  int32_t* q_off = nullptr;
  int32_t* q_two = nullptr;
  int32_t* q_rank = nullptr;
  double* kbuf = nullptr;        // [W][Q][kstride] LU factors of B, row order, -det B, det B
  int32_t* kguard = nullptr;     // [W][Q][F] 1: the block's pivot guard fired
  double* bwd_stage = nullptr;   // [cta][T][mn_max] adjoint staging
  size_t bwd_stage_bytes = 0;
  double* bwd_accs = nullptr;    // [cta][kmax][T] adjoint dw_src accumulators
  size_t bwd_accs_bytes = 0;
  double* bwd_r2 = nullptr;      // [cta][kmax][4][T] adjoint coefficients of two-row families
  size_t bwd_r2_bytes = 0;
  double* bwd_dets = nullptr;    // [cta][F][kmax][T + 1] adjoint member determinants / gammas
  size_t bwd_dets_bytes = 0;
  double* cw_tmp = nullptr;      // [4][2] real-weight correlators of mhc_correlator_cw
  double* kinv = nullptr;        // [W][Q][sum_f (n_f-1)^2] B^{-1} of two-sided blocks (adjoint)
  size_t kinv_bytes = 0;
  int kstride = 0;
  bool two_sided = false;
  double* w_src = nullptr;       // [n_src] plan weights
  double* w_snk = nullptr;       // [n_snk]
  double* partials = nullptr;    // [items][2] per-work-item partial sums
  unsigned long long* counters = nullptr;  // [kNumCounters]: status bits, refactor parent, child,
                                           // refactor flops, row-difference updates
  int64_t n_items = 0;
  int32_t n_tiles = 0;           // sink tiles per family
  int32_t tile = 0;              // sinks per tile (threads per block)
  // backward workspace (lazy)
  double* bwd_rows = nullptr;    // per (family, chunk) row accumulators
  size_t bwd_rows_bytes = 0;
  double* bwd_wsrc = nullptr;    // [n_src][2] complex dC/dw_src partial sums per sink chunk
  size_t bwd_wsrc_bytes = 0;
  double* bwd_wsnk = nullptr;    // [n_snk][2] per family-chunk partials
  size_t bwd_wsnk_bytes = 0;
  struct BwdIndex {
    int32_t* off = nullptr;      // [L_f + 1]
    int2* ent = nullptr;         // (family, slot) of every accumulator row of label a
  };
  std::vector<BwdIndex> bwd_index;  // per flavour
};

struct Plan {
  // inputs (host copies)
  int F = 0;
  std::vector<int32_t> n_f, L_f, off_f;  // off_f: label offset of flavour f inside a term
  int Tn = 0;                            // sum n_f
  int64_t n_src = 0, n_snk = 0;
  std::vector<int32_t> labels_src, labels_snk;
  std::vector<double> w_src, w_snk;
  mhc_plan_opts opts{};
  // work families
  int64_t n_fam = 0;
  std::vector<int64_t> fam_off;          // [W+1]
  std::vector<int32_t> fam_rank;         // [W][F]
  std::vector<int32_t> fam_rows;         // [W][F][MHC_MAX_RANK]
  std::vector<int32_t> fam_ref;          // [W][Tn]
  std::vector<int32_t> fam_arow;         // [W][Tn]
  std::vector<int64_t> mem_term;         // [n_src]
  std::vector<int32_t> mem_sign;         // [n_src] +-1 (product over flavours)
  std::vector<int32_t> mem_par;          // [n_src] bit f: sign parity of flavour f
  std::vector<int32_t> mem_lab;          // [n_src][F][MHC_MAX_RANK]
  std::vector<int32_t> src_member;       // [n_src] member slot of each source term
  std::vector<int32_t> mem_family;       // [n_src]
  int max_members = 0;
  // sink families (two-sided update): sinks in family-major order, columns aligned to
  // the family's reference with the changed column last in every flavour
  int64_t n_qfam = 0;
  std::vector<int32_t> snk_order;        // [n_snk] original sink index at position jj
  std::vector<int32_t> snk_lab2;         // [n_snk][Tn] aligned column labels
  std::vector<int32_t> snk_par2;         // [n_snk] bit f: column-permutation parity
  std::vector<int32_t> snk_q;            // [n_snk] sink family of position jj
  std::vector<int32_t> q_off;            // [Q+1] first position of each sink family
  std::vector<int32_t> q_two;            // [Q] 1 when the family uses the two-sided update
  std::vector<int32_t> q_rank;           // [Q][F] changed columns (1 or 2) per flavour
  int64_t two_sided_pairs = 0;           // (family, sink family) blocks using it, x flavours
  int max_n = 0;
  // stats
  mhc_stats stats{};
  // device state
  DevicePlan dev;
};

// Builds every host table of `p` from its inputs; returns MHC_OK or sets the error.
mhc_status build_plan(Plan& p);

// Algorithmic flop counts (counting rule: real add/mul 1, fma 2, complex mul 6,
// complex fma 8, complex reciprocal 6, pivot measure |re|+|im| 1).
double flops_shared_rows(int n, int rho);   // factorise + solve for one (family, sink, flavour)
double flops_member(int n, int rho);        // one member's det from the cached solve
double flops_fresh_lu(int n);               // one fresh partial-pivot LU determinant
double flops_kapply(int n);                 // y = [-det(B) B^{-1} a; det B] for one sink
double flops_adjugate(int m);               // LU factors of one m x m two-sided block
double flops_kapply2(int n);                // z2 for one sink (two-row family)
double flops_kapply22(int n);               // z1, z2 for one sink (two-row x two-column block)
double flops_rank2_block(int n);            // LU factors and -U1^{-1}u of one two-row block
double flops_block12(int n);                // LU factors of one (one-row, two-column) block
double flops_kapply12(int n);               // y for one sink of a two-column sink family

}  // namespace mhc
