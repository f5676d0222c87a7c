/*
 * mhc.h -- C ABI of the GB300 multi-hadron correlator library.
 *
 * The library evaluates, on one GPU in complex FP64, the nuclear correlator of
 * Vachaspati & Detmold, "Fast Evaluation of Multi-Hadron Correlation Functions"
 * (Lattice 2014):
 *
 *     C = sum_{i in src} sum_{j in snk} w_i w_j prod_f det G_f^{(ij)},
 *     G_f^{(ij)}[m][n] = S_f[a_i^{f,m}][a_j^{f,n}]
 *
 * (Sec. 1: the correlator as a double sum over wavefunction terms of w_i w_j det G^{(ij)};
 * the definition of G^{(ij)} from the propagator; det G as the product of per-flavour
 * blocks because G is block diagonal in flavour).  The 1/Z and the gauge average of
 * Sec. 1 are not part of a call: one call is one gauge configuration and one time.
 *
 * The determinants follow the determinant-update scheme of Sec. 2 and Sec. 3: source
 * terms are grouped (greedy dominating set of the source-term graph, Sec. 3) into
 * families that share all but one row (or two rows) per flavour; per (family, sink,
 * flavour) the shared rows are LU-factorised once with partial pivoting, and one
 * triangular solve gives det(G) G^{-1} e_r, so each member costs one O(n) dot product
 * (matrix determinant lemma and the cached-solve remark of Sec. 2.1).  A member whose
 * lemma factor, or whose family's pivots, fall below a threshold is refactored from
 * scratch.  Sums are reduced in a fixed order: results are bitwise reproducible.
 *
 * Conventions for every entry point:
 *   - All pointers marked "device" are CUDA device pointers on the current device;
 *     "host" pointers are read during the call only, and the library keeps copies.
 *   - Device calls are asynchronous on the given stream and never synchronise, except
 *     where stated.  Outputs are written (not accumulated) unless stated.
 *   - Every entry point returns an mhc_status; on failure a message is available from
 *     mhc_last_error() (thread-local) and device outputs are left undefined.
 *   - Complex numbers are two doubles (re, im), interleaved.
 *   - S_f is complex128, L_f x L_f, row-major: entry (a, b) at doubles 2(a L_f + b).
 *   - Term labels are int32 [N][sum_f n_f], flavour-major inside a term: the labels of
 *     flavour f of term i start at i * sum_f n_f + sum_{f' < f} n_f'.
 */
#ifndef MHC_H
#define MHC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhc_plan_s* mhc_plan_t;   /* opaque, owned by the library */
typedef struct mhc_batch_s* mhc_batch_t; /* opaque, owned by the library */
typedef void* mhc_stream_t;              /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  MHC_OK = 0,
  MHC_EINVAL = 1,       /* bad argument (validated on the host)                  */
  MHC_ENOMEM = 2,       /* host or device allocation failed                      */
  MHC_ECUDA = 3,        /* a CUDA runtime call failed                            */
  MHC_ETIMEOUT = 4,     /* a bounded device wait ran out                         */
  MHC_ENONFINITE = 5,   /* a non-finite value reached a result (NaN/Inf input)   */
  MHC_EUNSUPPORTED = 6  /* valid request that the library does not implement    */
} mhc_status;

#define MHC_NMAX 32     /* largest n_f (quarks of one flavour in a term) */
#define MHC_FMAX 8      /* largest number of flavours */
#define MHC_MAX_RANK 6  /* most changed rows per family and flavour (stride of the
                           changed-row tables of mhc_plan_families) */

/* Planner options.  mhc_plan_opts_default() fills the defaults listed here. */
typedef struct {
  double tau_parent;   /* refactor all members of a (family, sink, flavour) when the
                          smallest pivot of the shared-row LU is below tau_parent times
                          the largest (magnitudes compared as powers of two). 1e-4   */
  double tau_child;    /* refactor one member when |det| < tau_child * |row| * |y|,
                          the normalised lemma factor (powers of two).          1e-3  */
  int32_t sink_tile;   /* sinks per thread block; 0 = chosen by n class.        0     */
  int32_t rank2;       /* 1: families may differ in two rows per flavour with
                          n_f >= 10 (rank-2 update by a 2x2 generalised cofactor);
                          0: one row.                                           1     */
  int32_t max_family;  /* largest number of members per family, 1..64.          32    */
  int32_t one_sided;   /* 1: only source-side families (Sec. 3 as printed); 0: sink
                          terms are grouped too, and each (source family, sink
                          family) block shares the LU factors of its common rows and
                          columns (two-sided update).                           0     */
  int32_t rank3;       /* 1 (with rank2): source families may also differ in three
                          rows per flavour with n_f >= 14 (rank-3 update: a 3x3
                          generalised cofactor with three null vectors).        0     */
  int32_t max_rank;    /* with rank2: the most rows per flavour in which a source
                          family's members may differ, 2..MHC_MAX_RANK (the rank-k
                          update of Sec. 5: k null vectors of the shared rows and a
                          k x k determinant per member); rank k is used for a
                          flavour with n_f >= 4k + 2 (rank 2: n_f >= 10, rank 3:
                          n_f >= 14, rank 4: 18, 5: 22, 6: 26).  0: 3 with rank3,
                          else 2.                                               0     */
  int32_t first_fit;   /* how a dominated set (Sec. 3) is split into work families whose
                          members differ from the dominator in the same rows:
                          0: by cost -- members with the same changed rows form
                          groups, and the pair of groups whose merge (one shared
                          factorisation per sink, possibly a higher rank for all
                          members) most lowers the plan's flop count is merged
                          until no merge lowers it; 1: first fit in term order
                          (each member joins the first family it fits).        0     */
  int32_t row_difference; /* 0: a member that fails the lemma guard is refactored from
                          scratch; 1: a member of a one- or two-row family is first
                          updated with one of its rows replaced by its difference
                          from the nearest shared row (det [A; b] = det [A; b - a_r]:
                          no cancellation when b nearly repeats a_r), guarded again,
                          and refactored only if that guard fails too.          0     */
  int32_t reserved[3];
} mhc_plan_opts;

/* Planner and run statistics. */
typedef struct {
  int64_t n_src, n_snk;          /* term counts                                       */
  int32_t n_flavours;
  int32_t max_n;                 /* largest n_f                                       */
  int64_t dominators;            /* greedy dominating-set size (Sec. 3)               */
  int64_t families;              /* work families after splitting by changed rows     */
  int64_t rank2_family_flavours; /* (family, flavour) blocks updated at rank 2        */
  int64_t members;               /* == n_src                                          */
  int64_t graph_edges;           /* edges of the source-term graph                    */
  double flops_per_call;         /* algorithmic FP64 flops of one mhc_correlator call,
                                    without refactors (real add/mul 1, FMA 2, complex
                                    multiply 6, complex FMA 8, complex reciprocal 6)  */
  double fresh_lu_flops_per_pair;/* flops of one refactored pair (all flavours)        */
  double bytes_per_call;         /* algorithmic bytes: S_f once, labels, weights, out */
  double plan_seconds;           /* host time spent in mhc_plan                       */
  /* device counters of the last mhc_correlator / backward call (mhc_get_status): */
  int64_t refactor_parent;       /* (member, sink, flavour) refactored by the pivot guard */
  int64_t refactor_child;        /* (member, sink, flavour) refactored by the lemma guard */
  int64_t sink_families;         /* sink-side families (two-sided update)             */
  int64_t two_sided_blocks;      /* (family, sink family, flavour) blocks sharing B's LU */
  double backward_flops_per_call;/* algorithmic FP64 flops of one mhc_correlator_backward */
  int64_t rank3_family_flavours; /* (family, flavour) blocks updated at rank 3        */
  double refactor_flops;         /* algorithmic FP64 flops of the refactor path in the calls
                                    read by the last mhc_get_status (same counting rule as
                                    flops_per_call; a group of pairs refactored together
                                    counts its shared elimination once)                */
  int64_t rank4plus_family_flavours; /* (family, flavour) blocks updated at rank >= 4   */
  int64_t row_difference;        /* (member, sink, flavour) that failed the lemma guard and
                                    took the row-difference update instead of a refactor
                                    (mhc_plan_opts.row_difference = 1)                 */
} mhc_stats;

/* Thread-local message describing the last failure of this thread's last call. */
const char* mhc_last_error(void);

/* Fill *opts with the defaults. */
void mhc_plan_opts_default(mhc_plan_opts* opts);

/*
 * Build a plan (host only; Sec. 3 execution order).  Validates the inputs, builds the
 * source-term graph (two terms are adjacent when, in every flavour, their label
 * multisets differ in at most one label, or two with opts->rank2), takes the greedy
 * maximum-degree dominating set (ties to the lowest term index), aligns every member
 * to its dominator's label positions (the permutation sign goes into the member's
 * sign) and splits each dominated set into work families whose members change the
 * same row (or row pair) per flavour.
 *   n_flavours      : F, 0 < F <= MHC_FMAX
 *   n_f, L_f        : host int32[F]; 0 <= n_f <= MHC_NMAX, 1 <= L_f <= 4096
 *   n_src, n_snk    : term counts, > 0
 *   labels_src/_snk : host int32 [N][sum n_f], each label of flavour f in [0, L_f)
 *   w_src, w_snk    : host float64 [N]; default weights of the correlator calls
 *   opts            : NULL for the defaults
 * The plan is reusable across propagators S_f (Sec. 3: the graph and the dominating
 * set do not depend on the gauge configuration).  Its device tables are uploaded by
 * the first device call that uses it (a synchronous copy on the current device);
 * issue that first call outside any stream capture.  Repeated labels are allowed and
 * give det = 0.  n_f = 0 makes flavour f a factor 1.
 * Errors: MHC_EINVAL (bad sizes or labels, null pointers), MHC_ENOMEM.
 */
mhc_status mhc_plan(mhc_plan_t* out, int32_t n_flavours, const int32_t* n_f, const int32_t* L_f,
                    int64_t n_src, const int32_t* labels_src, const double* w_src, int64_t n_snk,
                    const int32_t* labels_snk, const double* w_snk, const mhc_plan_opts* opts);

/* Release a plan and its device tables (synchronises the device first). NULL is a no-op. */
void mhc_plan_destroy(mhc_plan_t plan);

/* Copy the plan's statistics (including the last run's device counters, as of the
 * last mhc_get_status). */
mhc_status mhc_plan_stats(mhc_plan_t plan, mhc_stats* out);

/*
 * Export the work families (host; for inspection and tests).  Pass NULL for the
 * arrays to query the sizes only.  With W = *n_families and Tn = sum_f n_f:
 *   fam_member_offset : int64 [W+1]; members of family w are [off[w], off[w+1])
 *   fam_rank          : int32 [W][F]; 0 (n_f = 0), else 1..MHC_MAX_RANK changed rows
 *   fam_rows          : int32 [W][F][MHC_MAX_RANK]; changed-row positions in the reference
 *                       tuple (ascending; -1 when unused)
 *   fam_ref           : int32 [W][Tn]; the dominator's labels (reference tuple)
 *   member_term       : int64 [n_src]; source term of each member
 *   member_sign       : int32 [n_src]; +-1: det of the term's own label order equals
 *                       member_sign times prod_f det [shared rows; member rows]
 *   member_labels     : int32 [n_src][F][MHC_MAX_RANK]; the member's labels at the changed
 *                       rows
 * "[shared rows; member rows]" is the matrix whose rows are, in order, the reference
 * tuple's labels at the positions not in fam_rows (ascending), then the member's labels
 * at fam_rows (ascending), and whose columns are the sink term's labels.
 */
mhc_status mhc_plan_families(mhc_plan_t plan, int64_t* n_families, int64_t* fam_member_offset,
                             int32_t* fam_rank, int32_t* fam_rows, int32_t* fam_ref,
                             int64_t* member_term, int32_t* member_sign, int32_t* member_labels);

/*
 * Export the sink-side families of the two-sided update (host; for inspection and
 * tests).  Sinks are evaluated in family-major order; for every flavour the columns of a
 * sink are aligned to its family's reference tuple with the family's changed column last,
 * so all members of a family share their first n_f - 1 columns.  NULL arrays skip.
 *   n_sink_families : number of sink families Q
 *   order           : int32 [n_snk]; original sink index at each position
 *   labels          : int32 [n_snk][sum n_f]; aligned column labels at each position
 *   parity          : int32 [n_snk]; bit f = parity of the column permutation (the
 *                     determinant in the original column order is (-1)^bit times the
 *                     determinant in the aligned order)
 *   family          : int32 [n_snk]; sink family of each position
 *   two_sided       : int32 [Q]; 1 when the family shares B's factors (two or more sinks)
 * With opts->one_sided every sink is its own family and the update is one-sided.
 */
mhc_status mhc_plan_sinks(mhc_plan_t plan, int64_t* n_sink_families, int32_t* order,
                          int32_t* labels, int32_t* parity, int32_t* family, int32_t* two_sided);

/*
 * Forward correlator on the GPU: C = sum_i sum_j w_i w_j prod_f det G_f^{(ij)} for one gauge
 * configuration (Sec. 1: the correlator as a double sum over wavefunction terms, G^{(ij)}
 * gathered from the propagator, det G the product of the flavour blocks), each determinant
 * by the update scheme of Sec. 2 (LU of the shared rows) and Sec. 2.1 (matrix determinant
 * lemma with the solve G^{-1}e_r cached for every member that changes the same row).
 *   S_f        : host array of F device pointers, each complex128 L_f x L_f (may alias)
 *   w_src_dev  : device float64 [n_src] source weights, or NULL for the plan's
 *   w_snk_dev  : device float64 [n_snk] sink weights, or NULL for the plan's
 *   out_dev    : device float64 [2]: (Re C, Im C), written
 *   stream     : cudaStream_t
 * The plan holds the workspace: calls with the same plan must not overlap on the GPU.
 * Non-finite results set a device status bit reported by mhc_get_status.
 */
mhc_status mhc_correlator(mhc_plan_t plan, const double* const* S_f, const double* w_src_dev,
                          const double* w_snk_dev, double* out_dev, mhc_stream_t stream);

/*
 * Forward correlator with complex weights w_i = w_src_re[i] + i w_src_im[i] and
 * w_j = w_snk_re[j] + i w_snk_im[j] (all four device float64 arrays, required), for
 * wavefunctions with complex coefficients.  The sum is bilinear in the weights, so
 *   C = C(re, re) - C(im, im) + i (C(re, im) + C(im, re))
 * with C(x, y) the real-weight correlator of mhc_correlator (Sec. 1); the block factors
 * are computed once for the four passes and the combination runs on the device.
 * out_dev: device float64 [2], (Re C, Im C).  Not a separate method in the paper.
 */
mhc_status mhc_correlator_cw(mhc_plan_t plan, const double* const* S_f, const double* w_src_re,
                             const double* w_src_im, const double* w_snk_re, const double* w_snk_im,
                             double* out_dev, mhc_stream_t stream);

/*
 * Adjoint (hand-written; Jacobi's formula d det G / dG = cofactor matrix: the member
 * rows' cofactors are the forward's cached solves, the shared rows' come from B^{-1} of
 * each two-sided block or from the recomputed shared-row LU, never dividing by det G).  With g = g_out[0] + i g_out[1] = dL/dRe C + i dL/dIm C and the
 * holomorphic derivatives D_S = dC/dS_f, D_w = dC/dw:
 *   dS_f[a][b] = g * conj(D_S[a][b])      (complex128 L_f x L_f, device, written)
 *   dw_src[i]  = Re(conj(g) * D_w_src[i]) (float64, device, written)
 *   dw_snk[j]  = Re(conj(g) * D_w_snk[j]) (float64, device, written)
 * which is PyTorch's convention for the gradient of a real loss.  g_out_dev is a device
 * pointer to 2 doubles.  Any of dS_f (the whole array or single entries), dw_src_dev or
 * dw_snk_dev may be NULL to skip that output.  The dS_f buffers must not alias each
 * other.  Families of k = 2 ... MHC_MAX_RANK changed rows are differentiated through the
 * null vectors of their shared rows; where those rows fail the pivot guard for a sink, the
 * null vectors are recomputed with complete pivoting, and where the shared rows are exactly
 * rank-deficient (every member's determinant and member-row cofactor is then 0) the shared
 * rows' cofactors come from signed minors.  A member whose lemma guard fails takes its
 * determinant (which weights the other flavours' cofactors) from a fresh LU, or with
 * opts.row_difference from the row-difference update first, as in the forward.  The plan
 * holds the adjoint's workspace (per block of sinks: row accumulators, staged cofactors,
 * member determinants; allocated on the first call and grown when needed): calls with the
 * same plan must not overlap on the GPU.  Not in the paper.
 */
mhc_status mhc_correlator_backward(mhc_plan_t plan, const double* const* S_f,
                                   const double* w_src_dev, const double* w_snk_dev,
                                   const double* g_out_dev, double* const* dS_f,
                                   double* dw_src_dev, double* dw_snk_dev, mhc_stream_t stream);

/*
 * Allocation-free forward correlator.  The paper has no counterpart: this entry point
 * exists for callers that cannot let the library allocate device memory during a call,
 * for example a process whose device memory is entirely reserved up front by its own
 * pool allocator (where a cudaMalloc can fail or fragment the pool), or a latency-critical
 * loop that must not pay for an allocation (cudaMalloc and cudaFree may synchronise the
 * device).  Same arguments and result as mhc_correlator; the call allocates nothing.
 *   - Its scratch (one partial sum per work item) is a fixed array of
 *     MHC_NOALLOC_MAX_ITEMS entries (1 MiB) in the library's own device memory; every GPU
 *     that loads the library holds it until the process exits.  A plan with more work
 *     items (families x ceil(n_snk / sink tile)) is rejected with MHC_EINVAL.
 *   - The plan's device tables must already be on the current device: call
 *     mhc_correlator once with the plan first (that call allocates and uploads them).
 *     Otherwise MHC_EINVAL.
 *   - The first call on a device looks up the array's device address (a one-time set-up);
 *     make that first call before any stream capture.  The address is kept for the life of
 *     the process: a cudaDeviceReset (which reloads the library's device code) is not
 *     supported after that first call.
 *   - Every call shares the array, which keeps the last call's contents (each work item
 *     overwrites its own slot before it is read, so nothing needs clearing).  Calls that
 *     overlap on the GPU race on it: issue them on one stream or otherwise in order.
 *   - Status and refactor counters go to the plan's status word (mhc_get_status).
 */
#define MHC_NOALLOC_MAX_ITEMS 65536
mhc_status mhc_correlator_noalloc(mhc_plan_t plan, const double* const* S_f,
                                  const double* w_src_dev, const double* w_snk_dev,
                                  double* out_dev, mhc_stream_t stream);

/*
 * Per-pair determinants through the same update path (families, lemma, guards):
 *   i_dev, j_dev : device int64 [n_pairs] source and sink term indices
 *   dets_dev     : device float64 [n_pairs][F][2], det of each flavour block in the
 *                  terms' own label order, written
 *   path_dev     : device int32 [n_pairs] or NULL; bit f set when flavour f of the
 *                  pair was refactored from scratch by a guard, bit 8 + f when it took
 *                  the row-difference update (see mhc_plan_opts.row_difference)
 * Indices out of range give MHC_EINVAL through the device status (mhc_get_status).
 */
mhc_status mhc_pair_dets(mhc_plan_t plan, const double* const* S_f, int64_t n_pairs,
                         const int64_t* i_dev, const int64_t* j_dev, double* dets_dev,
                         int32_t* path_dev, mhc_stream_t stream);

/*
 * Wait for the stream, read the plan's device status word and counters, clear them.
 * Returns MHC_OK, MHC_ENONFINITE, MHC_EINVAL (bad pair index) or MHC_ETIMEOUT.
 */
mhc_status mhc_get_status(mhc_plan_t plan, mhc_stream_t stream);

/*
 * Batching: many independent correlators (each its own plan, flavour sizes and term
 * counts) in one persistent launch, captured once into a CUDA graph.
 * mhc_batch_create splits the correlators by n class (largest n_f <= 8, <= 18, <= 32; one
 * persistent kernel each) and chooses each class's sink tile (32, 64 or 128 threads per
 * block, one thread per sink: 1, 2 or 4 warps) on the current device.  A class's tile is
 * read from the tuning cache when the cache holds its key -- the GPU, this build of the
 * library, the class and the (n_f, L_f) of its correlators -- and otherwise timed (the
 * class's kernel alone on scratch propagators, every candidate tile) and written to the
 * cache.  The cache is the file named by the environment variable MHC_TUNE_CACHE (empty:
 * no cache), else $HOME/.cache/mhc/tune.jsonl, one JSON object per line.  The call
 * synchronises and uploads the plans.
 *   plans : host array of `count` plans; they must outlive the batch.  A plan may appear
 *           more than once: one plan evaluated on several propagator sets (gauge
 *           configurations, time slices) in one launch, as the paper amortises the plan
 *           (Sec. 3); its later entries get their own block-factor buffers.
 */
mhc_status mhc_batch_create(mhc_batch_t* out, int32_t count, const mhc_plan_t* plans);
void mhc_batch_destroy(mhc_batch_t batch);

/*
 * Evaluate every correlator of the batch:
 *   S    : host array [count] of host arrays [F_b] of device pointers (each plan's S_f)
 *   outs : host array [count] of device pointers to 2 doubles, written
 * The plans' own weights are used.  The first call with a given set of pointers captures
 * a CUDA graph; later calls with the same pointers replay it.
 */
mhc_status mhc_batch_correlator(mhc_batch_t batch, const double* const* const* S,
                                double* const* outs, mhc_stream_t stream);

/* Launch shape of the batch: the sink tile (threads per block) of the n class with the most
 * work items, and the total number of work items. */
mhc_status mhc_batch_info(mhc_batch_t batch, int32_t* threads_per_block, int32_t* tiles_total);

/*
 * Chosen launch shape per n class (classes: largest n_f <= 8, <= 18, <= 32):
 *   tiles      : host int32 [3], the sink tile (threads per block) of each class, 0 if unused
 *   from_cache : host int32 [3] or NULL, 1 where the tile came from the tuning cache
 *   tune_ms    : host float64 [3][3] or NULL, the class kernel's time (ms) at tiles 32, 64,
 *                128 when it was timed (0: not timed, -1: did not fit in shared memory)
 */
mhc_status mhc_batch_shape(mhc_batch_t batch, int32_t* tiles, int32_t* from_cache, double* tune_ms);

/*
 * Tuning cache access (host only; see mhc_batch_create for the file and its keys).
 * mhc_tune_cache_get writes the cached tile for `key` to *tile, or 0 when there is none.
 * mhc_tune_cache_put appends `key` -> tile (32, 64 or 128); the key must hold no quote,
 * backslash or newline.  MHC_EINVAL when the cache is disabled or not writable.
 */
mhc_status mhc_tune_cache_get(const char* key, int32_t* tile);
mhc_status mhc_tune_cache_put(const char* key, int32_t tile);

/*
 * FP64 peak probe: runs independent DFMA chains on every SM for about `iters` x 8 FMAs
 * per thread and returns the measured rate in FLOP/s (2 per DFMA) in *flops.  Used to
 * state the roofline denominator on the same GPU and clocks as a measurement.
 */
mhc_status mhc_fp64_peak(int32_t iters, double* flops, mhc_stream_t stream);

/*
 * Diagnostic: the device complex reciprocal that every pivot of the factorisations uses,
 * applied elementwise: out[i] = 1 / z[i] (z_dev, out_dev: device complex128 [n]).  It forms
 * 1/z = conj(z) / |z|^2 with |z|^2 unscaled and 1/|z|^2 by Newton-Raphson refinement of the
 * hardware approximation, so it is accurate for 2^-510 <= |z| <= 2^510 (outside, |z|^2
 * leaves the normal range): there each component is within 5 u of the exact value's
 * component (u = 2^-53; first-order bound 4 u).  Not a step of the paper's method; it lets
 * a test state that accuracy.  Asynchronous on `stream`.
 */
mhc_status mhc_complex_reciprocal(int64_t n, const double* z_dev, double* out_dev, mhc_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MHC_H */
