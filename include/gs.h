/*
 * gs.h -- C ABI of the GB300 epsilon-relative Gaussian summation library.
 *
 * The library computes, for M query points x_q, N weighted reference points
 * x_r (weights w_r > 0) in D dimensions and nh bandwidths h_j,
 *
 *     G(x_q; h_j) = sum_{r=1..N} w_r exp(-||x_q - x_r||^2 / (2 h_j^2))
 *
 * (Lee & Gray, "Faster Gaussian Summation: Theory and Experiment", Section 1),
 * either exhaustively (eps == 0) or by the dual-tree method of Sections 5-6
 * with every result within relative error eps of the exact sum.
 *
 * Conventions shared by every entry point
 *   - Point arrays are row-major (point-major): element (i, d) at i*D + d,
 *     float (GS_F32) or double (GS_F64) as the dtype argument says.
 *   - Unless an argument says "host", every array pointer is DEVICE memory on
 *     the current CUDA device, owned by the caller, and must stay valid until
 *     the call returns.  The library never frees caller memory.
 *   - Bandwidth lists h and scalars are HOST values.
 *   - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Work is enqueued on that stream; each call synchronises with
 *     the stream once at its end to read the device status word, so outputs
 *     are ready when the call returns GS_OK.
 *   - Scratch memory is taken with cudaMallocAsync on the stream and returned
 *     before the call returns.
 *   - Return value: GS_OK (0) or one of the negative GS_ERR_* codes below; a
 *     short description of the last error is available from gs_last_error().
 *     No C++ exception crosses this boundary.  On error the contents of out
 *     are unspecified.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define GS_OK               0
#define GS_ERR_ARG         -1   /* bad size, pointer, dtype, h <= 0, eps outside [0,1) ... */
#define GS_ERR_WEIGHT      -2   /* a weight <= 0 (Section 1 requires w_r > 0)              */
#define GS_ERR_NONFINITE   -3   /* a coordinate or weight is NaN or infinite               */
#define GS_ERR_OOM         -4   /* device scratch allocation failed                        */
#define GS_ERR_CAPACITY    -5   /* a device work list outgrew its capacity (see gs_opts)   */
#define GS_ERR_TIMEOUT     -6   /* a bounded device wait gave up                           */
#define GS_ERR_CUDA        -7   /* a CUDA runtime call or kernel launch failed             */
#define GS_ERR_UNSUPPORTED -8   /* valid request the library does not implement            */

/* ---- element types ---------------------------------------------------- */
#define GS_F32 0
#define GS_F64 1

/* ---- traversal method selectors (gs_opts.selector) --------------------- */
#define GS_SEL_RULE        0    /* FD, then the cheapest certified series method (Fig. 6)  */
#define GS_SEL_MLP         1    /* learned ordering of the same certified choices          */
#define GS_SEL_FD_ONLY     2    /* finite-difference pruning only (DFD / DFDO)             */
#define GS_SEL_EXHAUSTIVE  3    /* no pruning: every pair summed exactly                   */

/* Tuning and behaviour switches.  Zero-initialised fields take defaults, so
 * `gs_opts o = {0};` (or a NULL pointer) is the default configuration. */
typedef struct gs_opts {
    int32_t leaf_size;      /* kd-tree leaf capacity L; 0 -> 32                          */
    int32_t plimit;         /* highest series order PLIMIT; 0 -> Section 6 table by D   */
    int32_t selector;       /* GS_SEL_*                                                  */
    int32_t no_tokens;      /* 1 disables the W_T token scheme (plain Theorem 2 rule)   */
    int32_t floor_log2;     /* relative floor: results are certified to
                               |G~ - G| <= eps * max(G, 2^floor_log2 * W), W = sum w;
                               0 -> -40                                                 */
    int32_t flags;          /* GS_FLAG_* bits                                            */
    int64_t pair_capacity;  /* initial work-list capacity in pairs; 0 -> automatic     */
    double  cost_weight[4]; /* multipliers of the Fig. 6 costs c_DH, c_DL, c_H2L and
                               c_Direct; all 0 -> GS_COST_* defaults below (calibrated
                               to GB300 unit costs); all 1 -> the paper's cost model   */
    const float *selector_params;  /* GS_SEL_MLP: DEVICE array of GS_MLP_NPARAM floats (the
                               pair-selector network, see gs_mlp_train); read during the
                               call; required for GS_SEL_MLP, ignored otherwise        */
    double  small_work;     /* GS_FLAG_SMALL_EXHAUSTIVE threshold on M N nh; 0 -> GS_SMALL_WORK,
                               or GS_SMALL_WORK_D2 when D <= 2                          */
    int64_t reserved[2];
} gs_opts;

/* gs_opts.flags */
#define GS_FLAG_NO_MERGE 1  /* base case per bandwidth, without merging the leaf pairs
                               that several bandwidths share                           */
#define GS_FLAG_SMALL_EXHAUSTIVE 2  /* eps > 0 problems whose exhaustive work M N nh is at
                               most gs_opts.small_work (0: GS_SMALL_WORK, or GS_SMALL_WORK_D2
                               for D <= 2) are summed exhaustively (their error,
                               about 1e-5, is within eps).  GS_SMALL_WORK = 2^39 is the
                               crossover measured on GB300 for D = 3: 1e5 points x 16
                               bandwidths (1.6e11 terms) take 21 ms exhaustively and 35 ms
                               by the dual tree; 1e6 points x 16 (1.6e13) take 2.1 s and
                               1.1 s.  In higher D the crossover is later still.        */
#define GS_SMALL_WORK 549755813888.0
#define GS_SMALL_WORK_D2 68719476736.0  /* the same threshold for D <= 2 (2^36), where the tree
                               prunes best: measured per problem on 256 uneven batch problems
                               (8 bandwidths from 1e-3 to 1 times the diameter, eps 1e-2),
                               the dual tree wins from about 4e10 terms in D = 2 (1e5 points:
                               7.4 ms against 12.7 ms exhaustively; 2e5: 14.3 against 42.8) and
                               loses up to 2e5 points for every D >= 3 (D = 8, 1.3e5 points:
                               79 ms against 23 ms)                                    */
#define GS_FLAG_NO_TC 4     /* 9 <= D <= 16: no tensor-core base case (every leaf pair summed
                               by the direct FP32 kernel; the FP32 charge drops its extra
                               tensor-core term)                                         */
#define GS_FLAG_BEST_FIRST 8 /* best-first ordering inside each frontier level (the
                               priority-queue traversal of Section 1, ordered by bound
                               gap): in every (query node, bandwidth) group the pairs whose
                               gap W_R (K(delta_min) - K(delta_max)) is at least 1/8 of the
                               group's total are expanded one level on the reference side
                               before the group's decisions, and their children's lower
                               bound replaces theirs in G^min when larger.  Same eps
                               guarantee; an ablation, off by default                    */

/* Default cost weights: a series action runs in FP64 on the GPU while a
 * direct (base-case) term is an FP32 exponential, so on GB300 one unit of
 * series cost is weighted 32 units of direct cost. */
#define GS_COST_DH      32.0
#define GS_COST_DL      32.0
#define GS_COST_H2L     32.0
#define GS_COST_DIRECT   1.0

/* Phases timed into gs_stats.ms_phase (CUDA events on the call's stream). */
#define GS_PH_INGEST    0   /* input checks and packing                              */
#define GS_PH_TREE      1   /* kd-tree build, node statistics, moments (a2, a3)      */
#define GS_PH_FRONTIER  2   /* node-pair frontier iterations (a4)                    */
#define GS_PH_SERIES    3   /* DH / DL / H2L kernels (a5-a7)                         */
#define GS_PH_BASE      4   /* exhaustive or leaf-leaf base-case kernel (a8, a14)    */
#define GS_PH_DOWN      5   /* downward pass and output (a9)                         */
#define GS_PH_OTHER     6   /* everything else (e.g. LSCV reduction)                 */
#define GS_PH_BASE_TC   7   /* the tensor-core base-case kernel (9 <= D <= 16), timed
                               apart from the rest of GS_PH_BASE                        */
#define GS_NPHASE       8

/* Per-call counters (host struct filled by the call when non-NULL; timing
 * events are only recorded when it is non-NULL). */
typedef struct gs_stats {
    int64_t pairs_fd;        /* node pairs pruned by finite differences                 */
    int64_t pairs_dh;        /* ... by direct Hermite evaluation (Lemma 4)              */
    int64_t pairs_dl;        /* ... by direct local accumulation (Lemma 5)              */
    int64_t pairs_h2l;       /* ... by Hermite-to-local translation (Lemma 6)           */
    int64_t pairs_base;      /* leaf-leaf pairs summed exhaustively                     */
    int64_t pairs_split;     /* node pairs split into children                          */
    int64_t point_pairs_base;/* point-point kernel evaluations (x bandwidths) in the
                                base case or exhaustive kernel                          */
    int64_t launches;        /* kernels this call launched                              */
    int64_t launches_base;   /* of which base-case / exhaustive kernels                 */
    int32_t levels;          /* frontier iterations                                     */
    int32_t retries;         /* capacity-driven reruns                                  */
    double  fp32_rel_bound;  /* a-priori relative error bound of the FP32 base case     */
    double  eps_traversal;   /* eps left for pruning after the FP32 charge              */
    double  ms_total;        /* device time of the whole call (CUDA events)             */
    double  ms_phase[GS_NPHASE]; /* device time per GS_PH_* phase                       */
    double  ms_series[3];     /* device time of the DH, DL and H2L kernels (within GS_PH_SERIES) */
    int64_t point_pairs_tc;  /* of point_pairs_base, those summed by the tensor-core base
                                case (9 <= D <= 16)                                     */
    double  ms_base_kernels[2]; /* device time of the base-case summation kernels proper
                                (CUDA events around their launches, without the list
                                building): [0] the tensor-core kernel (point_pairs_tc
                                terms), [1] the direct kernel (the other base-case
                                terms)                                                  */
} gs_stats;

/* Library version string (static storage). */
const char *gs_version(void);

/* Description of the last error returned on the calling host thread
 * (static thread-local storage; "" when none). */
const char *gs_last_error(void);

/* Fill *o with the defaults; returns GS_OK, or GS_ERR_ARG when o is NULL. */
int gs_opts_default(gs_opts *o);

/*
 * gs_sum -- Gaussian sums of M queries against N weighted references for nh
 * bandwidths (Section 1's G(x_q); Sections 5-6 for eps > 0).
 *
 *   queries  device, M x D, dtype                  (may equal refs: monochromatic)
 *   M        number of queries, >= 1
 *   refs     device, N x D, dtype
 *   weights  device, N floats, every w_r > 0 and finite
 *   N        number of references, >= 1
 *   D        dimension, 1 <= D <= 32
 *   dtype    GS_F32 or GS_F64 (both point arrays)
 *   h        HOST, nh bandwidths, each finite and > 0
 *   nh       1 <= nh <= 64
 *   eps      0 selects the exhaustive sum (every term, FP32 kernel arithmetic
 *            with FP64 per-query accumulation); 0 < eps < 1 selects the
 *            dual-tree method with |G~ - G| <= eps * max(G, floor) per query
 *   out      device, M x nh doubles, row-major: out[q*nh + j] = G~(x_q; h_j),
 *            queries in the caller's order
 *   opts     host, may be NULL (defaults)
 *   stream   cudaStream_t as void*, may be NULL
 *   stats    host, may be NULL
 */
int gs_sum(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N,
           int D, int dtype, const double *h, int nh, double eps, double *out,
           const gs_opts *opts, void *stream, gs_stats *stats);

/*
 * gs_sum_trace -- gs_sum (eps > 0 only) that also records how the traversal
 * treated every node pair, for verification against a reference traversal.
 *   trace      device, 4 x trace_cap int32; record i = (query node, reference
 *              node, bandwidth index, action | order << 8 | iteration << 16)
 *              in processing order (iterations ascending; inside one,
 *              groups (bandwidth, query node) ascending, reference nodes
 *              ascending).  Nodes are heap-numbered (root 0, children of k at
 *              2k+1, 2k+2).  Actions: 0 FD, 1 DH, 2 DL, 3 H2L, 4 base case,
 *              5 split.  Records past trace_cap are dropped.
 *   trace_len  host, written with the total number of records (may exceed
 *              trace_cap)
 *   qperm      device, M int32 or NULL: sorted position -> query index
 *   rperm      device, N int32 or NULL: sorted position -> reference index
 * Errors as gs_sum; GS_ERR_ARG when eps == 0.
 */
int gs_sum_trace(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N,
                 int D, int dtype, const double *h, int nh, double eps, double *out,
                 const gs_opts *opts, void *stream, gs_stats *stats, int32_t *trace, int64_t trace_cap,
                 int64_t *trace_len, int32_t *qperm, int32_t *rperm);

/*
 * gs_lscv -- least-squares cross-validation scores of a weighted Gaussian
 * kernel density estimate over a bandwidth sweep (Section 7: the bandwidth
 * range "according to the standard least-squares cross-validation scores").
 * With normalised weights wbar_i = w_i / W and phi_h the normalised Gaussian,
 *   LSCV(h) = int f^2 - 2 sum_i wbar_i f_{-i}(x_i)
 *           = (4 pi h^2)^{-D/2} sum_i wbar_i G_{sqrt2 h}(x_i) / W
 *             - 2 (2 pi h^2)^{-D/2} sum_i wbar_i (G_h(x_i) - w_i) / (W - w_i),
 * so one monochromatic dual-tree pass over the 2 nh bandwidths
 * {h_j} u {sqrt2 h_j} gives every score.
 *   pts        device, N x D, dtype (queries = references)
 *   weights    device, N floats > 0
 *   h          HOST, nh bandwidths, 1 <= nh <= 32
 *   eps        relative error of every Gaussian sum (0 = exhaustive)
 *   score      HOST, nh doubles: LSCV(h_j)
 *   score_err  HOST, nh doubles or NULL: a-posteriori bound on |score error|
 *              implied by eps, eps * [(4 pi h^2)^{-D/2} sum wbar G_{sqrt2 h}/W
 *              + 2 (2 pi h^2)^{-D/2} sum wbar G_h / (W - w_i)]
 * stats, if given, describe the underlying gs_sum call.  Errors as gs_sum;
 * GS_ERR_ARG when N < 2.
 */
int gs_lscv(const void *pts, int64_t N, int D, int dtype, const float *weights, const double *h, int nh,
            double eps, double *score, double *score_err, const gs_opts *opts, void *stream, gs_stats *stats);

/*
 * gs_sum_host -- gs_sum for callers whose data lives in HOST memory: every
 * array argument (queries, refs, weights, out) is host memory.  The call
 * copies the inputs to device scratch, runs gs_sum on `stream`, copies out
 * back and returns when out is ready.  Same argument meaning and errors as
 * gs_sum.
 */
int gs_sum_host(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N,
                int D, int dtype, const double *h, int nh, double eps, double *out,
                const gs_opts *opts, void *stream, gs_stats *stats);

/*
 * gs_lscv_host -- gs_lscv for callers whose points and weights live in HOST
 * memory (pts: host N x D, dtype; weights: host N floats).  The call copies
 * them to device scratch, runs gs_lscv on `stream` and returns the scores in
 * the HOST arrays score / score_err as gs_lscv does.  Same arguments,
 * results and errors as gs_lscv (Section 7's LSCV sweep).
 */
int gs_lscv_host(const void *pts, int64_t N, int D, int dtype, const float *weights, const double *h, int nh,
                 double eps, double *score, double *score_err, const gs_opts *opts, void *stream,
                 gs_stats *stats);

/*
 * gs_sum_exhaustive_noalloc -- the exhaustive sum (gs_sum with eps = 0) for
 * callers that cannot let the library allocate device memory: runtimes that
 * own all device memory through their own allocator and forbid direct
 * cudaMalloc calls, or processes that allocate everything up front and must
 * not fail or stall on an allocation mid-run.  The paper has no counterpart;
 * this is a deployment variant of the same computation.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its scratch
 * (a status word and the packed reference records) lives in one fixed 16 MiB
 * array of the library's device memory, which stays resident on each device
 * that used it until the process exits.  Limits: the packed references must
 * fit that array -- e.g. up to about 1.0e6 references for FP32 data with
 * D <= 3, 5.2e5 for D <= 7, 2.1e5 for D = 16; larger N returns GS_ERR_ARG with
 * a message naming the limit.
 *
 * First call per device: the CUDA runtime loads the library's device code on
 * a device lazily, at its first use there, and that load maps the array and
 * may allocate inside the driver (and can fail with an out-of-memory error).
 * A caller that must not allocate mid-run makes one warm-up call per device
 * at start-up, before any stream capture; later calls allocate nothing.
 * Each call looks up the array's address for the current device
 * (cudaGetSymbolAddress, a host-side lookup once the code is loaded), so the
 * call stays correct after cudaDeviceReset -- which frees the array: the next
 * call on that device is a first call again.  Every call shares the array
 * and each call resets what it needs, but calls whose GPU work overlaps
 * (other streams, other host threads) race on it: serialise them.
 *
 * Arguments, layouts and results are those of gs_sum (device queries, refs,
 * weights and out; HOST h; dtype GS_F32 or GS_F64; 1 <= nh <= 64).  Returns
 * when out is ready, with GS_OK or GS_ERR_ARG, GS_ERR_WEIGHT,
 * GS_ERR_NONFINITE or GS_ERR_CUDA.
 */
int gs_sum_exhaustive_noalloc(const void *queries, int64_t M, const void *refs, const float *weights,
                              int64_t N, int D, int dtype, const double *h, int nh, double *out,
                              void *stream);

/* ---- trees built once, summed many times ---------------------------------
 *
 * A gs_tree holds the kd-tree of one point set (Section 5: the node boxes,
 * weight sums and the packed point records, in the library's own device
 * memory) so that several sums over the same data -- other bandwidths, other
 * eps, other query sets -- do not rebuild it.  A reference tree (built with
 * weights) also keeps a copy of the weights and the weight range. */
typedef struct gs_tree gs_tree;

/*
 * gs_build_tree -- build the tree of n points (DEVICE, n x D, dtype) with
 * optional weights (DEVICE, n floats; NULL for a query-only tree).  The
 * leaf size is opts->leaf_size (0 or NULL opts -> 32).  The inputs are
 * copied; the caller may free them afterwards.  *out receives the handle.
 * Returns GS_OK, GS_ERR_ARG, GS_ERR_NONFINITE, GS_ERR_WEIGHT, GS_ERR_OOM or
 * GS_ERR_CUDA; synchronises the stream.
 */
int gs_build_tree(const void *pts, int dtype, int64_t n, int D, const float *weights, const gs_opts *opts,
                  void *stream, gs_tree **out);

/* gs_tree_free -- release a tree (waits for the device to be idle); NULL is a no-op. */
void gs_tree_free(gs_tree *tree);

/*
 * gs_sum_trees -- gs_sum on built trees: queries from q, references and
 * weights from r (q == r: monochromatic), same D, dtype and leaf size.
 * h HOST (1 <= nh <= 64), 0 < eps < 1 (the exhaustive sum needs no tree:
 * use gs_sum), out DEVICE M x nh in the query tree's caller order.  opts as
 * for gs_sum except leaf_size, which the trees fix.  Same results and
 * errors as gs_sum on the same data and options.
 */
int gs_sum_trees(const gs_tree *q, const gs_tree *r, const double *h, int nh, double eps, double *out,
                 const gs_opts *opts, void *stream, gs_stats *stats);

/*
 * gs_lscv_trees -- gs_lscv on a built reference tree (gs_build_tree with
 * weights): the LSCV score of each bandwidth h[j] (nh in [1, 32]) from the
 * dual-tree sums at h[j] and sqrt(2) h[j] (the score gs_lscv computes for
 * Section 7's bandwidth selection), reusing the tree across calls -- the
 * building block of a search for the minimising bandwidth.
 *   score, score_err   HOST arrays of nh doubles: scores and the bounds eps
 *                      implies on them (score_err may be NULL)
 * eps in (0, 1).  Returns gs_sum_trees' codes; GS_ERR_ARG also for a tree
 * without weights or with fewer than 2 points.  Synchronises the stream.
 */
int gs_lscv_trees(const gs_tree *t, const double *h, int nh, double eps, double *score, double *score_err,
                  const gs_opts *opts, void *stream, gs_stats *stats);

/* ---- many problems in one call ------------------------------------------
 *
 * One independent Gaussian-sum problem (the arguments of gs_sum). */
typedef struct gs_problem {
    const void  *queries;   /* DEVICE, M x D (may equal refs: monochromatic)        */
    int64_t      M;
    const void  *refs;      /* DEVICE, N x D                                        */
    const float *weights;   /* DEVICE, N                                            */
    int64_t      N;
    int32_t      D;
    int32_t      dtype;     /* GS_F32 / GS_F64                                      */
    const double *h;        /* HOST, nh bandwidths                                  */
    int32_t      nh;
    int32_t      pad;
    double       eps;       /* 0: exhaustive; > 0: dual tree                        */
    double      *out;       /* DEVICE, M x nh (written)                             */
} gs_problem;

/*
 * gs_sum_batched -- nprob independent problems (uneven N, M, D, bandwidths)
 * with the same options.  Each is computed exactly as gs_sum would; up to
 * nworkers problems (0 -> 8) run at once on library-owned streams, largest
 * (M N nh) first.  Work starts after what is already enqueued on `stream`,
 * and `stream` waits for all of it; the call returns when every out is ready.
 *   stats   HOST, nullable: counters summed over problems, ms_phase and
 *           ms_series summed device time, ms_total the batch's wall time
 *   status  HOST, nullable, nprob: each problem's return code
 * Returns GS_OK, or the first failing problem's code (its message names it).
 */
int gs_sum_batched(int nprob, const gs_problem *probs, const gs_opts *opts, int nworkers, void *stream,
                   gs_stats *stats, int32_t *status);

/* ---- learned pair selector (not in the paper) ---------------------------
 *
 * GS_SEL_MLP orders the certified actions of a node pair with a small
 * network instead of Fig. 6's cost rule.  It is consulted only for pairs
 * whose finite-difference test failed, for which at least one series
 * method is certified at some order <= PLIMIT (Lemmas 4-6 against the
 * Theorem 2 budget, the same FP64 test the rule uses) and whose exhaustive
 * work N_Q N_R is at least GS_MLP_MIN_WORK: it scores DH, DL, H2L
 * (each at its smallest certified order) and split / leaf base case, and the
 * highest-scoring certified action is taken (ties: lowest action number).
 * Every choice is therefore one the paper's bounds certify and the eps
 * guarantee is unchanged; only the work done differs.
 *
 * Network: 12 inputs -> 64 -> 64 (ReLU) -> 5 scores (FD, DH, DL, H2L, split /
 * base case), FP32.  Parameters are one array of GS_MLP_NPARAM floats, in this
 * order: mu[12], sc[12] (input normalisation z = (x - mu) * sc), W1[12][64],
 * b1[64], W2[64][64], b2[64], W3[64][5], b3[5] (row-major, input index first).
 * Inference rounds every product and sum to FP32 separately, inputs in
 * ascending order.
 *
 * Features of a pair (Q, R, h), with plog2(x) = e + (m - 1) for x = m 2^e,
 * m in [1, 2) (0 -> -150, +inf -> 128), all FP32:
 *   0 plog2(K upper bound at delta_min)      1 plog2(K lower bound at delta_max)
 *   2 plog2(N_Q)                             3 plog2(N_R)
 *   4 D                                      5 plog2(FD budget ratio
 *                                              (1 + token share) / ((K(dmin) - K(dmax)) W / (2 eps G_lb)))
 *   6 plog2(r_Q / h)                         7 plog2(r_R / h)
 *   8 plog2(W_R / W)                         9 frontier iteration
 *  10 plog2(diameter / h)                   11 PLIMIT
 */
#define GS_MLP_NIN    12
#define GS_MLP_NOUT   5
#define GS_MLP_NPARAM 5341
/* The network is consulted only for pairs with N_Q * N_R >= GS_MLP_MIN_WORK:
 * one inference is about 5.3e3 FP32 multiply-adds, so below that the
 * exhaustive work a decision can save is not worth the inference; such pairs
 * take Fig. 6's choice among the certified orders (as GS_SEL_RULE does). */
#define GS_MLP_MIN_WORK (1 << 18)

/*
 * gs_mlp_forward -- scores of n inputs with the selector's FP32 inference.
 *   params  DEVICE, GS_MLP_NPARAM floats
 *   x       DEVICE, n x 12 floats;  logits  DEVICE, n x 5 floats (written)
 * Returns GS_OK, GS_ERR_ARG or GS_ERR_CUDA; synchronises the stream.
 */
int gs_mlp_forward(const float *params, const float *x, int64_t n, float *logits, void *stream);

/*
 * gs_mlp_loss_grad -- mean weighted softmax cross entropy
 *   L = (1/n) sum_i s_i (logsumexp(o_i) - o_i[y_i])
 * and its gradient with respect to every parameter (0 for mu and sc),
 * computed in FP32 per sample and summed in FP64.
 *   x DEVICE n x 12, y DEVICE n labels in [0, 5), s DEVICE n weights (NULL: 1)
 *   grad DEVICE GS_MLP_NPARAM doubles (overwritten), loss DEVICE 1 double (overwritten)
 * Returns GS_OK, GS_ERR_ARG or GS_ERR_CUDA; synchronises the stream.
 */
int gs_mlp_loss_grad(const float *params, const float *x, const int32_t *y, const float *s, int64_t n,
                     double *grad, double *loss, void *stream);

/*
 * gs_mlp_train -- trains params (DEVICE, updated in place) with Adam
 * (beta1 0.9, beta2 0.999, 1e-8) on minibatches of `batch` samples for
 * `epochs` passes; each epoch visits the samples in the order of the affine
 * permutation i -> (a i + b) mod n drawn from `seed`.  set_norm != 0 first
 * sets mu and sc from the data (mean, 1 / max(std, 1e-3)).  epoch_loss
 * (HOST, epochs doubles, nullable) receives each epoch's mean batch loss.
 * Returns GS_OK, GS_ERR_ARG, GS_ERR_OOM or GS_ERR_CUDA.
 */
int gs_mlp_train(float *params, const float *x, const int32_t *y, const float *s, int64_t n, int epochs,
                 int batch, double lr, uint64_t seed, int set_norm, double *epoch_loss, void *stream);

/*
 * gs_selector_samples -- training samples for the selector from one problem
 * (same arguments as gs_sum, eps > 0; opts->selector is ignored).  The
 * traversal runs with FD-only decisions and logs every pair; a bottom-up
 * pass then gives each pair the modelled cost of its cheapest certified
 * handling (FD-pruned 0; leaf pair: base case or certified series; internal:
 * its children's costs plus u_pair each, or certified series) with
 *   unit_cost (HOST, 6): u_pair per frontier pair, u_base per base-case term,
 *   u_dh, u_dl, u_h2l per FP64 operation slot of each series kernel, u_act
 *   per series action; DH = u_act + N_Q (T_p (D+1) + 3Dp + 30) u_dh,
 *   DL = u_act + N_R (T' (D+1) + 3Dp + 30) u_dl with T' = T_p if T_p <= 32
 *   else 32 ceil(T_p / 32), H2L = u_act + U_p u_h2l with
 *   U_p = 4D + 30 (p = 1), 16D + 30 (p = 2), 2 p T_p + (p(p+1)/2)^2 + 80
 *   (D = 3, p = 3..6), T_p^2 (D+1) + T_p D + 3D(2p-1) + 30 (T_p <= 20,
 *   D(2p-1) <= 32), else 32 (ceil(T_p/32) T_p (D+1) + 40).
 * Every pair the selector would be consulted on (FD test failed, a certified
 * series method, N_Q N_R >= GS_MLP_MIN_WORK) becomes a sample: x (DEVICE, 12
 * floats each), y (DEVICE, the cheapest action 1..4), s (DEVICE, nullable:
 * the pair's regret -- second cheapest minus cheapest certified action --
 * over the mean regret of the problem's samples).  *n_samples (HOST) gets the
 * count; more than cap samples returns GS_ERR_CAPACITY with *n_samples set.
 * model_cost (HOST, 2, nullable): modelled cost of the cheapest policy and of
 * the FD-only policy over the same pairs.
 */
int gs_selector_samples(const void *queries, int64_t M, const void *refs, const float *weights, int64_t N,
                        int D, int dtype, const double *h, int nh, double eps, const gs_opts *opts,
                        const double *unit_cost, float *x, int32_t *y, float *s, int64_t cap,
                        int64_t *n_samples, double *model_cost, void *stream);

/*
 * gs_debug_fail_alloc -- fault injection for tests: after n more device
 * scratch allocations (of any call, any thread) the next one fails as if the
 * device were out of memory, once; n < 0 disarms.  The call that meets the
 * failure returns GS_ERR_OOM and later calls work normally (the tree build,
 * the traversal buffers, the outputs and every phase's scratch are freed on
 * that path, so the library's pool gets all of it back).
 */
void gs_debug_fail_alloc(long long n);

/*
 * gs_probe_rates -- measures this device's throughput, in lanes per SM per
 * SM clock cycle, of the two instructions the base case is built from: MUFU
 * ex2.approx.ftz.f32 and FP32 FFMA.  A short kernel with independent chains
 * on every SM is timed with the SM cycle counter, so the figures do not depend
 * on the clock the GPU happens to run at.  Used for roofline reporting.
 *   ex2_per_sm_clk, ffma_per_sm_clk   HOST doubles, written on success
 * Returns GS_OK, GS_ERR_ARG (NULL pointer) or GS_ERR_CUDA.
 */
int gs_probe_rates(double *ex2_per_sm_clk, double *ffma_per_sm_clk, void *stream);

/*
 * gs_tc_dot_check -- diagnostic of the tensor-core cross term of the base case
 * (9 <= D <= 16): U (HOST, 128 x 16 int32) and V (HOST, N x 16 int32), every
 * entry in [-2^29, 2^29], are split into three base-2^10 digits each
 * (U = U2 2^20 + U1 2^10 + U0, U0 and U1 in [-512, 511]) and the tensor
 * cores form, in FP32 accumulators,
 *     P[0] = U2 V2^T,  P[1] = U2 V1^T + U1 V2^T,  P[2] = U2 V0^T + U1 V1^T + U0 V2^T
 * (128 x N each), written to P (HOST, 3 x 128 x N floats, row-major).  Each
 * entry is an integer below 2^24 in magnitude, so the result is exact; the
 * check compares it with integer arithmetic.  N is a multiple of 16 in
 * [16, 128].  Returns GS_OK, GS_ERR_ARG, GS_ERR_TIMEOUT (the completion wait
 * gave up) or GS_ERR_CUDA; synchronises the stream.
 */
int gs_tc_dot_check(const int32_t *U, const int32_t *V, int N, float *P, void *stream);

/*
 * gs_trim_memory -- device scratch of every call comes from a stream-ordered
 * memory pool that the library owns, one per device.  Memory a call frees
 * stays in that pool for later calls (a traversal synchronises once per
 * frontier iteration, and a pool that gave memory back at each
 * synchronisation would map its work lists afresh every time).  This call
 * waits for the current device and returns to the CUDA driver all but keep_bytes
 * of that device's pool.  Memory held by built trees (gs_tree) is not
 * affected.
 * Returns GS_OK, or GS_ERR_CUDA (message in gs_last_error).
 */
int gs_trim_memory(size_t keep_bytes);

/*
 * gs_pool_bytes -- bytes the library's pool of the current device holds
 * from the CUDA driver (reserved) and bytes of it in use, written to the HOST
 * pointers (either may be NULL).  Returns GS_OK or GS_ERR_CUDA.
 */
int gs_pool_bytes(uint64_t *reserved, uint64_t *used);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
