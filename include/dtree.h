/*
 * dtree.h -- C ABI of the GB300 dual-tree exact k-nearest-neighbour library.
 *
 * The library instantiates the dual-tree meta-algorithm of Curtin et al.,
 * "Tree-Independent Dual-Tree Algorithms" (ICML 2013, Section 2) for exact
 * k-nearest-neighbour search (Section 5): a kd-tree space tree (Definition 1,
 * with the kd-tree bounds of Section 3), a pruning dual-tree traversal (the
 * pruning dual-tree traversal definition of Section 4), the kNN BaseCase
 * (Algorithm 2) and the kNN Score (Algorithm 3) with the bound B(N_q) of
 * Section 5.  The same trees serve three more instances the paper derives:
 * k-furthest neighbours (dtree_kfn, the extension after Algorithm 4), range
 * search (dtree_range_count / dtree_range_fill, Section 6) and the Euclidean
 * minimum spanning tree by Boruvka rounds (dtree_emst, Section 7).
 *
 * Conventions for every entry point:
 *   - Point arrays are row-major n x d float32.  Pointers marked "device" must
 *     be CUDA device (or managed) memory on the current device; pointers
 *     marked "host" are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it.
 *   - Every function returns a dtree_status (0 = success, negative = error);
 *     no C++ exception crosses the ABI.  On error no output is valid.
 *   - Handles are not thread-safe: calls that share a handle must not run
 *     concurrently.
 */
#ifndef DTREE_H
#define DTREE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum dtree_status {
    DTREE_OK = 0,
    DTREE_ERR_INVALID_ARG = -1,  /* null pointer, n <= 0, d outside [1, 64], d mismatch,
                                    leaf_size outside [1, 1024], unknown option value */
    DTREE_ERR_INVALID_K = -2,    /* k <= 0, or k >= m (bichromatic: the problem statement
                                    of Section 5 requires 0 < k < m), or k > m - 1
                                    (monochromatic, the query itself is excluded) */
    DTREE_ERR_CUDA = -3,         /* a CUDA runtime call or kernel launch failed */
    DTREE_ERR_OOM = -4,          /* device allocation failed */
    DTREE_ERR_TIMEOUT = -5,      /* a bounded device-side wait gave up (the kernel
                                    recorded it and returned; the context stays usable) */
    DTREE_ERR_NOT_TRAINED = -6,  /* a learned proposal was requested without a model */
    DTREE_ERR_UNSUPPORTED = -7,  /* valid request this build/device cannot serve
                                    (e.g. tensor-core precision on a non-sm_103 device) */
    DTREE_ERR_TOO_LARGE = -8,    /* the problem exceeds the fixed scratch of
                                    dtree_knn_noalloc (see its limits) */
    DTREE_ERR_IO = -9            /* a model file could not be written, read, or is not a
                                    well-formed model file */
} dtree_status;

/* Distance arithmetic of the BaseCase tiles.  Whatever the choice, results
 * are exact: candidates near each query's k-th distance are re-ranked in
 * float64, and a query whose candidate band overflows is recomputed in
 * float64 (see dtree_knn). */
typedef enum dtree_precision {
    DTREE_PREC_FP32 = 0,   /* CUDA-core float32 differences and squares */
    DTREE_PREC_TF32 = 1,   /* tensor cores (tcgen05), TF32 inputs, FP32 accumulate */
    DTREE_PREC_BF16 = 2    /* tensor cores (tcgen05), BF16 inputs, FP32 accumulate: each
                              centred coordinate is carried as a hi + lo pair of BF16
                              values (three BF16 products per term, operand error about
                              2^-16) */
} dtree_precision;

/* The lower bound d_min(N_q, N_r) that Score (Algorithm 3) compares with
 * B(N_q), and that the search's other pruning and ordering steps use for a
 * point against a node.  The method is the same for any bound that is a true
 * lower bound on the distance between the nodes' points (the paper's
 * tree-independence: Section 3's space tree asks only for d_min, rho and
 * lambda); results are identical for all three, only the pruning differs. */
typedef enum dtree_bound {
    DTREE_BOUND_BOX = 0,   /* the nodes' bounding hyperrectangles (a kd-tree) */
    DTREE_BOUND_BALL = 1,  /* balls around the box centres with radius lambda, the largest
                              distance from the centre to a point of the node (a ball tree
                              over the same median splits): |C_q - C_r| - lambda_q - lambda_r */
    DTREE_BOUND_BOTH = 2   /* the larger of the two (both are lower bounds) */
} dtree_bound;

/* Options; zero-initialise and set what you need (0 = default). */
typedef struct dtree_opts {
    int32_t leaf_size;     /* dtree_build: max points per kd-tree leaf, 1..1024 (default 32) */
    int32_t precision;     /* dtree_knn: dtree_precision (default FP32) */
    int32_t query_block;   /* dtree_knn: max queries per query block (the query-tree node that
                              is the traversal's unit), 16..512 (default 128); a block of
                              more than 128 queries is processed as chunks of 128 that
                              share its candidate leaves */
    int32_t seed_points;   /* dtree_knn: min reference points of the seed subtree evaluated
                              before the traversal (default 64) */
    int32_t proposal;      /* dtree_knn: M > 0 evaluates each query block's top-M cells of the
                              proposal attached to the reference tree (see
                              dtree_attach_proposal) in the seed pass, M <= 8; 0: none */
    int32_t spin_budget;   /* dtree_knn: polls of a device-side wait before it gives up
                              with DTREE_ERR_TIMEOUT (default 1 << 20, about a second) */
    int32_t cap_leaves;    /* dtree_knn: reference leaves each query's best-first cap search
                              may evaluate before the traversal, 1..17 (default 8); -1
                              skips the cap pass.  The cap only tightens bounds: results
                              are the same whatever its value */
    int32_t bound;         /* dtree_knn: dtree_bound of the node-pair lower bound (default
                              DTREE_BOUND_BOX) */
    int32_t reserved[8];   /* must be zero */
} dtree_opts;

/* Counters of one dtree_knn call (all zero if not requested). */
typedef struct dtree_stats {
    int64_t node_pairs_scored;   /* Score() evaluations of the traversal */
    int64_t node_pairs_pruned;   /* pairs whose d_min exceeded B(N_q) */
    int64_t leaf_pairs_emitted;  /* (query block, reference leaf) pairs that survived */
    int64_t leaf_pairs_skipped;  /* emitted pairs pruned later by the tightened B */
    int64_t leaf_pairs_evaluated;/* pairs whose BaseCase tile ran (seed pairs included) */
    int64_t point_pairs;         /* BaseCase(p_q, p_r) evaluations of the main pass */
    int64_t rerank_candidates;   /* candidates re-ranked in float64 */
    int64_t fallback_queries;    /* queries whose error band overflowed the candidate list
                                    and were recomputed over their own candidate leaves
                                    (float32 keys, float64 re-rank of the band) */
    int64_t query_blocks;        /* work units */
    int64_t kernel_launches;     /* kernels this call launched */
    /* device time of each phase in nanoseconds, from CUDA events recorded on
       `stream` around the phase (only filled when stats are requested) */
    int64_t ns_seed;             /* seed selection + seed BaseCase */
    int64_t ns_traverse;         /* bounds + dual-tree traversal + candidate lists */
    int64_t ns_basecase;         /* main BaseCase pass (tiles, re-rank, output) */
    int64_t ns_fallback;         /* recomputation of overflowed queries */
    int64_t fallback64_queries;  /* of those, queries whose float32 band overflowed as
                                    well, recomputed with float64 keys throughout */
    int64_t seed_point_pairs;    /* point pairs the seed pass evaluated (not in point_pairs) */
} dtree_stats;

typedef struct dtree dtree_t;

/*
 * dtree_build -- build a kd-tree (a space tree, Definition 1) on the device.
 *
 *   pts     device, n x d float32 row-major; read during the call only (the
 *           tree keeps its own permuted copy, so the caller may free `pts`
 *           once the call returns).
 *   n       number of points, 1 <= n < 2^31.
 *   d       dimension, 1 <= d <= 64.
 *   opts    nullable; uses leaf_size.
 *   stream  cudaStream_t or NULL.
 *   out     receives a library-owned handle; free it with dtree_free.
 *
 * The tree is balanced: every split puts floor(n/2) points on the left (the
 * smallest along the widest dimension of the node's tight bounding box, the
 * convex set of Definition 1), and all leaves sit at one depth, the smallest
 * at which every leaf holds at most leaf_size points.  Per node it stores the
 * box, the box centre (the centroid of Section 3) and an upper bound on the
 * maximum descendant distance lambda (Section 3).  The call returns after the
 * tree is complete on `stream`.
 */
int dtree_build(const float* pts, int64_t n, int32_t d, const dtree_opts* opts, void* stream,
                dtree_t** out);

/*
 * dtree_knn -- exact k nearest neighbours of every point of `query` among the
 * points of `ref` (problem statement of Section 5).
 *
 *   query     tree of the queries, or NULL / the same handle as `ref` for the
 *             monochromatic case, where a point never returns itself (the
 *             footnote to Algorithm 2; exclusion is by index, so duplicates at
 *             distance 0 are valid neighbours).
 *   ref       tree of the references (m points).
 *   k         0 < k < m (bichromatic), 0 < k <= m - 1 (monochromatic), and
 *             k <= 63 (DTREE_ERR_UNSUPPORTED beyond).
 *   out_idx   device, n_q x k int64, row i = the query's row in the array it
 *             was built from; entries are row indices of the reference array,
 *             ascending by (distance, index) -- ties go to the lower index.
 *   out_dist  device, n_q x k float32, Euclidean distances (not squared),
 *             the float64 distance rounded to float32.
 *   opts      nullable; uses precision, query_block, seed_points, proposal,
 *             spin_budget.
 *   stream    cudaStream_t or NULL.
 *   stats     nullable; receives the call's counters.
 *
 * The call enqueues its kernels on `stream`, blocks the calling thread until
 * they finish (it reads device-side sizes between phases) and returns the
 * device-side status, so the outputs are ready on return.  Scratch memory
 * comes from the device's stream-ordered pool.  With a tensor-core
 * precision, the first search against a reference tree also converts its
 * points once into the MMA's operand rows (centred on the root box's centre,
 * rows x (32 to 288) bytes by dimension), which the tree keeps until
 * dtree_free.
 */
int dtree_knn(const dtree_t* query, const dtree_t* ref, int32_t k, int64_t* out_idx,
              float* out_dist, const dtree_opts* opts, void* stream, dtree_stats* stats);

/*
 * dtree_kfn -- exact k-furthest-neighbour search: for every query the k
 * reference points at the LARGEST Euclidean distance (Section 5, the
 * paragraph on k-furthest neighbour search after Algorithm 4: the kNN rules
 * inverted -- lists by descending distance, a candidate kept when it is
 * farther than the k-th, a node pruned when its farthest possible point is
 * nearer than the k-th furthest so far).
 *   query     query tree, or NULL (or == ref) for the monochromatic problem,
 *             where a point never returns itself (by index)
 *   ref       reference tree
 *   k         1 <= k <= 63, and k < n_ref (k <= n_ref - 1 monochromatic)
 *   out_idx   device, n_q x k int64, row-major in the caller's query order:
 *             row indices into the caller's reference array, descending by
 *             (distance), ties by the lower index
 *   out_dist  device, n_q x k float32: the Euclidean distance, computed in
 *             float64 and rounded once
 *   opts      nullable; precision must be DTREE_PREC_FP32 (float32 keys with a
 *             float64 re-rank, float64 keys for queries whose error band
 *             overflows: results are exact either way); other fields ignored
 *   stream    cudaStream_t or NULL
 *   stats     nullable; point_pairs (point distances evaluated),
 *             leaf_pairs_evaluated (leaves visited), node_pairs_pruned,
 *             fallback_queries, kernel_launches, ns_basecase
 * Status: DTREE_ERR_INVALID_ARG (null tree or outputs, dimension mismatch,
 * trees on another device, non-zero reserved options), DTREE_ERR_INVALID_K,
 * DTREE_ERR_UNSUPPORTED (k > 63, another precision, a reference tree deeper
 * than 30 levels), or a CUDA error.  Waits for the result.  Scratch comes
 * from the device's stream-ordered pool.
 */
int dtree_kfn(const dtree_t* query, const dtree_t* ref, int32_t k, int64_t* out_idx,
              float* out_dist, const dtree_opts* opts, void* stream, dtree_stats* stats);

/*
 * dtree_range_count / dtree_range_fill -- exact range search (Section 6): for
 * every query all reference points with d_lo <= ||q - r|| <= d_hi, both ends
 * inclusive, decided on the float64 distance (the correctly rounded square
 * root of the float64 sum of squared float32 differences); a monochromatic
 * query (query NULL or == ref) never returns itself.  Two calls, count then
 * fill:
 *   dtree_range_count writes offsets[0..n_q] (device, int64, n_q + 1):
 *     query row i's neighbours will occupy [offsets[i], offsets[i + 1]) of
 *     the outputs (rows in the caller's query order), and *total (host) gets
 *     offsets[n_q]; stats (nullable): point_pairs (distances evaluated),
 *     leaf_pairs_evaluated, node_pairs_pruned, rerank_candidates (points
 *     decided in float64), kernel_launches, ns_basecase.
 *   dtree_range_fill writes each query's segment: out_idx (device, int64,
 *     *total) the caller's reference row indices, out_dist (device, float32)
 *     the distances rounded once from float64.  Within a segment the order is
 *     the search's visit order (the problem's lists are sets); it is the same
 *     from call to call.
 * The same trees and range must be passed to both.  opts: nullable,
 * precision must be DTREE_PREC_FP32.  Status: DTREE_ERR_INVALID_ARG (null
 * tree or buffer, dimension mismatch, d_lo < 0, d_hi < d_lo, NaN, trees on
 * another device), DTREE_ERR_UNSUPPORTED (another precision, a reference tree
 * deeper than 30 levels), or a CUDA error.  Both wait for the result.
 */
int dtree_range_count(const dtree_t* query, const dtree_t* ref, double d_lo, double d_hi,
                      int64_t* offsets, int64_t* total, const dtree_opts* opts, void* stream,
                      dtree_stats* stats);
int dtree_range_fill(const dtree_t* query, const dtree_t* ref, double d_lo, double d_hi,
                     const int64_t* offsets, int64_t* out_idx, float* out_dist,
                     const dtree_opts* opts, void* stream);

/*
 * dtree_emst -- the Euclidean minimum spanning tree of a tree's points by
 * Boruvka rounds (Section 7): each round, every component's shortest edge to
 * a point outside it (a pruning search per point, float64 distances), then
 * the components joined by those edges merge.  Edges compare by float64
 * squared length, equal lengths by (lower index, higher index), so the tree
 * is unique.
 *   tree      the points (any dimension the library builds)
 *   out_edges device, (n - 1) x 2 int64: (lower, higher) caller row indices
 *   out_dist  device, n - 1 float32: edge lengths, rounded once from float64
 *   opts      nullable; precision must be DTREE_PREC_FP32
 *   stats     nullable; point_pairs (distances), leaf_pairs_evaluated,
 *             kernel_launches, ns_basecase
 * Edges come round by round, and within a round by component; the order is
 * the same from call to call.  Status: DTREE_ERR_INVALID_ARG (null tree or
 * outputs with n > 1, a tree on another device), DTREE_ERR_UNSUPPORTED
 * (another precision, a tree deeper than 30 levels), or a CUDA error.  One
 * point gives no edge.  Waits for the result.
 */
int dtree_emst(const dtree_t* tree, int64_t* out_edges, float* out_dist, const dtree_opts* opts,
               void* stream, dtree_stats* stats);

/* One problem of a batch: the arguments of one dtree_knn call. */
typedef struct dtree_problem {
    const dtree_t* query;   /* NULL (or == ref): monochromatic */
    const dtree_t* ref;
    int32_t k;
    int32_t query_block;    /* queries per block of this problem, 16..512, or 0 for
                               opts->query_block */
    int64_t* out_idx;       /* device, n_q x k */
    float* out_dist;        /* device, n_q x k */
} dtree_problem;

/*
 * dtree_knn_batch -- many independent kNN problems (Section 5's problem, as in
 * dtree_knn) in one call.  Problems whose points share a width bucket
 * (d <= 4, 8, 16, 32, 64) run together: each phase of the search (seed,
 * bounds, traversal levels, BaseCase tiles, re-rank, fallback) is one launch
 * over all their blocks, pairs and queries, so a batch of small problems
 * fills the GPU as one large problem would.  The lists of a group are sized
 * for its largest k.
 *   nprob     number of problems (0 returns DTREE_OK)
 *   probs     host array of nprob problems; their trees must live on the
 *             current device and each problem's outputs must not overlap
 *             another's
 *   opts      as in dtree_knn, shared by every problem
 *   stats     nullable; counters summed over the batch
 * Results are exactly those of one dtree_knn call per problem.  Status: the
 * first failing problem's argument check (nothing is launched), or the
 * search's status.  Waits for the result.  (The paper runs one problem at
 * a time; batching is this library's addition.)
 */
int dtree_knn_batch(int32_t nprob, const dtree_problem* probs, const dtree_opts* opts,
                    void* stream, dtree_stats* stats);

/*
 * dtree_knn_noalloc -- dtree_knn with no device allocation: the same search,
 * arguments, results and status codes, but every scratch buffer the call
 * needs is carved from one file-scope static device array of
 * DTREE_NOALLOC_SCRATCH_BYTES bytes instead of the stream-ordered pool.  The
 * paper has no counterpart; this serves callers that must not allocate (a
 * serving loop with a fixed memory budget, or a caller whose allocator must
 * not be touched).  The call makes no cudaMalloc/cudaFree or other
 * allocating call; the trees and the outputs are the caller's.
 *
 * Limits (checked before any work; beyond them it returns
 * DTREE_ERR_TOO_LARGE):
 *   - at most DTREE_NOALLOC_MAX_QUERIES queries (the query tree's points, or
 *     the reference tree's points in the monochromatic problem);
 *   - the traversal's candidate pairs must fit what is left of the array
 *     after the per-query buffers (checked on the device, before the pairs
 *     are used; the call then returns DTREE_ERR_TOO_LARGE).
 * `stats` is not offered (the phase timers would create CUDA events).
 *
 * The array's address on the current device is looked up on every call
 * (cudaGetSymbolAddress, with that device current; it allocates nothing), so
 * a device reset cannot leave a stale address behind.  The trees must live on
 * the current device (else DTREE_ERR_INVALID_ARG).  With a tensor-core
 * precision, a reference tree whose operand rows were not made by an earlier
 * dtree_knn call gets them in the array for this call only (they count
 * against its size).
 *
 * The array keeps whatever the previous call left in it; every buffer whose
 * contents must start at zero (work counters, per-block pair counts,
 * statistics, the error word) is cleared on `stream` by the call itself.
 *
 * Concurrency: there is one array per device.  Calls that overlap in time
 * on one device (different streams, or different host threads) share it and
 * race; callers must serialise them.
 */
#define DTREE_NOALLOC_SCRATCH_BYTES (128u << 20)
#define DTREE_NOALLOC_MAX_QUERIES 65536
int dtree_knn_noalloc(const dtree_t* query, const dtree_t* ref, int32_t k, int64_t* out_idx,
                      float* out_dist, const dtree_opts* opts, void* stream);

/*
 * Learned leaf proposal (no counterpart in the paper's method; it only changes
 * which leaves are evaluated first, never the result).  A small MLP
 * (d -> 256 -> 256 -> C, FP16 tensor-core GEMMs, FP32 master weights, Adam)
 * maps a point to the C cells of the reference tree (its subtrees at the
 * seed level, the subtrees the seed pass evaluates) most likely to hold the
 * point's nearest neighbours.  With opts->proposal = 1, dtree_knn evaluates
 * each query block's top-M proposed cells together with the greedy seed
 * subtree before the traversal, so B(N_q) starts tight; the traversal still
 * visits every leaf the bound does not prune, so the result is exact whatever
 * the network predicts.
 */
typedef struct dtree_model dtree_model;

typedef struct dtree_train_opts {
    int32_t epochs;           /* passes over the training examples (default 20) */
    int32_t batch;            /* examples per Adam step, <= 4096 (default 256) */
    float lr;                 /* Adam step size (default 1e-3) */
    int32_t example_queries;  /* queries per example: the training tree's nodes at the level
                                 holding about this many (default 16) */
    int32_t seed_points;      /* cells: the reference subtrees at the level whose subtrees hold
                                 >= this many points (default 512, the search's seed level) */
    uint32_t seed;            /* initialisation and shuffling seed (0 = default) */
    float* loss_out;          /* optional host array: mean training loss of each epoch */
    int32_t loss_out_len;
    int32_t precision;        /* dtree_precision of the search that makes the labels (default
                                 FP32); the labels are the exact neighbours at every precision */
    int32_t reserved[7];      /* must be zero */
} dtree_train_opts;

/*
 * dtree_proposal_train -- train a proposal for `ref` on the method's own
 * answers: dtree_knn(train, ref, k) gives each training query's neighbours;
 * each node of the training tree holding about example_queries queries is one
 * example (input: its box centre, standardised with the reference points'
 * mean and spread; target: the distribution of its queries' neighbours over
 * the cells; loss: softmax cross-entropy).  `train` must be a different tree
 * from `ref`, of the same dimension.  *out is library-owned (dtree_model_free).
 * Returns DTREE_ERR_UNSUPPORTED off sm_103 or when the reference tree has a
 * single cell.  Waits for the result.
 */
int dtree_proposal_train(const dtree_t* ref, const dtree_t* train, int32_t k,
                         const dtree_train_opts* opts, void* stream, dtree_model** out);
void dtree_model_free(dtree_model* model);

/*
 * dtree_model_save / dtree_model_load -- keep a trained proposal across
 * processes (no counterpart in the paper).  The file (host path) holds the
 * network's shape, the input standardisation, the FP32 weights and a
 * fingerprint of the reference tree the model was trained for (its size,
 * dimension, height and the bounding boxes of its cells), closed by a
 * checksum.  Loading checks the file before it touches the device, then
 * compares the fingerprint with `ref` (a tree built from the same points with
 * the same leaf size matches) and returns a new library-owned model
 * (dtree_model_free) whose searches propose exactly the cells the saved one
 * did.  Status: DTREE_ERR_INVALID_ARG (null arguments, or a model for another
 * tree: dimension, depth or fingerprint differ), DTREE_ERR_IO (the file cannot
 * be written or read, is truncated, or fails the format or checksum checks),
 * DTREE_ERR_OOM, or a CUDA error.  Both wait for their copies on `stream`.
 */
int dtree_model_save(const dtree_model* model, const char* path, void* stream);
int dtree_model_load(const char* path, const dtree_t* ref, void* stream, dtree_model** out);
/* Number of cells (output classes) of a model; -1 for NULL. */
int dtree_model_classes(const dtree_model* model);
/*
 * dtree_attach_proposal -- use `model` (NULL detaches) for searches against
 * `ref` that set opts->proposal.  The model must outlive its use and have
 * been trained for a tree of the same dimension.
 */
int dtree_attach_proposal(dtree_t* ref, const dtree_model* model);

/*
 * dtree_mlp_loss_grad -- one forward and backward pass of the proposal's
 * network with the caller's parameters, for checking the kernels:
 *   params  device FP32: W1 [256 x d], b1 [256], W2 [256 x 256], b2 [256],
 *           W3 [C x 256], b3 [C] (row-major, W_l maps layer l-1 to layer l)
 *   X       device FP32 [n x d] inputs (used as given, not standardised)
 *   T       device FP32 [n x C] target distributions (rows sum to 1)
 *   loss    host: mean over rows of -sum_c T log softmax(Z)
 *   grads   device FP32, the gradients of `loss`, shaped like params
 * GEMMs run in FP16 on the tensor cores with FP32 accumulation.  n <= 4096.
 */
int dtree_mlp_loss_grad(int32_t d, int32_t C, const float* const* params, const float* X,
                        const float* T, int32_t n, float* loss, float* const* grads, void* stream);

/* dtree_free -- release every device allocation of the handle.  NULL-safe.
 * Must not be called while work that uses the handle is still in flight. */
void dtree_free(dtree_t* tree);

/* Number of points / dimension / depth (leaves sit at this depth) / leaf
 * count of a tree; -1 for NULL. */
int64_t dtree_size(const dtree_t* tree);
int32_t dtree_dim(const dtree_t* tree);
int32_t dtree_depth(const dtree_t* tree);
int64_t dtree_leaf_count(const dtree_t* tree);

/*
 * dtree_export -- copy the tree's layout to device buffers supplied by the
 * caller (any of them may be NULL):
 *   perm    n int32: position in tree order -> row of the build input
 *   box     nodes x 2 x d float32: lo[0..d) then hi[0..d) per node
 *   lambda  nodes float32: the stored upper bound on lambda per node
 *   begin   nodes int32 / count nodes int32: each node's range in tree order
 * Nodes are numbered in heap order: node i has children 2i+1 and 2i+2,
 * nodes = 2^(depth+1) - 1.  Enqueued on `stream` and waited for.
 */
int dtree_export(const dtree_t* tree, int32_t* perm, float* box, float* lambda, int32_t* begin,
                 int32_t* count, void* stream);

/* ---------------------------------------------------------------------------
 * Diagnostics.  No counterpart in the paper: hooks for the tests and for
 * profiling the hardware path.  They do not change any result.
 * ------------------------------------------------------------------------- */

/*
 * dtree_debug_mma -- diagnostic: one 128 x 128 tensor-core tile through the
 * operand layout, descriptors and TMEM read-out the BaseCase tiles use.
 *   A, B  device, 128 x K float32 row-major (K <= 64), rounded to
 *         `precision` (DTREE_PREC_BF16 or DTREE_PREC_TF32) on the way in
 *   out   device, 128 x 128 float32: out[i][j] = sum_k A~[i][k] * B~[j][k]
 *         accumulated in FP32 by tcgen05.mma
 * Returns DTREE_ERR_UNSUPPORTED on a device other than sm_103, and
 * DTREE_ERR_TIMEOUT if the completion wait gave up.  Waits for the result.
 * (No counterpart in the paper: this checks the hardware path only.)
 */
int dtree_debug_mma(const float* A, const float* B, int32_t K, int32_t precision, float* out,
                    void* stream);

/*
 * dtree_debug_tmem_min -- diagnostic: dtree_debug_mma's tile, plus the
 * minima the BaseCase epilogue takes from the loads themselves
 * (tcgen05.ld.red ... .min.f32): min32 (device, 128 x 4 float32) holds row
 * i's minimum over columns [32c, 32c + 32) from a 32-column read, min64
 * (device, 128 x 2) over [64c, 64c + 64) from a 64-column read.  Each must
 * equal the float32 minimum of the same columns of `out`.  Status as
 * dtree_debug_mma, and DTREE_ERR_INVALID_ARG for a null min32 or min64.
 * (No counterpart in the paper: this checks the hardware path only.)
 */
int dtree_debug_tmem_min(const float* A, const float* B, int32_t K, int32_t precision, float* out,
                         float* min32, float* min64, void* stream);

/*
 * dtree_debug_tc_timers -- diagnostic: while `counters` (device, 64 zeroed
 * uint64, or NULL to stop) is set, the tensor-core BaseCase pass ORs into
 * counter TT_FAIL_SITES (the binding's TC_TIMERS order) a bit for each kind
 * of bounded wait that gave up.  A library built with DTREE_TC_TIMERS=1
 * also adds per-role clock64 cycle counts and event counts (window
 * preparation, slot waits and filling, MMA-issue waits, epilogue waits and
 * work, list insertions, tiles, items, TMEM reads); the default build leaves
 * them at zero, because their code slows the pass even when detached.
 * Process-wide; not thread-safe.  (No counterpart in the paper: a
 * performance probe.)
 */
int dtree_debug_tc_timers(unsigned long long* counters);

/*
 * dtree_debug_tc_stall -- diagnostic of the bounded waits: while `on` is
 * non-zero, the tensor-core BaseCase pass makes every block's planner wait,
 * before it ends the block, on a barrier that nothing completes.  That wait
 * gives up after opts->spin_budget polls, the pass abandons its work items,
 * lets its own copies and MMAs finish, releases its tensor memory, and the
 * call returns DTREE_ERR_TIMEOUT with the context still usable (its outputs
 * are not valid).  Process-wide; not thread-safe.
 */
int dtree_debug_tc_stall(int32_t on);

/* Static description of a status code. */
const char* dtree_error_string(int status);

/* Kernels launched by this library since the process started (all threads). */
int64_t dtree_launch_count(void);

/* Device allocations the library has made so far (tree storage and per-call
 * scratch), for tests. */
int64_t dtree_alloc_count(void);

#ifdef __cplusplus
}
#endif

#endif /* DTREE_H */
