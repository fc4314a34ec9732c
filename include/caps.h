/*
 * caps.h -- C ABI of the GB300 (sm_103a) CAPS filtered-search library.
 *
 * CAPS = Constrained Approximate Partitioned Search (arXiv 2308.15014).
 * The data model is the paper's Def. 1-2: a dataset of N pairs (x_i, a_i),
 * x_i in R^d, a_i an attribute vector; a query (q, b) asks for the k nearest
 * x_i among the points whose attributes satisfy the AND-filter C(a_i, b).
 * The index is the paper's two-level partition (Alg. 1): a first-level
 * partition function f(.) (k-means here, Sec. 5.2) and, inside each of the B
 * partitions, an attribute-frequency tree (AFT) of height h that splits the
 * partition into h+1 disjoint sub-partitions laid out contiguously.  A query
 * (Alg. 2) probes the m best partitions, selects the sub-partitions that can
 * hold valid points, filters them and keeps the k best distances.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Pointers.  Every array argument may point to host memory or to device
 * memory of the current CUDA device (the library tells them apart with
 * cudaPointerGetAttributes).  Host inputs are copied to the device inside the
 * call; when an output is in host memory the call synchronises `stream` and
 * the output is complete on return.  With device inputs and outputs the call
 * only enqueues work on `stream` and returns.
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).
 * Ownership.  The caller owns every array it passes; the library never keeps
 * a caller pointer past the call.  A caps_index owns all of its device
 * memory and releases it in caps_free.
 * Errors.  Every int-returning call returns CAPS_OK (0) or one of the codes
 * below and never aborts; caps_last_error() returns a message for the last
 * failure on the calling thread.
 * Layouts.  Row-major, 0-based.  float = IEEE fp32.
 * Concurrency.  A caps_index keeps per-index search workspace: searches on
 * one index must not overlap (serialise them on one stream); distinct
 * indexes are independent.
 */
#ifndef CAPS_H_
#define CAPS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CAPS_OK 0
#define CAPS_EINVAL 1   /* bad argument (shape, range, unsupported option) */
#define CAPS_ENOMEM 2   /* device or host allocation failed */
#define CAPS_ECUDA 3    /* a CUDA runtime call or kernel launch failed */
#define CAPS_ETIMEOUT 4 /* a bounded device-side wait expired */

typedef struct caps_index caps_index;

typedef enum { CAPS_L2 = 0, CAPS_IP = 1 } caps_metric;
typedef enum { CAPS_PART_KMEANS = 0, CAPS_PART_MLP = 1 } caps_partitioner;
typedef enum {
  CAPS_FP32 = 0,
  CAPS_BF16 = 1,
  CAPS_FP8E4M3 = 2,
  CAPS_FP32_SPLIT = 3
} caps_precision;

/*
 * Attribute vectors (Def. 1, "attribute model") -- exactly one of the two
 * forms is used:
 *   dense:  L > 0, dense = [N*L] int32, dense[i*L+f] in [0, vocab[f]);
 *           vocab = [L] int32 (values per field).  For a query constraint
 *           array the same layout holds with -1 meaning "field f is
 *           unconstrained" (variable constraints, Sec. 6.1).
 *   sparse: L = 0, dense = NULL; point i carries the label set
 *           sp_labels[sp_offsets[i] .. sp_offsets[i+1]) (int32 in
 *           [0, sp_vocab), sorted ascending, no repeats), sp_offsets = [N+1]
 *           int64.  For a query the set lists the REQUIRED labels (any
 *           order; an empty set constrains nothing, a label outside
 *           [0, sp_vocab) matches no point); the filter holds when every
 *           required label is present.  sp_vocab may be 0 for queries.
 *           On the GPU each row also carries a 64-bit signature of its
 *           labels: the scans test it first and run the exact subset test
 *           on the row's sorted labels only for the pairs that pass it.
 *           The learned partitioner, query plans and the no-allocation
 *           query serve dense attributes only (CAPS_EINVAL).
 */
typedef struct {
  int32_t L;
  const int32_t* dense;
  const int32_t* vocab;
  const int64_t* sp_offsets;
  const int32_t* sp_labels;
  int32_t sp_vocab;
} caps_attrs;

/*
 * Build parameters (Alg. 1 inputs).
 *   B            first-level partitions (k-means clusters), 1 <= B <= N.
 *   h            AFT height, 0 <= h <= 63: each partition is split into h+1
 *                sub-partitions (Alg. 1; Sec. 6.1 ablation on h+1).
 *   kmeans_iters Lloyd iterations (Sec. 5.2), >= 0.
 *   seed         used only when init_idx is NULL: the B seed points are then
 *                drawn without replacement by Floyd's method driven by
 *                SplitMix64(seed).
 *   metric       CAPS_L2 (squared Euclidean, smaller is better) or CAPS_IP
 *                (inner product, larger is better; k-means then normalises
 *                each centroid to unit length).
 *   part         CAPS_PART_KMEANS: f(x) = nearest centroid (Sec. 5.2).
 *                CAPS_PART_MLP: learned partitioner (Sec. 5.2, BLISS-style):
 *                k-means first, then labels = normalised histogram of the
 *                k-means partitions of each training point's mlp_label_k
 *                exact filtered neighbours (the filter being the point's own
 *                attributes on a subset of fields), an MLP
 *                d -> mlp_hidden -> B (ReLU) trained with Adam on the mean
 *                softmax cross-entropy, and f(x) = argmax of its logits
 *                (ties to the lower partition); queries probe the m largest
 *                logits.
 *   prec         CAPS_FP32: every distance in fp32.
 *                CAPS_BF16: the index also keeps a bf16 copy of the rows;
 *                searches score all selected rows with bf16 tensor-core
 *                tiles (fp32 accumulation; L2 candidates ranked by
 *                |x|^2 - 2 q.x, the query's own |q|^2 being common to all its
 *                keys) and re-score the best rerank_factor * k candidates of
 *                each query exactly in fp32 before keeping k.  Needs d % 8 == 0 and
 *                64 <= d <= 128; searches with k > 32 use the fp32 scan instead.
 *                CAPS_FP8E4M3: as CAPS_BF16 with e4m3 rows and queries, each
 *                row and query scaled by s = max |x| / 448 (e4m3 value =
 *                x / s rounded to nearest even, saturating); the tile's fp32
 *                dot product is multiplied back by both scales.  The filter
 *                is tested per (probe, row) (no penalty chunk).  Needs
 *                d % 16 == 0 and 64 <= d <= 128.
 *                CAPS_FP32_SPLIT: fp32 distances on the tensor cores.  Each
 *                fp32 coordinate v of a row or query is held as two bf16
 *                terms, hi = bf16(v) and lo = bf16(v - hi); a tile's score
 *                is hi.hi + hi.lo + lo.hi with fp32 accumulation (the
 *                dropped lo.lo term is below 2^-16 of sum |q_j x_j|), the
 *                filter folded into the MMA as in the bf16 penalty form;
 *                the best rerank_factor * k candidates of each query are
 *                then re-scored exactly in fp32 (the fixed-order chain of
 *                CAPS_FP32) before keeping k.  Needs d % 8 == 0,
 *                64 <= d <= 128 and the penalty form (the packed attribute
 *                bits fit its code chunk); other indexes and k > 32 use the
 *                fp32 scan.
 *   rerank_factor candidates re-scored per result in the bf16 and e4m3
 *                forms (0 = 4, at most 16): min(256, rerank_factor * k)
 *                candidates per query; each probed partition keeps its best
 *                10, 16 or 32 keys per probe -- at least k and at least a
 *                quarter of that depth.
 *   mlp_hidden   hidden units H (0 = 512).
 *   mlp_epochs   passes over the training points (0 = use mlp_init as the
 *                trained network).
 *   mlp_samples  training points S (0 = min(N, 32768)).
 *   mlp_batch    minibatch size (0 = 4096); minibatches follow the sample
 *                order, the same every epoch.
 *   mlp_lr       Adam step size (0 = 1e-3; beta 0.9/0.999, eps 1e-8).
 *   mlp_label_k  neighbours per label (0 = 10).
 *   mlp_sample_idx  optional [S] int64 training point ids (else drawn with
 *                SplitMix64(seed + 1)).
 *   mlp_sample_cons optional [S*L] int32 label filters, -1 = free field
 *                (else each field kept with probability 1/2, at least one).
 *   mlp_init     optional initial weights, fp32, W1 [H*d] | b1 [H] |
 *                W2 [B*H] | b2 [B] (row-major, output index first); else
 *                U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and zero biases
 *                from SplitMix64(seed + 2).
 *   mlp_rounds   training rounds (0 = 1).  BLISS's iterative scheme (Sec.
 *                5.2): after each round every point is assigned anew (see
 *                mlp_balance_r); before the next round each training point's
 *                label is recomputed from its same filtered neighbours'
 *                new partitions, and training continues from the current
 *                weights (fresh Adam moments).
 *   mlp_balance_r  0: a point's partition is the argmax of its logits.
 *                R >= 1 (at most 64 and B, B <= 25600): BLISS's balanced
 *                assignment -- in id order, each point goes to the
 *                least-loaded of its R largest logits (ties to the earlier
 *                of them), loads counted from zero; insertions into such an
 *                index use the same rule starting from the current
 *                partition sizes.
 *   mlp_bf16     1: train with bf16 weights and activations on the tensor
 *                cores, fp32 master weights (caps_mlp_train_bf16); 0: the
 *                fp32 step.  Assignment and probing use the fp32 weights.
 *   mlp_arbiter_queries, mlp_arbiter_m  k-means as the fallback, exact recall
 *                as the arbiter (0 queries = always keep the learned
 *                partitioner): that many data points (SplitMix64(seed + 5),
 *                each filtered on its own attributes, each field kept with
 *                probability 1/2, at least one) are searched with k = 10
 *                and m = mlp_arbiter_m on the k-means index and on the learned
 *                one (fp32 scan); the point itself is left out of its
 *                results and of its exact filtered neighbours.  The learned
 *                partitioner is kept unless k-means reaches a higher
 *                recall@10; both recalls are reported by caps_get_info.
 *   init_idx     optional [B] int64: k-means seed point ids (distinct).
 *   centroids    optional [B*d] fp32: fixed first-level centroids; k-means is
 *                skipped and f(x) = best centroid (Alg. 1 first loop).
 */
typedef struct {
  int32_t B, h, kmeans_iters;
  uint64_t seed;
  caps_metric metric;
  caps_partitioner part;
  caps_precision prec;
  int32_t rerank_factor;
  int32_t mlp_hidden, mlp_epochs;
  const int64_t* init_idx;
  const float* centroids;
  int32_t mlp_samples, mlp_batch;
  float mlp_lr;
  int32_t mlp_label_k;
  const int64_t* mlp_sample_idx;
  const int32_t* mlp_sample_cons;
  const float* mlp_init;
  int32_t mlp_rounds, mlp_balance_r;
  int32_t mlp_arbiter_queries, mlp_arbiter_m;
  int32_t mlp_bf16;
} caps_build_params;

/*
 * caps_build -- Alg. 1 (CAPS index construction) on the GPU.
 * X = [N*d] fp32 vectors, attrs = the points' attributes.  Steps: k-means
 * first level (fp64 centroid sums in id order), assignment f(x_i), per
 * partition the greedy attribute-frequency peel (most frequent code among the
 * points not yet peeled, ties to the lowest code; a dense code is
 * sum(vocab[0..f-1]) + value), then a stable sort by (partition, block, id)
 * into contiguous sub-partitions.  Inputs may be freed on return.
 * Returns CAPS_EINVAL for N < 1, d < 1, B outside [1, N], h outside [0, 63],
 * bad attribute values (dense: outside [0, vocab[f]); sparse: outside
 * [0, sp_vocab) or not strictly ascending within a point), a dense packing
 * wider than 128 bits, sparse attributes with the learned partitioner, or an
 * MLP build without epochs and without initial weights.  For sparse
 * attributes a code is the label itself and the peel counts labels.
 */
int caps_build(const caps_build_params* params, const float* X, int64_t N,
               int32_t d, const caps_attrs* attrs, void* stream,
               caps_index** out);

/*
 * caps_search_batch -- Alg. 2 (CAPS query) for nq queries.
 * Q = [nq*d] fp32; constraints = the queries' attribute constraints in the
 * form the index was built with (dense: [nq*L], -1 = unconstrained;
 * sparse: the required labels, CSR).
 * For each query: the m partitions with the best centroid score are probed
 * (ties to the lower partition); in each, the sub-partitions that can hold a
 * valid point are selected (Alg. 2; every block up to the first block whose
 * tag the query carries, skipping blocks whose tag contradicts the query (a
 * label set contradicts no tag), and the remainder block only when no tag
 * matches); every row of those blocks
 * is filtered with Def. 1 and its distance computed in fp32 (coordinates in
 * order, one fused multiply-add each); the k best are kept.
 * out_ids = [nq*k] int64 original point ids, best first, ties to the lower
 * id, -1 where fewer than k valid points were found; out_dist = [nq*k] fp32
 * (squared L2 or inner product), +inf (L2) / -inf (IP) on padded slots.
 * 1 <= k <= 128, 1 <= m <= B; m > 128 also needs B <= 16384 (the top-m
 * choice then sorts all B scores of a query in shared memory), CAPS_EINVAL
 * otherwise.  nq = 0 is a no-op.
 */
int caps_search_batch(const caps_index* index, const float* Q, int64_t nq,
                      const caps_attrs* constraints, int32_t k, int32_t m,
                      int64_t* out_ids, float* out_dist, void* stream);

/* caps_free -- release an index and all its device memory (NULL is a no-op).
 * Synchronises the device first so no enqueued work still uses it. */
void caps_free(caps_index* index);

/* caps_device_status -- synchronise `stream` and report whether a bounded
 * device-side wait expired in an earlier search on this index (the kernel
 * then stops, sets a flag and returns instead of waiting forever; that
 * search returns padding only: ids -1, distances +inf / -inf).  Returns
 * CAPS_ETIMEOUT once per such event (and clears the flag), CAPS_OK
 * otherwise; until it has been reported, tensor-core searches on the index
 * also return padding.  caps_search_batch calls it itself whenever it
 * synchronises for host outputs. */
int caps_device_status(const caps_index* index, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* caps_last_error(void);

/* ---- allocation accounting and failure injection (failure detection) -----
 * Not part of the method (the paper has no counterpart): hooks to test the
 * library's handling of an exhausted device.  Every device allocation the
 * library makes (index arrays, plan buffers, per-call stream-ordered
 * scratch) goes through one gate.
 * caps_alloc_count: device allocations made so far by this process
 *   (successful or not), all threads and devices together.
 * caps_inject_alloc_failure(n): the n-th device allocation from now (n = 1:
 *   the next one) fails without reaching the CUDA allocator, exactly as an
 *   out-of-memory device would: the call that needed it returns CAPS_ENOMEM,
 *   releases what it had taken and leaves every existing index and plan
 *   usable.  One failure per arming; n <= 0 disarms. */
int64_t caps_alloc_count(void);
void caps_inject_alloc_failure(int64_t n);

/* caps_test_scan_stall -- test hook of the bounded device waits (failure
 * detection; the paper has no counterpart).  item >= 0: every tensor-core
 * scan launched afterwards by this process (caps_search_batch on a
 * CAPS_BF16 or CAPS_FP8E4M3 index, and plans created afterwards) issues no
 * copy and no MMA for its work item number `item` (items are handed out in
 * order from 0), so the kernel's wait for that item's first tile cannot
 * complete; every bounded wait then gives up after wait_ns nanoseconds
 * (0: the default 1 s), the kernel stops with nothing in flight, and
 * caps_device_status reports CAPS_ETIMEOUT.  item < 0 restores normal
 * operation and the default limit.  Nothing faults, traps or hangs. */
void caps_test_scan_stall(int64_t item, uint64_t wait_ns);

/* ---- introspection and single steps (used to check each step alone) ---- */

typedef struct {
  int64_t N;
  int32_t d, B, h, L, metric;
  int64_t n_codes;       /* dense: sum(vocab); sparse: sp_vocab */
  int32_t attr_words;    /* packed 32-bit attribute words per row */
  int64_t device_bytes;  /* device memory held by the index */
  int32_t part;          /* caps_partitioner of the index */
  int32_t mlp_hidden;    /* H of the learned partitioner (0 for k-means) */
  int64_t n_labels;      /* training points of the learned partitioner */
  int64_t n_label_bins;  /* N when the learned partitioner was built (the
                            length of CAPS_ARR_LABEL_BINS) */
  int32_t mlp_balance_r; /* R of the balanced assignment, 0 = argmax */
  float arbiter_recall_kmeans, arbiter_recall_mlp; /* recall@10 of the build's
                            arbiter (mlp_arbiter_queries), -1 when not decided */
} caps_index_info;

int caps_get_info(const caps_index* index, caps_index_info* out);

/*
 * caps_export -- copy one index array to `dst` (host or device), `bytes`
 * must equal the array size.  Arrays (the paper's objects in brackets):
 *   CAPS_ARR_CENTROIDS [B*d] fp32    first-level centroids (Sec. 5.2)
 *   CAPS_ARR_BIN       [N] int32     f(x_i), by original id (Alg. 1 loop 1)
 *   CAPS_ARR_TAGS      [B*h] int32   A(p_j) codes, -1 = empty (Alg. 1)
 *   CAPS_ARR_KEY       [N] uint8     sub-partition j in 1..h+1 of point i
 *   CAPS_ARR_PERM      [N] int32     row r of the layout holds point perm[r]
 *   CAPS_ARR_OFFSETS   [B*(h+1)+1] int32  rows of block (b, j) are
 *                      [offsets[b*(h+1)+j-1], offsets[b*(h+1)+j])
 */
enum {
  CAPS_ARR_CENTROIDS = 0,
  CAPS_ARR_BIN = 1,
  CAPS_ARR_TAGS = 2,
  CAPS_ARR_KEY = 3,
  CAPS_ARR_PERM = 4,
  CAPS_ARR_OFFSETS = 5,
  CAPS_ARR_MLP = 6,     /* [H*d + H + B*H + B] fp32 W1|b1|W2|b2 (MLP index) */
  CAPS_ARR_LABELS = 7,  /* [S*B] fp32 labels of the last training round (MLP index) */
  CAPS_ARR_LABEL_BINS = 8 /* [N] int32 the partition of every point those labels
                             were made from (k-means, or the previous round's
                             assignment) (MLP index) */
};
int caps_export(const caps_index* index, int32_t which, void* dst,
                size_t bytes, void* stream);

/*
 * caps_assign -- Alg. 1 first loop, f(x) = best centroid: out_bin[i] = the
 * centroid with the smallest fp32 squared distance (CAPS_L2) or largest
 * inner product (CAPS_IP) to X[i], coordinates accumulated in order with one
 * fused multiply-add each, ties to the lower centroid.  X = [N*d],
 * C = [B*d], out_bin = [N] int32.
 */
int caps_assign(const float* X, int64_t N, int32_t d, const float* C,
                int32_t B, int32_t metric, int32_t* out_bin, void* stream);

/*
 * caps_probe -- Alg. 2 "select top m partitions": out_probe = [nq*m] int32,
 * partitions of each query best first (same score and tie rule as
 * caps_assign).
 */
int caps_probe(const caps_index* index, const float* Q, int64_t nq, int32_t m,
               int32_t* out_probe, void* stream);

/*
 * caps_probe_set -- the probe set of each query exactly as caps_search_batch
 * computes it (Alg. 2 "select top m partitions"): out_probe = [nq*m] int32,
 * the same m partitions as caps_probe's row (same scores, same tie rule),
 * in an unspecified order within the row.  For m <= 64 (and m <= B, hidden
 * width or d <= 2048) the scores of all partitions are first bounded by one
 * split-bf16 tensor-core product (v = hi + lo, hi*hi + hi*lo + lo*hi) with
 * a per-partition error interval; partitions whose interval lies wholly
 * above the m-th largest upper bound are in the set, those wholly below the
 * m-th largest lower bound are not, and only the rest are re-scored with the
 * fixed-order fp32 chain.  Other m: the same as caps_probe.  Q and
 * out_probe are host or device pointers; a bounded device wait that expires
 * is reported by caps_device_status.
 */
int caps_probe_set(const caps_index* index, const float* Q, int64_t nq, int32_t m,
                   int32_t* out_probe, void* stream);

/*
 * caps_select -- Alg. 2 sub-partition selection for given probes:
 * probe = [nq*m] int32 partition ids, out_sel = [nq*m] uint64, bit j-1 set
 * when block j (1..h+1) of that partition is scanned.
 */
int caps_select(const caps_index* index, const int32_t* probe, int64_t nq,
                int32_t m, const caps_attrs* constraints, uint64_t* out_sel,
                void* stream);

/* ---- learned partitioner steps (Sec. 5.2), for checking each alone -------- */

/* Mean softmax cross-entropy of the MLP on n rows X [n*d] against label
 * distributions Y [n*B], and its gradients (same layouts as the weights).
 * All fp32; loss = one float. */
int caps_mlp_loss_grad(int32_t d, int32_t H, int32_t B, const float* W1,
                       const float* b1, const float* W2, const float* b2,
                       const float* X, int64_t n, const float* Y, float* gW1,
                       float* gb1, float* gW2, float* gb2, float* loss,
                       void* stream);

/* Adam training in place: W = [H*d + H + B*H + B] fp32 (W1|b1|W2|b2),
 * minibatches of `batch` rows of X/Y in order, `epochs` passes, step lr
 * (beta 0.9/0.999, eps 1e-8).  losses (optional, host) receives the loss of
 * every step (epochs * ceil(n / batch) floats). */
int caps_mlp_train(int32_t d, int32_t H, int32_t B, float* W, const float* X,
                   int64_t n, const float* Y, int32_t epochs, int32_t batch,
                   float lr, float* losses, void* stream);

/* The same step and training with bf16 weights and activations and fp32
 * master weights (the weights the optimizer updates): every matrix product
 * runs on the tensor cores with bf16 operands and fp32 accumulation --
 * H = relu(bf16(X) bf16(W1)^T + b1), Z = bf16(H) bf16(W2)^T + b2,
 * gW2 = bf16(dZ)^T bf16(H), dH = bf16(dZ) bf16(W2) where H > 0,
 * gW1 = bf16(dH)^T bf16(X) -- while the biases, the softmax and the bias
 * gradients (fp32 column sums of dZ and dH) stay fp32.  CAPS_ETIMEOUT if a
 * bounded device wait expired. */
int caps_mlp_loss_grad_bf16(int32_t d, int32_t H, int32_t B, const float* W1,
                            const float* b1, const float* W2, const float* b2,
                            const float* X, int64_t n, const float* Y, float* gW1,
                            float* gb1, float* gW2, float* gb2, float* loss,
                            void* stream);
int caps_mlp_train_bf16(int32_t d, int32_t H, int32_t B, float* W, const float* X,
                        int64_t n, const float* Y, int32_t epochs, int32_t batch,
                        float lr, float* losses, void* stream);

/* f(x) = argmax of the logits (ties to the lower partition) for n rows;
 * every logit accumulates its products in index order with one fma each,
 * bias added last, ReLU on the hidden layer. */
int caps_mlp_assign(int32_t d, int32_t H, int32_t B, const float* W,
                    const float* X, int64_t n, int32_t* out_bin, void* stream);

/* The balanced assignment of BLISS's rounds (Sec. 5.2): each row's R largest
 * logits (same fp32 logits and tie rule as caps_mlp_assign), then in row
 * order the least-loaded of them (ties to the earlier), loads starting at
 * load0 ([B] int64, host or device; NULL = zeros).  1 <= R <= min(64, B),
 * B <= 25600. */
int caps_mlp_balance(int32_t d, int32_t H, int32_t B, const float* W, const float* X,
                     int64_t n, int32_t R, const int64_t* load0, int32_t* out_bin,
                     void* stream);

/* ---- dynamic insertion ------------------------------------------------------ */

/*
 * caps_insert -- add n points to a built index (the paper lists dynamic
 * insertion among CAPS's properties, Table 1, without giving a mechanism;
 * this is the library's reading).  Point i of X [n*d] / attrs (dense, the
 * index's L fields) gets the original id N + i, where N is the index's size
 * before the call.  Its partition is f(x) -- the nearest centroid, or the
 * learned partitioner's argmax -- and inside it the first block whose
 * attribute-frequency tag it carries, else the remainder block h+1: the
 * block the peel of Alg. 1 gives a point, with the partition's tags, the
 * centroids and the network kept as they are.  The index is then laid out
 * again by (partition, block, id), so searches see every point exactly as an
 * index built with those partitions and tags would hold it.  Cost: one pass
 * over the whole index (the layout is rebuilt), so insert in batches.
 * The call synchronises `stream`.  Query plans made before it refuse to run
 * afterwards (CAPS_EINVAL): make new ones.  Label-set (sparse) indexes:
 * CAPS_EINVAL.  Errors leave the index as it was.
 */
int caps_insert(caps_index* index, const float* X, int64_t n, const caps_attrs* attrs,
                void* stream);

/* ---- disjunctive (OR) constraints (Sec. 5.3) ------------------------------- */

/*
 * Per-(query, field) lists of allowed values: field f of query i allows
 * values[offsets[i*L+f] .. offsets[i*L+f+1]) (int32 >= 0; a value outside
 * [0, vocab[f]) matches no point); an empty list leaves the field
 * unconstrained.  offsets = [nq*L+1] int64, offsets[0] = 0, non-decreasing.
 */
typedef struct {
  int32_t L;
  const int64_t* offsets;
  const int32_t* values;
} caps_or_constraints;

/*
 * caps_search_batch_or -- Alg. 2 with disjunctive constraints.  The paper
 * maps several constraints to several sub-partitions (Sec. 5.3); here a
 * point passes when every constrained field's value is in its list, and in
 * each of the m probed partitions the blocks scanned are the union of the
 * blocks Alg. 2 selects for every single-valued query of the cross product
 * of the lists.  The library expands each query into those single-valued
 * queries (at most 256 per query, CAPS_EINVAL beyond), answers them as one
 * batch of caps_search_batch, and keeps each query's k best results by
 * (distance, id); the single-valued queries' valid sets are disjoint, so
 * this is the k best of the union.  Arguments as in caps_search_batch
 * (dense attribute indexes only); the value lists are read on the host, so
 * the call synchronises `stream` and returns with the outputs complete.
 */
int caps_search_batch_or(const caps_index* index, const float* Q, int64_t nq,
                         const caps_or_constraints* constraints, int32_t k, int32_t m,
                         int64_t* out_ids, float* out_dist, void* stream);

/* ---- batched query without device allocation ------------------------------ */

/*
 * caps_search_batch_noalloc -- the same batched query as caps_search_batch
 * (same arguments; on a CAPS_FP32 index the same results), for callers that
 * cannot allocate device
 * memory: a process whose device memory is reserved up front by another
 * framework, a serving loop that must never wait on the allocator or on the
 * device-wide synchronisation that freeing implies, or an integration that
 * forbids allocator calls after start-up.  The paper has no counterpart;
 * this is a property of the library, not of the method.
 *
 * The call makes no cudaMalloc, cudaMallocAsync or cudaFree call and no
 * allocating library call.  Its intermediates live in one fixed 16 MiB
 * device array compiled into the library, which every GPU that loads the
 * library holds until the process exits.  Batches that need more run in
 * several passes over that array; the call returns CAPS_EINVAL when even one
 * query does not fit (about 4*B + 12*m + 4*L + 33 bytes per query, i.e.
 * B up to about 4 million) and, as caps_search_batch, for m > 128 with
 * B > 16384.
 *   - It always runs the exact fp32 scan over the index's fp32 rows: on a
 *     CAPS_BF16 or CAPS_FP8E4M3 index it returns what caps_search_batch
 *     returns on a CAPS_FP32 index with the same partitions, not the
 *     tensor-core form's results.  Only k-means indexes are served.
 *   - Q, constraints->dense, out_ids and out_dist must be device memory of
 *     the current device (host memory would need a staging allocation):
 *     CAPS_EINVAL otherwise.  The call only enqueues work on `stream`.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call on a device shares the one array and it keeps the previous
 *     call's contents (nothing in it has to start at zero).  Calls that
 *     overlap on the GPU -- on different streams, or from different threads
 *     without ordering -- race on it and corrupt each other's results.
 */
int caps_search_batch_noalloc(const caps_index* index, const float* Q,
                              int64_t nq, const caps_attrs* constraints,
                              int32_t k, int32_t m, int64_t* out_ids,
                              float* out_dist, void* stream);

/* ---- tuned, graph-captured query plans -------------------------------------
 *
 * One batch shape (nq queries, k, m) against one index, prepared once and
 * then replayed: the whole batched query of Alg. 2 (filter packing, probe,
 * sub-partition selection, grouping, the persistent scan, merge and
 * re-rank) is captured into one CUDA graph, so a later batch costs two input
 * copies, one graph launch and two output copies.  Before the capture an
 * autotuner times the scan's launch shapes on the batch given to
 * caps_plan_create and keeps the fastest: where the block selection and the
 * attribute filter are applied (per pair in the epilogue, with 256 or 128
 * rows per tensor-core tile, i.e. 2 or 4 accumulator stages in tensor memory;
 * or folded into the MMA through a one-hot code chunk, 128 rows, when the
 * index has that chunk) and the most probes per work item (128 or 64).  All shapes compute the same per-probe lists, so
 * the tuner also checks that their results agree to the bit.  The index
 * remembers the chosen shape for this (k, m): later caps_search_batch calls
 * with the same k and m use it too.  Indexes that do not use the tensor-core
 * scan have nothing to tune; their plan is only the captured graph.
 *
 * The plan owns device copies of one batch's inputs and outputs
 * (nq*(4d + 4L + 12k) bytes); the graph owns its temporaries.  The index must
 * outlive the plan.  Calls on one plan must be ordered (one stream, or
 * synchronised): they share those buffers.
 */
typedef struct caps_plan caps_plan;

#define CAPS_PLAN_MAX_CANDIDATES 8
typedef struct {
  int64_t nq;
  int32_t k, m;
  int32_t tile_n;        /* chosen rows per tensor-core tile; 0 without that scan */
  int32_t item_cap;      /* chosen most probes per work item; 0 without that scan */
  int32_t n_candidates;  /* launch shapes the autotuner timed (0: none) */
  int32_t cand_tile_n[CAPS_PLAN_MAX_CANDIDATES];
  int32_t cand_item_cap[CAPS_PLAN_MAX_CANDIDATES];
  float cand_ms[CAPS_PLAN_MAX_CANDIDATES]; /* median device ms of one search each */
  int32_t graph_nodes;   /* nodes of the captured graph */
  int32_t pen;           /* chosen: 1 = block selection and filter folded into the MMA */
  int32_t cand_pen[CAPS_PLAN_MAX_CANDIDATES];
} caps_plan_info;

/* Prepare a plan for batches of nq queries (Q [nq*d] fp32, constraints dense
 * [nq*L], host or device).  These queries are the autotuner's sample: it
 * runs the full search 4 times per candidate shape on them (autotune = 0:
 * keep the default shape, 256 rows and 128 probes).  The call synchronises
 * `stream`.  CAPS_EINVAL on bad arguments, CAPS_ECUDA if the capture or the
 * instantiation fails; *out is set only on success. */
int caps_plan_create(const caps_index* index, const float* Q, int64_t nq,
                     const caps_attrs* constraints, int32_t k, int32_t m,
                     int32_t autotune, void* stream, caps_plan** out);

/* Run the plan on a batch of nq <= plan nq queries (arguments as in
 * caps_search_batch; host or device).  The graph always processes the
 * plan's nq rows (rows beyond this call's nq hold earlier inputs and their
 * results are not copied out).  Asynchronous on `stream` when both outputs
 * are device memory; with a host output the call waits and also reports an
 * expired bounded device wait as CAPS_ETIMEOUT. */
int caps_plan_search(caps_plan* plan, const float* Q, int64_t nq,
                     const caps_attrs* constraints, int64_t* out_ids,
                     float* out_dist, void* stream);

int caps_plan_get_info(const caps_plan* plan, caps_plan_info* out);

/* Destroys the graph and frees the plan's buffers (synchronises the device). */
void caps_plan_free(caps_plan* plan);

/* ---- stage timing (measurement aid, off by default) ---------------------- */

/* Per-stage device time of the last caps_search_batch call made on this
 * thread while timing was on, in milliseconds, summed over query chunks.
 * The stages are the kernels of Alg. 2: query filter packing, centroid
 * scores, top-m partition choice, sub-partition selection, grouping of the
 * probes by partition, the fused attribute match + distance + top-k scan, and
 * the merge of the per-partition top-k lists. */
typedef struct {
  float prep_ms, scores_ms, topm_ms, select_ms;
  float group_ms; /* probes grouped by partition into work items */
  float scan_ms;  /* the fused attribute match + distance + top-k kernel */
  float merge_ms; /* per-query merge of the m partial top-k lists */
  int32_t launches; /* kernels launched by that call */
} caps_stage_times;

/* enable = 1: record CUDA events between the stages of every following
 * caps_search_batch on this thread (adds event records, no syncs).
 * enable = 0: stop. */
int caps_set_timing(int32_t enable);

/* Wait for the last timed search and read its stage times (CAPS_EINVAL if
 * no search was timed on this thread). */
int caps_get_stage_times(caps_stage_times* out);

#ifdef __cplusplus
}
#endif
#endif /* CAPS_H_ */
