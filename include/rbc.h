/*
 * rbc.h -- C ABI of the randomized bilinear computation (RBC) library for GB300 (sm_103a).
 *
 * The library evaluates C = F^(L)(A, B), the recursive randomized bilinear computation of
 * Malik & Becker, "Randomization of approximate bilinear computation for matrix
 * multiplication" (arXiv 1905.07439), Section 2.1.1, Eq. recursive-random-formula:
 * at every node of an L-level recursion the n0 x n0 block indices of a bilinear formula
 * (U, V, W) (Section 1, Eq. (1)) are randomized by signed permutations M_i = P_i S_i
 * (Section 2.1), folded into coefficient tables u^, v^, w^ (Prop. 10, Eq. randomized-algorithm):
 *
 *     u^_klr  = u_{pi1(k) pi2(l) r} s1(k) s2(l)
 *     v^_k'l'r = v_{pi2(k') pi3(l') r} s2(k') s3(l')
 *     w^_ijr  = (1 - kappa)^{-1} s1(i) s3(j) w_{pi1(i) pi3(j) r}
 *
 * and the node computes S_r = sum u^_klr A_kl, T_r = sum v^_k'l'r B_k'l' (encode),
 * M_r = F^(q-1)(S_r, T_r) (the leaves, q = 0, are standard products) and
 * C_ij = sum_r w^_ijr M_r (decode).  kappa is Eq. epsilon-def.
 *
 * Conventions for every call:
 *   - Matrices are row-major with a leading dimension (ld, in elements, >= N).
 *   - Tensors U, V, W are float64 arrays of n0*n0*R entries, entry (k, l, r) at
 *     index (k*n0 + l)*R + r (0-based), as in Eq. (1).
 *   - Device pointers are caller-owned CUDA global memory on the current device;
 *     host pointers are caller-owned host memory.  The library keeps no pointer
 *     past the return of a call.
 *   - Every call returns an rbc_status and never aborts the process; the text of the
 *     last error of the calling thread is available from rbc_last_error().
 *   - Device work is enqueued on the given stream (a cudaStream_t passed as void*;
 *     NULL is the legacy default stream) and is asynchronous with respect to the host.
 */
#ifndef RBC_H_
#define RBC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbc_plan_s* rbc_plan_t;

typedef enum {
  RBC_OK = 0,
  RBC_EINVAL = 1,       /* invalid argument (shape, size, enum, null pointer)           */
  RBC_ENOMEM = 2,       /* workspace too small or a host allocation failed              */
  RBC_ECUDA = 3,        /* a CUDA runtime call failed (no device, launch error, ...)    */
  RBC_ETIMEOUT = 4,     /* a bounded device-side wait expired                           */
  RBC_EBUSY = 5,        /* queue full / request still in flight                         */
  RBC_EKAPPA = 6,       /* kappa == 1, the randomized formula is undefined (Def. RandABC) */
  RBC_EUNSUPPORTED = 7  /* valid but not implemented combination (dtype pair, tree size) */
} rbc_status;

/* Element type of A, B and C. */
typedef enum { RBC_IO_F64 = 0, RBC_IO_F32 = 1 } rbc_io_dtype;

/* Arithmetic of the leaf products F^(0) (Section 2.1.1).  Encode and decode run in the
 * I/O type; leaves accumulate in fp32 (fp64 for RBC_LEAF_F64).  The split modes store
 * x = hi + lo with hi = round(x), lo = round(x - hi) and compute hi*hi' + hi*lo' + lo*hi'.
 * RBC_LEAF_BF16X6 stores three bf16 pieces x = b0 + b1 + b2 (b0 = round(x),
 * b1 = round(x - b0), b2 = round(x - b0 - b1); exact for normal fp32 x) and adds the six
 * products whose pieces carry the leading 24 bits, b0*b2' + b2*b0' + b1*b1' + b0*b1' +
 * b1*b0' + b0*b0' (the bf16x6 method of Henry, Tang & Heinecke, 2019): an fp32-accurate
 * product on the bf16 tensor cores.
 * RBC_LEAF_F16X3 scales every row of the left leaf operands and every column of the right
 * ones by a power of two (the same for all leaves: from the largest |entry| of the rows of A
 * congruent mod m, of the columns of B congruent mod m, times the formula's growth bound per
 * level), so that the scaled entries stay below 2^15, stores two fp16 pieces x = h0 + h1
 * (h0 = round(x), h1 = round(x - h0), kept as 2^11 h1: 22 significant bits), adds
 * h0*h1' + h1*h0' and h0*h0' in two accumulators drained every 64 elements of K (the tensor
 * cores' truncating accumulation of 22-bit products is biased on same-signed data), and removes
 * the scales in the leaf epilogue (exact powers of two).  Half the tensor-core products of
 * bf16x6 at about 2^-22 relative representation error; entries 2^29 or more below the largest
 * of their class lose relative accuracy gradually (fp16 subnormals). */
typedef enum {
  RBC_LEAF_F64 = 0,    /* fp64 FMA (SIMT); I/O must be F64                         */
  RBC_LEAF_F32 = 1,    /* fp32 FMA (SIMT)                                          */
  RBC_LEAF_TF32 = 2,   /* tcgen05 kind::tf32, fp32 accumulate in TMEM               */
  RBC_LEAF_BF16 = 3,   /* tcgen05 kind::f16 with bf16 operands                      */
  RBC_LEAF_F16 = 4,    /* tcgen05 kind::f16 with fp16 operands                      */
  RBC_LEAF_3XBF16 = 5, /* three bf16 tcgen05 products (split compensated)          */
  RBC_LEAF_3XTF32 = 6, /* three tf32 tcgen05 products (split compensated)         */
  RBC_LEAF_BF16X6 = 7, /* six bf16 tcgen05 products of three-piece splits (fp32 level) */
  RBC_LEAF_F16X3 = 8   /* three fp16 tcgen05 products of scaled two-piece splits      */
} rbc_leaf_dtype;

/* Which parts of the signed permutations are drawn (Section 3.2: fully randomized,
 * random sign, random permutation; deterministic F^(Q) has s = 1, pi = id). */
typedef enum { RBC_RAND_FULL = 0, RBC_RAND_SIGN = 1, RBC_RAND_PERM = 2, RBC_RAND_NONE = 3 } rbc_rand_mode;

/* One independent draw set per recursion node, or one per recursion level
 * (the literal definition of Section 2.1.1). */
typedef enum { RBC_DRAW_PER_NODE = 0, RBC_DRAW_PER_LEVEL = 1 } rbc_draw_scope;

typedef struct {
  const double* U;   /* host, n0*n0*R, copied by the plan                             */
  const double* V;
  const double* W;
  int R;             /* number of products, 1 <= R <= 4096; the kernels need
                        n0*n0*R <= 256 and, per launch, at most 1024 draw sets        */
  int n0;            /* block dimension of the formula (the paper's n), 2 <= n0 <= 4  */
  int levels;        /* recursion levels L (the paper's Q), 0 <= L <= 8               */
  uint64_t seed;     /* seed of the counter-based draws                               */
  int rand_mode;     /* rbc_rand_mode                                                 */
  int draw_scope;    /* rbc_draw_scope                                                */
  int rescale_kappa; /* -1: rescale by (1-kappa)^-1 iff randomized; 0: never; 1: always */
} rbc_plan_desc;

typedef struct {
  int R, n0, levels, rand_mode, draw_scope;
  int64_t draw_count;  /* draw sets held: sum_{d<L} R^d (per node) or L (per level)   */
  int64_t leaf_count;  /* R^L leaf products                                           */
  double kappa;        /* Eq. epsilon-def                                             */
  double tau;          /* ||Y - X||, Def. ABC                                          */
  double gamma;        /* Eq. square-root-of-sum                                      */
  double scale;        /* (1 - kappa)^{-1} if rescaled, else 1                         */
  uint64_t seed;
  /* 1: U, V, W are exactly Strassen's formula, 2: exactly Laderman's (the two formulas of
   * Section 1, in the forms of the library's built-in tables); 0: any other formula.  The
   * built-in formulas run one-level passes with their sparsity compiled in. */
  int builtin_formula;
} rbc_plan_info;

/* Draws (Section 2.1).  Counter-based: draw set `key` uses the six words
 *   w_c = mix64(seed + 0x9E3779B97F4A7C15 * (1 + 8*key + c)),  c = 0..5,
 * mix64 being the SplitMix64 output function.  pi_{c+1} (c = 0,1,2) is Fisher-Yates
 * from i = n0-1 down to 1 swapping p[i] and p[j], j = floor(mix64(w_c + i) * (i+1) / 2^64),
 * pi(j) = p[j]; s_{c-2}(j) = -1 iff bit j of w_c (c = 3,4,5) is set.  key is the node id in
 * heap order (root 0, child r of node p is p*R + r + 1) for per-node scope, or the depth
 * (root 0) for per-level scope. */

/* Create a plan with full randomization, per-node draws, default rescaling.
 * Errors: RBC_EINVAL (null pointer, R/n0/levels out of range), RBC_EKAPPA (kappa == 1),
 * RBC_ENOMEM.  Host-only: touches no device.  *out is owned by the caller and released
 * with rbc_plan_destroy. */
rbc_status rbc_plan_create(const double* U, const double* V, const double* W, int R, int n0,
                           int levels, uint64_t seed, rbc_plan_t* out);

/* Same with every option of rbc_plan_desc (Section 3.2 variants, draw scope, rescaling). */
rbc_status rbc_plan_create_ex(const rbc_plan_desc* desc, rbc_plan_t* out);

/* Release a plan (NULL is ignored).  No device work may still use it. */
void rbc_plan_destroy(rbc_plan_t plan);

/* Constants of the plan (Eq. epsilon-def, Def. ABC, Eq. square-root-of-sum). */
rbc_status rbc_plan_query(rbc_plan_t plan, rbc_plan_info* info);

/* Export draw sets [first, first+count) for bit-exact checks: perms[(t*3 + c)*n0 + j] =
 * pi_{c+1}(j), signs[(t*3 + c)*n0 + j] = s_{c+1}(j) in {-1, +1}.  Host buffers of
 * count*3*n0 bytes each.  RBC_EINVAL if the range exceeds draw_count. */
rbc_status rbc_plan_draws(rbc_plan_t plan, int64_t first, int64_t count, int8_t* perms,
                          int8_t* signs);

/* Expanded tables u^, v^, w^ (Prop. 10) of draw set `key`, each n0*n0*R float64 in the
 * layout of U.  w^ includes the plan's scale. */
rbc_status rbc_plan_tables(rbc_plan_t plan, int64_t key, double* Uhat, double* Vhat,
                           double* What);

/* Bytes of device workspace rbc_matmul needs for an N x N product with these types
 * (0 when the combination is invalid; 256-byte aligned pointer required). */
size_t rbc_workspace_size(rbc_plan_t plan, int64_t N, int io_dtype, int leaf_dtype);

/* C = F^(L)(A, B) for N x N matrices, N a multiple of n0^L (pad first, Section 2.1.1).
 * A, B: device, read only; C: device, overwritten (must not alias A or B).
 * workspace: device scratch of at least rbc_workspace_size() bytes, contents undefined
 * on return; two calls in flight at once need two workspaces.
 * Errors: RBC_EINVAL (N, ld, dtype pair, alignment), RBC_ENOMEM (workspace too small),
 * RBC_EUNSUPPORTED (tree deeper than the kernel tables hold), RBC_ECUDA (launch failure). */
rbc_status rbc_matmul(rbc_plan_t plan, const void* A, const void* B, void* C, int64_t N,
                      int64_t lda, int64_t ldb, int64_t ldc, int io_dtype, int leaf_dtype,
                      void* workspace, size_t workspace_bytes, void* stream);

/* Options of rbc_matmul_ex.  decode: 0 = fused into the leaf products when the kernel
 * tables hold the whole tree, else level by level; 1 = fused (RBC_EUNSUPPORTED if the tree
 * is too large); 2 = level by level (the leaf products are stored, then each level's
 * C_ij = sum_r w^_ijr M_r runs as its own pass, r in order, so the result is bitwise
 * reproducible).  The fused decode adds each leaf's contribution to C with atomic adds,
 * so its summation order, and the last bits of C, may vary from call to call. */
typedef struct {
  int decode;
  /* Test hook for the bounded-wait path (0 = off; tensor-core leaf modes only, else
   * RBC_EINVAL): the leaf kernel issues no operand copies, so the first wait of its MMA warp
   * expires after 2 s; the kernel then records RBC_ETIMEOUT in the workspace status word (read
   * by rbc_workspace_check), releases its tensor memory and returns without the product.
   * Nothing faults and the CUDA context stays usable. */
  int stall_leaf_copies;
  int reserved[6];
  /* Optional timing hooks: CUDA events (cudaEvent_t as void*, NULL = skip) recorded on the
   * call's stream at [0] the start, [1] the end of the encode, [2] the end of the leaf
   * products (including a fused decode), [3] the end of the call. */
  void* events[4];
  /* Output: number of kernels the call launched (memsets not counted). */
  int64_t launches;
} rbc_matmul_opts;

/* rbc_workspace_size / rbc_matmul with options (opts may be NULL = defaults; rbc_matmul_ex
 * writes opts->launches). */
size_t rbc_workspace_size_ex(rbc_plan_t plan, int64_t N, int io_dtype, int leaf_dtype,
                             const rbc_matmul_opts* opts);
rbc_status rbc_matmul_ex(rbc_plan_t plan, const void* A, const void* B, void* C, int64_t N,
                         int64_t lda, int64_t ldb, int64_t ldc, int io_dtype, int leaf_dtype,
                         void* workspace, size_t workspace_bytes, void* stream,
                         rbc_matmul_opts* opts);

/* Independent realizations F^(L)_1 .. F^(L)_K of one plan's product (Section 3: the error
 * of an average of realizations, Eq. error-of-average, and the spread of single
 * realizations, Eq. average-of-error).  Realization k is the plan's computation with its
 * draws taken from seed seeds[k] instead of the plan's own (the same draws a plan created
 * with that seed has; seeds[k] == the plan's seed reuses its draws).  A, B: device, N x N,
 * shared by all realizations.  Output k: C + k * strideC (elements; strideC >= ldc * N when
 * count > 1), N x N with leading dim ldc.  As many realizations as the workspace holds run
 * together, their encode/decode passes batched across realizations (staged decode) and their
 * leaf products in one launch; rbc_realizations_workspace_size(plan, N, io, leaf, count) is
 * the workspace that holds `count` at once, and any workspace of at least the size for
 * count = 1 works (batches then follow one another on the stream).  Leaf modes and dtypes
 * as rbc_matmul.  L = 0 computes the same standard product K times. */
size_t rbc_realizations_workspace_size(rbc_plan_t plan, int64_t N, int io_dtype, int leaf_dtype,
                                       int64_t count);
rbc_status rbc_matmul_realizations(rbc_plan_t plan, const uint64_t* seeds, int64_t count,
                                   const void* A, const void* B, void* C, int64_t N, int64_t lda,
                                   int64_t ldb, int64_t ldc, int64_t strideC, int io_dtype,
                                   int leaf_dtype, void* workspace, size_t workspace_bytes,
                                   void* stream);

/* Relative Frobenius errors of K realizations against a reference product (Section 3),
 * in fp64 with a fixed summation order (bit-identical on repeated calls):
 *   RBC_ERR_EACH:    err[k]     = ||C_k - Ref||_F / ||Ref||_F              (Eq. average-of-error)
 *   RBC_ERR_AVERAGE: err[n - 1] = ||(1/n) sum_{k<n} C_k - Ref||_F / ||Ref||_F, n = 1..K
 *                                                                          (Eq. error-of-average)
 * C: device, K matrices N x N of dtype c_dtype (rbc_io_dtype) at C + k * strideC, leading dim
 * ldc.  Ref: device fp64, N x N, leading dim ldr.  err: device, K doubles.  work: device
 * scratch of rbc_realization_errors_work_size(K, N) bytes.  ||Ref|| = 0 gives inf/nan. */
typedef enum { RBC_ERR_EACH = 0, RBC_ERR_AVERAGE = 1 } rbc_err_mode;
rbc_status rbc_realization_errors(const void* C, int c_dtype, int64_t K, int64_t N, int64_t ldc,
                                  int64_t strideC, const double* Ref, int64_t ldr, int mode,
                                  double* err, void* work, size_t work_bytes, void* stream);
size_t rbc_realization_errors_work_size(int64_t K, int64_t N);

/* rbc_matmul without a caller workspace, for callers that cannot allocate device memory
 * when they multiply (a framework that has reserved the whole device heap for its own
 * allocator, code allowed to allocate only at start-up, paths that cannot handle an
 * allocation failure).  The paper has no counterpart: this is a property of the library.
 *
 * Scratch comes from a fixed 64 MiB array inside the library's device image (every GPU
 * that loads the library holds it until exit; rbc_static_scratch_bytes() reports the size).
 * Products needing more scratch than that (rbc_workspace_size) return RBC_ENOMEM with a
 * message.  The call itself allocates nothing.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array and it keeps the previous call's contents (only
 * the status word is cleared per call), so calls whose device work overlaps -- on
 * different streams or threads -- race and give wrong results: order them on one stream.
 * The address is cached per device for the life of the process: resetting the device
 * (cudaDeviceReset) after the first call is not supported.  The device status word of the
 * bounded waits lives at the start of the array: read it with rbc_static_scratch_check. */
rbc_status rbc_matmul_static(rbc_plan_t plan, const void* A, const void* B, void* C, int64_t N,
                             int64_t lda, int64_t ldb, int64_t ldc, int io_dtype, int leaf_dtype,
                             void* stream);
size_t rbc_static_scratch_bytes(void);
/* rbc_workspace_check on the static array of the current device: waits for `stream`, copies
 * the status word of the calls that used the array to *device_status (0, or RBC_ETIMEOUT when
 * a bounded wait inside a kernel expired and the result is invalid) and clears it.
 * Synchronizes the stream. */
rbc_status rbc_static_scratch_check(void* stream, int* device_status);
/* Device address of the static array on the current device (NULL on error), e.g. to pass it
 * as the workspace of rbc_matmul_ex for its options; the sharing rules above apply. */
void* rbc_static_scratch_ptr(void);

/* Grouped batch of independent products with fp32 I/O and tensor-core leaves (many
 * instances of uneven sizes, formulas, depths and seeds).  Each instance follows Section
 * 2.1.1 exactly as rbc_matmul does (staged decode); the R^L leaf products of ALL instances
 * run in one persistent tensor-core launch.  Items are copied at creation; their plans and
 * device buffers must stay valid while the group is used.  A group is used by one host
 * thread at a time. */
typedef struct {
  rbc_plan_t plan;
  const void* A;   /* device, fp32, N x N, leading dimension lda */
  const void* B;
  void* C;         /* device, fp32, overwritten */
  int64_t N, lda, ldb, ldc;
} rbc_group_item;

typedef struct rbc_group_s* rbc_group_t;

/* Tile configuration chosen by rbc_group_tune: tile width bn (128 or 256), tile order group
 * (0: per-instance default, 1: row-major, 8: groups of 8 tile rows), candidates timed, the
 * best grouped-launch time in milliseconds, and CTAs per SM (1; or 2, which plain, not split,
 * leaf modes may take with 128-wide tiles of two pipeline stages each). */
typedef struct {
  int bn, group, candidates;
  float best_ms;
  int ctas_per_sm;
} rbc_group_tuning;

#define RBC_GROUP_GRAPH 1  /* rbc_group_run flag: capture once into a CUDA graph, then replay */

/* Validate the items and lay out their workspaces.  A tuning found earlier in the process for
 * the same signature (leaf mode and instance shapes) is reused.  Host only. */
rbc_status rbc_group_create(const rbc_group_item* items, int count, int leaf_dtype, rbc_group_t* out);
size_t rbc_group_workspace_size(rbc_group_t group);
/* Enqueue the whole batch on `stream` (asynchronous).  With RBC_GROUP_GRAPH the first call
 * captures the sequence into a CUDA graph (the workspace and stream are bound to it) and
 * every call launches that graph; capture needs a created stream (RBC_EINVAL on the
 * default stream).  The first call with a new workspace uploads the instance
 * descriptors synchronously. */
rbc_status rbc_group_run(rbc_group_t group, void* workspace, size_t workspace_bytes, void* stream, int flags);
/* Autotuner: runs the batch once, then times the grouped leaf launch for every candidate tile
 * configuration and keeps the fastest (also for later groups of the same signature).
 * Synchronizes the stream.  `out` may be NULL. */
rbc_status rbc_group_tune(rbc_group_t group, void* workspace, size_t workspace_bytes, void* stream,
                          rbc_group_tuning* out);
/* Apply a tile configuration: bn, group and ctas_per_sm of `cfg` (its other fields are
 * ignored), e.g. one that rbc_group_tune chose in an earlier process.  The next
 * rbc_group_run rebinds the instance descriptors (and recaptures its graph).  RBC_EINVAL for
 * a NULL argument or a configuration the group does not admit: bn 256 needs every padded leaf
 * size to be a multiple of 256; group must be 0, 1, 2, 4, 8 or 16; ctas_per_sm 2 needs bn 128
 * and a plain (not split) leaf mode. */
rbc_status rbc_group_configure(rbc_group_t group, const rbc_group_tuning* cfg);
void rbc_group_destroy(rbc_group_t group);

/* Serving queue: independent products submitted as they arrive and served with continuous
 * batching.  A worker thread admits requests in arrival order as soon as enough of the queue's
 * device workspace pool is free (the pool is one region of `workspace_cap` bytes, allocated at
 * creation); a request that does not fit may be passed by later ones that do, at most 32 times,
 * after which admission waits for it.  Small requests (N <= 2048) with the same tensor-core leaf
 * mode admitted together form one unit whose leaf products share one grouped launch (the
 * decode then runs level by level); every other request is a unit of its own, computed
 * exactly as rbc_matmul computes it.  Units run on their own streams (one of `streams`), so
 * work from requests that arrived while others were running overlaps on the device.  Submit
 * and poll may be called from any host thread; the queue's lock is never held while work is
 * enqueued, and poll never blocks. */
typedef struct rbc_queue_s* rbc_queue_t;

typedef struct {
  rbc_plan_t plan;
  const void* A;   /* device; A, B, C stay valid and untouched until the request is collected */
  const void* B;
  void* C;
  int64_t N, lda, ldb, ldc;
  int io_dtype, leaf_dtype;
} rbc_request;

typedef struct {
  int64_t pending, running;      /* requests waiting / in flight                                */
  uint64_t admitted, completed;
  size_t workspace_used, workspace_peak, workspace_cap;
  int peak_running;              /* most requests in flight at once                             */
} rbc_queue_info;

/* Create a queue on `device` with a workspace pool of workspace_cap bytes (one cudaMalloc)
 * and `streams` streams (1..256).  RBC_ENOMEM if the pool cannot be allocated. */
rbc_status rbc_queue_create(int device, size_t workspace_cap, int streams, rbc_queue_t* out);
/* Enqueue `count` requests; they receive tickets *ticket, *ticket + 1, ...  A request whose
 * arguments are invalid completes at once with RBC_EINVAL; one whose workspace exceeds the
 * whole pool is refused (RBC_ENOMEM, nothing enqueued). */
rbc_status rbc_batch_submit(rbc_queue_t queue, const rbc_request* reqs, int count, uint64_t* ticket);
/* Non-blocking completion check: *done = 0 (waiting or running) or 1 (finished; the ticket is
 * then collected and forgotten).  Returns the request's own status when it finished with an
 * error (e.g. RBC_ETIMEOUT from a bounded device wait), RBC_EINVAL for an unknown ticket. */
rbc_status rbc_batch_poll(rbc_queue_t queue, uint64_t ticket, int* done);
rbc_status rbc_queue_stats(rbc_queue_t queue, rbc_queue_info* info);
/* Finish every submitted request, then release the streams and the pool. */
void rbc_queue_destroy(rbc_queue_t queue);

/* Device-side status of the calls that used `workspace` (its first 4 bytes, cleared by every
 * rbc_matmul): waits for `stream`, copies the word to *device_status and clears it.  0 means
 * no error; RBC_ETIMEOUT means a bounded wait inside a kernel expired and that kernel skipped
 * its remaining work (the result is then invalid).  Returns the word as a status.
 * Synchronizes the stream. */
rbc_status rbc_workspace_check(void* workspace, void* stream, int* device_status);

/* Frobenius reductions in fp64 (Section 3's relative errors): out[0] = sum (X - Y)^2,
 * out[1] = sum Y^2 (Y == NULL: out[0] = sum X^2, out[1] = 0).  X, Y: device, rows x cols
 * row-major with lds ldx, ldy, element types rbc_io_dtype.  out: device, 2 doubles.
 * work: device scratch of rbc_norms_work_size() bytes.  Deterministic order. */
rbc_status rbc_norms(const void* X, const void* Y, int64_t rows, int64_t cols, int64_t ldx,
                     int64_t ldy, int x_dtype, int y_dtype, double* out, void* work,
                     size_t work_bytes, void* stream);
size_t rbc_norms_work_size(void);

const char* rbc_status_string(rbc_status status);
const char* rbc_last_error(void);
int rbc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RBC_H_ */
