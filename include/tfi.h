/*
 * tfi.h — C ABI of libtfi: Structure-Adaptive Tree Field Integration (StAd-TFI)
 * on one B300 GPU (sm_103a).
 *
 * The operation (paper Eq. "integration", specialised to trees in Eq.
 * "stad-target"; weighted trees on the quantised metric of Appendix
 * "Distance quantization for FFT-Based Integrators"):
 *
 *     out[u, c] = sum_v f(delta * dhat(u, v)) * F[v, c]      for every vertex u
 *
 * where q_e = max(1, round(w_e / delta)) is the integer length of edge e
 * (round half to even) and dhat(u, v) is the sum of q_e on the tree path.
 * Vertices in different trees of a forest do not interact.
 *
 * The plan holds the paper's recursive decomposition (Section 2.1, Algorithm
 * 1 "DecomposeOffPathComponents", Algorithm 6 "ChooseBackbone", Eq.
 * "stad-score") flattened into arrays, the grid samples of f and the cached
 * kernel spectra. An apply evaluates every call's cross term (Eq.
 * "stad-split", Eq. "sumofFFTterms", Eq. "stad-E", Lemma "Cross-component
 * correction") with GPU kernels and adds the leaf terms.
 *
 * Conventions
 *   - No function throws; every function returns a tfi_status. A message for
 *     the last error of the calling thread is available from tfi_last_error().
 *   - Device pointers are CUDA device addresses on the current device; the
 *     caller owns them. Host pointers are read during the call only.
 *   - Applies are stream-ordered and asynchronous with respect to the host. A
 *     plan may be used by one stream at a time (it owns one workspace).
 *   - Fields are row-major N x d arrays (row stride d elements), dtype
 *     TFI_DTYPE_F32 (float) or TFI_DTYPE_BF16 (bfloat16); accumulation is
 *     FP32. Results are deterministic: no floating-point atomics.
 */
#ifndef TFI_H
#define TFI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tfi_status;
#define TFI_OK                 0
#define TFI_ERR_ARG            1  /* null pointer, bad size, bad enum, d > max_channels, ... */
#define TFI_ERR_NOT_TREE       2  /* edge list has a cycle, a self loop or an out-of-range vertex */
#define TFI_ERR_WEIGHT         3  /* an edge weight is not finite or not > 0 */
#define TFI_ERR_GRID_OVERFLOW  4  /* a grid distance exceeds 2^30, or a sampled table is too short */
#define TFI_ERR_OOM            5  /* host or device allocation failed */
#define TFI_ERR_CUDA           6  /* a CUDA runtime call failed (message in tfi_last_error) */
#define TFI_ERR_TIMEOUT        7  /* a bounded device wait gave up */
#define TFI_ERR_UNSUPPORTED    8  /* the plan needs an evaluator this build does not have */
#define TFI_ERR_NO_DEVICE      9  /* no CUDA device, or the plan was built host-only */

typedef struct tfi_plan_s *tfi_plan_t;
typedef void *tfi_stream_t;       /* a cudaStream_t; NULL = the legacy default stream */

/* A forest on vertices 0..n-1: n_edges undirected edges (u[i], v[i]) of
 * length w[i] > 0. A tree has n_edges = n - 1. Host memory, read only. */
typedef struct {
    int32_t n;
    int32_t n_edges;
    const int32_t *u;
    const int32_t *v;
    const double *w;
} tfi_tree;

/* Kernel f(x) of a distance x in original units. The plan samples it on the
 * grid, f(k * delta), in FP64 and rounds the samples once to FP32.
 *   TFI_F_EXPSUM   f(x) = sum_k a_k exp(-b_k x)   params = [a_1, b_1, a_2, b_2, ...]
 *   TFI_F_GAUSS    f(x) = a exp(-c x^2)           params = [a, c]
 *   TFI_F_RATIONAL f(x) = a / (1 + c x^e)^p       params = [a, c, e, p]
 *   TFI_F_POWEXP   f(x) = a x^p exp(-b x)          params = [a, p, b]
 *   TFI_F_TABLE    f(k delta) = table[k] for k < table_len; a plan that needs a
 *                  longer table fails with TFI_ERR_GRID_OVERFLOW. */
#define TFI_F_TABLE    0
#define TFI_F_EXPSUM   1
#define TFI_F_GAUSS    2
#define TFI_F_RATIONAL 3
#define TFI_F_POWEXP   4
typedef struct {
    int32_t kind;
    int32_t n_params;
    const double *params;   /* host */
    int64_t table_len;
    const double *table;    /* host; TFI_F_TABLE only */
} tfi_kernel;

/* Backbone policy per recursive call (Section 2.4, Algorithm 6):
 *   ADAPTIVE  diameter path vs single centroid by Eq. "stad-score" (grid units)
 *   DIAMETER  always the (weighted) diameter path
 *   CENTROID  always a single centroid vertex */
#define TFI_POLICY_ADAPTIVE 0
#define TFI_POLICY_DIAMETER 1
#define TFI_POLICY_CENTROID 2

#define TFI_PLAN_HOST_ONLY  1   /* build the decomposition on the host only (no GPU use) */
#define TFI_PLAN_SWEEP      2   /* exponential-sum kernels only: evaluate every call's cross table
                                   and corrections by the two backbone sweeps of Algorithm 7
                                   ("CrossSubRoutineExp"): G_q[s] = lambda^q G_0[s],
                                   E_alpha[q] = lambda^q E_alpha[0], O(J |V(S)|) per call */
#define TFI_PLAN_HANKEL     4   /* also consider the Hankel-matrix evaluator of the cross table
                                   (attention-width evaluation of Eq. "sumofFFTterms"): B = Fh A
                                   on tensor cores with Fh[l][r] = f(l + r), then prefix sums
                                   along antidiagonals. A job qualifies when H + 1 <= 64 and
                                   H + L + 1 <= 128 (grid units); it is chosen when the
                                   channel-aware cost model (at max_channels) ranks it below
                                   direct summation and the FFT */
#define TFI_PLAN_HANKEL_ALL 8   /* every qualifying job uses the Hankel evaluator */
#define TFI_PLAN_SWEEP_AUTO 32  /* exponential-sum kernels: each table (a call's cross table or a
                                   component's correction) is evaluated by the Algorithm 7 sweeps
                                   when their cost, J (6 per bin + 4 per backbone run) per channel,
                                   is below that of the evaluator the cost model picked otherwise;
                                   ignored for other kernels */
#define TFI_PLAN_FFT_BIG_ALL 64 /* every table beyond one CTA's shared memory (P1 P2 > 2^14 grid points;
                                   up to 2^25 points with a backbone axis of at most 2^13) is evaluated
                                   by the four-step FFT through global memory, whatever the cost model
                                   prefers (by default it competes with direct summation) */
#define TFI_PLAN_NO_TRUNCATE 128 /* keep every table whole. By default, when every FP32 sample f(k delta) from
                                   some distance T up to the largest one a table can pair is zero, bins at
                                   depth >= T (which then neither contribute nor receive anything) are left
                                   out of their tables and their table values set to zero: exact for the
                                   sampled kernel, and the tables shrink to depths below T. Not applied
                                   with TFI_PLAN_SWEEP / TFI_PLAN_SWEEP_AUTO */
#define TFI_PLAN_DIRECT_ALL 256 /* evaluate every table by direct summation (no FFT; Hankel and sweeps only if
                                   their flags ask). Its sums are of the field's terms themselves, so for a
                                   positive field and a decreasing kernel every output keeps a small error
                                   relative to itself, where an FFT's error is relative to its whole table:
                                   what Sinkhorn iterations at a small eps need (with the support truncation
                                   keeping those tables short) */
#define TFI_PLAN_LEAF_ALU   16  /* dense leaves on the FP32 ALUs for every d. By default the leaves of
                                   >= 64 vertices are f(D) x F products on the tensor cores (tcgen05
                                   kind::tf32, f(D) split into hi + lo) for BF16 fields with d >= 64
                                   and for FP32 fields with d >= 16 when the leaves are at least a
                                   quarter of the plan's leaf and table flops (F split too, three
                                   products, a fresh accumulator for every 32 sources, added in FP32
                                   registers: within the 1e-4 bound); the rest on the FP32 ALUs */
#define TFI_PLAN_LEAF_TC    512 /* FP32 fields: the tensor-core leaves for every d and plan (by default
                                   only from d = 16, below which the FP32 ALUs are faster, and when the
                                   leaves are a quarter of the work or more). Ignored when
                                   TFI_PLAN_LEAF_ALU is set. */
#define TFI_PLAN_TABLES_ALU 1024 /* tables evaluated by direct summation on the FP32 ALUs for every d.
                                   By default, for d > 16 (for d = 16 from 512 bins), a direct table
                                   of 64 .. 4096 bins is an
                                   f(r_i + r_j + |x_i - x_j|) x S product on the tensor cores
                                   (tcgen05 kind::tf32, both operands split into hi + lo, a fresh
                                   accumulator for every 32 source bins, added in FP32 registers) */

typedef struct {
    double delta;           /* grid step > 0 */
    int32_t policy;         /* TFI_POLICY_* */
    int32_t leaf_max;       /* s0 >= 1: a call with <= s0 vertices is summed densely (s0 = 1: base case f(0) x_u) */
    int32_t max_channels;   /* largest d any apply will use (sizes the workspace) */
    int32_t flags;          /* TFI_PLAN_* */
    int32_t fft_cta_points; /* shared-memory FFT tile: points x channel pairs one CTA transforms for tables
                               below 2^13 points (4096, 8192 or 16384, i.e. 32, 64 or 128 KB of shared
                               memory; 0 = 8192). A launch-shape knob, chosen by tfi_autotune */
} tfi_options;

#define TFI_DTYPE_F32  0
#define TFI_DTYPE_BF16 1

/* Build a plan: validate and quantise the forest, run the decomposition on the
 * host (Algorithms 1 and 6 per call, iteratively), flatten it, sample f,
 * compute the kernel spectra in FP64, and (unless TFI_PLAN_HOST_ONLY) upload
 * everything and allocate the workspace on the current device. On success
 * *out owns host and device memory until tfi_destroy. The host work runs on
 * all hardware threads (std::thread::hardware_concurrency; the calls of one
 * recursion level, or the trees of a forest, in parallel) and returns the same
 * plan whatever the thread count. */
tfi_status tfi_plan(const tfi_tree *tree, const tfi_kernel *kernel, const tfi_options *opt, tfi_plan_t *out);

/* Autotuner (launch-shape and leaf-cutoff choice for a given tree and width; the
 * paper has no counterpart: its cost model picks backbones, not launch shapes).
 * For each leaf cutoff in leaf_candidates (n_leaf of them; NULL / 0 = {64, 128,
 * 256, 512, 1024}) it plans the forest with *opt and that leaf_max, and for each
 * shared-memory FFT tile (fft_cta_points 4096, 8192, 16384) times `reps` applies
 * of d channels of dtype with CUDA events on a private stream after two warm-up
 * applies; the fastest configuration is written to *tuned (a copy of *opt with
 * leaf_max and fft_cta_points set) and its time per apply to *best_ms (nullable).
 * With sample_trees > 0 and a forest of more trees, the tuning runs on its first
 * sample_trees trees (by smallest vertex) and the whole forest is planned once
 * with the winner. When plan_out is non-NULL it receives that plan (owned by the
 * caller); otherwise nothing stays allocated. Host work as in tfi_plan; device
 * fields of n x d are allocated for the timing and freed. Synchronises the device
 * work it launches. */
tfi_status tfi_autotune(const tfi_tree *tree, const tfi_kernel *kernel, const tfi_options *opt, int32_t d,
                        int32_t dtype, const int32_t *leaf_candidates, int32_t n_leaf, int32_t sample_trees,
                        int32_t reps, tfi_options *tuned, double *best_ms, tfi_plan_t *plan_out);

/* out = K F (the operator above). F, out: device, n x d, dtype; out is
 * overwritten and must not alias F. 1 <= d <= max_channels. */
tfi_status tfi_apply(tfi_plan_t plan, const void *F, void *out, int32_t d, int32_t dtype, tfi_stream_t stream);

/* grad_F = K^T grad_out. K is symmetric (f(dhat(u,v)) = f(dhat(v,u)); the
 * paper uses the same operator for K and K^T in its Sinkhorn updates), so this
 * is one more apply on grad_out. Same layout rules as tfi_apply. */
tfi_status tfi_apply_backward(tfi_plan_t plan, const void *grad_out, void *grad_F, int32_t d, int32_t dtype,
                              tfi_stream_t stream);

/* The same out = K F evaluated densely on the tensor cores: per tree of the
 * forest, out[i] = sum_j f(dhat(i, j)) F[j] with the f(D) tile generated in
 * shared memory (root distances + a range minimum over the tree's preorder)
 * and multiplied by tcgen05.mma (BF16 operands split into hi + lo parts, FP32
 * accumulation; FP32 fields use three products). Cost O(sum over trees of
 * n_T^2 d): the dense evaluation the paper compares against (runtime
 * protocol of the attention appendix), and a fast path for small trees with
 * many channels. The first call builds the per-tree preorder and sparse table
 * on the device (allocates). Synchronises `stream` before returning; a
 * tensor-core completion wait that gives up returns TFI_ERR_TIMEOUT. */
tfi_status tfi_dense_apply(tfi_plan_t plan, const void *F, void *out, int32_t d, int32_t dtype, tfi_stream_t stream);

/* As tfi_apply, with F and out in HOST memory (pinned memory gives
 * asynchronous copies). Copies F in, applies, copies out, and synchronises the
 * stream before returning. Uses plan-owned device staging buffers. */
tfi_status tfi_apply_host(tfi_plan_t plan, const void *F_host, void *out_host, int32_t d, int32_t dtype,
                          tfi_stream_t stream);

/* out_host[i] = K F_host[i] for n_fields independent fields in HOST memory,
 * pipelined: field i + 1 is copied in and field i - 1 copied out while field i
 * is applied (two plan-owned staging slots, a copy-in and a copy-out stream
 * owned by the plan, the apply on `stream`). Overlap needs pinned host memory;
 * pageable buffers give the same results without it. Each array is n x d of
 * dtype; inputs are read and outputs written during the call only, and the
 * call returns when every output is in host memory. The first call allocates
 * four n x max_channels FP32 staging buffers and the two copy streams. */
tfi_status tfi_apply_host_many(tfi_plan_t plan, int32_t n_fields, const void *const *F_host, void *const *out_host,
                               int32_t d, int32_t dtype, tfi_stream_t stream);

/* Allocation-free apply: the same result as tfi_apply, for callers that must not
 * allocate device memory while they run. That includes hosts that own all
 * device memory through their own allocator or a fixed budget and forbid
 * libraries from calling cudaMalloc, and latency-critical loops that cannot
 * absorb cudaMalloc's implicit synchronisation. The paper has no counterpart:
 * this is a deployment variant of the apply.
 *
 * Instead of the plan's workspace and per-d work lists, this call uses one
 * file-scope device array of TFI_STATIC_SCRATCH_BYTES (32 MiB) that every GPU
 * loading libtfi holds until the process exits. It calls no cudaMalloc,
 * cudaFree or other allocating routine and copies nothing from host memory:
 * the work lists it needs for this d are written into that array by a small
 * kernel on `stream` from plan-owned lists built by tfi_plan.
 *   - The first call on a device does one-time set-up with that device
 *     current: it looks up the array's device address (cudaGetSymbolAddress)
 *     and raises the kernels' shared-memory limits. Make that first call
 *     before any stream capture.
 *   - Plans whose workspace at this d (bin sums, table values, leaf terms and
 *     work items) exceeds TFI_STATIC_SCRATCH_BYTES are rejected with
 *     TFI_ERR_ARG; use tfi_apply for them. Plans with exponential-sweep or
 *     Hankel-evaluator tables are rejected with TFI_ERR_UNSUPPORTED.
 *   - All calls share the one array, which keeps the last call's contents;
 *     each call writes every value it reads before reading it, so nothing
 *     needs clearing. Calls that overlap on the GPU (other streams, other
 *     plans, other threads) race on the array: serialise them.
 * F, out, d, dtype and stream follow tfi_apply. */
#define TFI_STATIC_SCRATCH_BYTES (32u << 20)
tfi_status tfi_apply_static(tfi_plan_t plan, const void *F, void *out, int32_t d, int32_t dtype, tfi_stream_t stream);

/* CUDA-graph replay of a whole step. tfi_graph_create captures, on `stream`,
 * one apply out = K F and, when grad_out and grad_F are both non-NULL, the
 * adjoint grad_F = K grad_out, with these fixed device buffers, into one
 * instantiated CUDA graph (all calls of every tree of the forest, leaf,
 * bin-sum, table and gather launches with their stream fork / join).
 * Capture runs on a private stream after a device synchronisation, so
 * `stream` of tfi_graph_create is not used. tfi_graph_launch replays the graph
 * on `stream`; refill the input buffers in place between launches. The plan must outlive the graph, and its workspace is
 * shared with other applies of the same plan (one stream at a time). */
typedef struct tfi_graph_s *tfi_graph_t;
tfi_status tfi_graph_create(tfi_plan_t plan, const void *F, void *out, const void *grad_out, void *grad_F, int32_t d,
                            int32_t dtype, tfi_stream_t stream, tfi_graph_t *graph);
tfi_status tfi_graph_launch(tfi_graph_t graph, tfi_stream_t stream);
tfi_status tfi_graph_destroy(tfi_graph_t graph);

/* Entropic optimal transport on the tree metric (Appendix "Sinkhorn
 * Implementation Details", Eq. "app-sinkhorn-updates"): starting from
 * u = v = 1, repeat `iters` times
 *     u = a / (K v + delta_reg),   v = b / (K^T u + delta_reg)
 * with K this plan's operator (symmetric, so K^T = K). a, b, u, v: device,
 * n x d FP32, one marginal pair per channel; u, v are overwritten with the
 * scalings (the plan is diag(u) K diag(v) per channel). One iteration is
 * captured once as a CUDA graph and replayed; the call synchronises `stream`.
 * The first call allocates an n x max_channels buffer for K x. At a small eps the
 * iteration divides by entries of K v far below their maximum; plan with
 * TFI_PLAN_DIRECT_ALL then (FFT tables are accurate to their table's norm only). */
tfi_status tfi_sinkhorn(tfi_plan_t plan, const float *a, const float *b, float *u, float *v, int32_t d, int32_t iters,
                        double delta_reg, tfi_stream_t stream);

/* Gradient with respect to the kernel f (learnable kernels). out = K F is
 * linear in the grid samples f_k = f(k delta), so for a loss L with
 * grad_out = dL/dout:
 *     C[k] = dL/df_k = sum over ordered pairs (u, v) with dhat(u, v) = k of <grad_out[u], F[v]>
 * and, for the analytic kinds, dL/dtheta = sum_k (d f(k delta) / d theta) C[k]
 * (theta in the order of tfi_kernel.params). C is computed with the plan's own
 * decomposition: per table job a 2D FFT correlation of the bin sums of
 * grad_out and F (channels summed in the frequency domain), per leaf its pair
 * histogram; every sum runs in a fixed order (deterministic).
 *   grad_out, F: device, n x d, dtype. C: device FP64 array of C_len >=
 *   tfi_plan_info.hist_len entries, or NULL. dtheta: FP64 array of n_params
 *   entries, or NULL (a TFI_F_TABLE kernel has no parameters). In device memory
 *   it is written on `stream` (no synchronisation); in host memory the call
 *   synchronises `stream` to copy it back. The first call allocates the
 *   gradient workspace. A table of more than 2^13 grid points is correlated
 *   directly (pair dot products binned by distance), which takes tables of up to
 *   8160 occupied bins; a plan with a larger table of that kind returns
 *   TFI_ERR_UNSUPPORTED. */
tfi_status tfi_kernel_grad(tfi_plan_t plan, const void *grad_out, const void *F, int32_t d, int32_t dtype, double *C,
                           int64_t C_len, double *dtheta, tfi_stream_t stream);

/* Replace the plan's kernel f without replanning (e.g. a training step on
 * learnable parameters): same kind and number of parameters (or, for
 * TFI_F_TABLE, a table at least as long as the plan needs). Recomputes the
 * FP32 samples and the FP64 spectra on the host and copies them into the
 * plan's device buffers (synchronous; no allocation). A plan whose tables were
 * truncated (tfi_plan_info.trunc_len >= 0) takes only kernels whose FP32 samples
 * are zero from trunc_len on; others return TFI_ERR_UNSUPPORTED (plan again, or
 * plan with TFI_PLAN_NO_TRUNCATE). */
tfi_status tfi_set_kernel(tfi_plan_t plan, const tfi_kernel *kernel);

/* Failure-detection self-test of the bounded device wait (no counterpart in the
 * paper). Every tensor-core kernel waits for its MMAs on an mbarrier with a poll
 * limit and, when the limit runs out, records the failure in a plan-owned flag
 * and returns instead of hanging (tfi_plan_info.device_errors counts such flags).
 * This call launches one CTA that initialises an mbarrier for one arrival,
 * arrives on it only if `arrive` is non-zero, and then waits on it through the
 * same bounded wait with at most max_polls polls (1 .. 2^26; with a short sleep
 * between polls, 10^4 polls take well under a millisecond). It issues no MMA
 * and allocates no tensor memory, so a wait that runs out leaves nothing in
 * flight. Returns TFI_OK when the wait completed and TFI_ERR_TIMEOUT when it
 * gave up, in which case the plan's self-test flag stays set (counted by
 * device_errors) until the next call. Synchronises `stream`. */
tfi_status tfi_selftest_wait(tfi_plan_t plan, int32_t arrive, int32_t max_polls, tfi_stream_t stream);

/* Release everything the plan owns. NULL is accepted and ignored. */
tfi_status tfi_destroy(tfi_plan_t plan);

/* Plan statistics. */
typedef struct {
    int64_t n;              /* vertices */
    int64_t n_calls;        /* non-leaf recursive calls */
    int64_t n_leaves;       /* leaf calls (|V(S)| <= s0) */
    int64_t n_levels;       /* recursion depth + 1 */
    int64_t n_records;      /* sum over non-leaf calls of |V(S)| */
    int64_t n_keys;         /* distinct (call, depth, coordinate) and (component, depth) bins */
    int64_t n_jobs_fft;     /* cross / correction tables evaluated by FFT */
    int64_t n_jobs_direct;  /* tables evaluated by direct summation */
    int64_t n_centroid;     /* calls whose backbone is a single centroid */
    int64_t sum_table;      /* sum over non-leaf calls of (H+1)(L+1), grid units */
    int64_t sum_fft_points; /* sum over FFT jobs of P1*P2 */
    int64_t sum_leaf_pairs; /* sum over leaves of |V(S)|^2 */
    int64_t ftab_len;       /* grid samples of f held on the device */
    int64_t device_bytes;   /* device memory owned by the plan (without per-d work lists) */
    double plan_seconds;    /* host wall time of tfi_plan */
    double device_keys_ms;  /* device time of the plan-time distance / bin-key pass (0 host-only) */
    int64_t n_jobs_sweep;   /* tables evaluated by exponential sweeps (TFI_PLAN_SWEEP) */
    int64_t hist_len;       /* length of the kernel-gradient histogram (1 + largest pair distance in a call) */
    int64_t n_jobs_hankel;  /* tables evaluated by the Hankel-matrix product (TFI_PLAN_HANKEL) */
    int64_t device_errors;  /* bounded device waits that gave up since the plan was built (0 when healthy;
                               reading it synchronises the device) */
    int64_t n_jobs_fft_big; /* tables beyond one CTA's shared memory evaluated by the four-step FFT through
                               global memory (P1 P2 > 2^14 points) */
    int64_t sum_fft_big_points; /* sum over those tables of P1*P2 */
    int64_t trunc_len;      /* T of TFI_PLAN_NO_TRUNCATE's truncation (grid units), or -1 when no table was cut */
    int64_t n_zero_bins;    /* bins left out of their tables by that truncation (their values are zero) */
} tfi_plan_info;
tfi_status tfi_plan_get_info(tfi_plan_t plan, tfi_plan_info *info);

/* Export the decomposition for inspection and tests (host copies, int64).
 *   TFI_EXPORT_CALLS    7 per non-leaf call: level, min vertex, |V(S)|, kind (0 diameter, 1 centroid),
 *                       m = |V(P)|, H (grid), L = X_m (grid)
 *   TFI_EXPORT_BACKBONE backbone vertices p_1..p_m of every call, concatenated in call order
 *   TFI_EXPORT_RECORDS  5 per (call, vertex): call index, vertex, depth d(u) (grid),
 *                       coordinate X(pi(u)) (grid), component id = min vertex of the component (-1 on P)
 *   TFI_EXPORT_LEAVES   3 per leaf call: level, min vertex, |V(S)|
 *   TFI_EXPORT_DEVICE_KEYS 4 per (call, vertex), in RECORDS order: call index, vertex, and the
 *                       depth d(u) and coordinate X(pi(u)) as computed on the device at plan time
 *                       from root distances (pointer doubling over the rooted forest) and
 *                       lowest common ancestors: d(u) = D(u) + D(pi u) - 2 D(lca(u, pi u)),
 *                       X = D(p_1) + D(pi u) - 2 D(lca(p_1, pi u)) (Eq. "stad-depth",
 *                       Eq. "projection"); they must equal the host planner's bit for bit.
 *                       Needs a device plan.
 *   TFI_EXPORT_LEAF_PACKS 4 per dense leaf of at least 64 vertices, in launch order: the CTA of
 *                       the big-leaf kernel that runs it, its [begin, end) range of leaf
 *                       positions, and the CTA's vertex capacity. A CTA has 8 warps; a leaf takes
 *                       ceil(size / 64) of them, a CTA holds leaves while their warps fit in 8 and
 *                       their vertices in the capacity (largest leaf first). The paper has no
 *                       counterpart: this is a launch layout (base case of Algorithm 5).
 *   TFI_EXPORT_LEAF_CTAS 4 per dense leaf of at least 64 vertices, CTA by CTA, for the FP32
 *                       tensor-core leaf kernel: its persistent CTA, the leaf's [begin, end) range of
 *                       leaf positions, and the number of CTAs (two per SM, at most one per leaf).
 *                       Leaves are sorted largest first and each goes to the CTA with the least
 *                       work so far (work: ceil(size / 128) x ceil(size / 32) + 4); each CTA runs its
 *                       list in that order. A launch layout, with no counterpart in the paper.
 *   TFI_EXPORT_GATHER_ORDER the n vertices in the order the output gather takes them: a
 *                       depth-first preorder of the forest, tree by tree. Launch layout only.
 *   TFI_EXPORT_JOBS     7 per table job (a call's cross table or a component's correction), in plan
 *                       order: evaluator (0 FFT in shared memory, 1 direct, 2 exponential sweep,
 *                       3 Hankel product, 4 four-step FFT through global memory), log2 of the
 *                       FFT points (-1 unless an FFT), 1 for a correction, occupied bins,
 *                       the first member vertex of its first bin and the last member of its last
 *                       bin (-1 for a job without bins), and its largest depth (grid units).
 *                       Vertices named here read this job's table in the gather.
 * If dst is NULL (or cap too small) only *len (number of int64 values) is set. */
#define TFI_EXPORT_CALLS    0
#define TFI_EXPORT_BACKBONE 1
#define TFI_EXPORT_RECORDS  2
#define TFI_EXPORT_LEAVES   3
#define TFI_EXPORT_DEVICE_KEYS 4
#define TFI_EXPORT_LEAF_PACKS  5
#define TFI_EXPORT_GATHER_ORDER 6
#define TFI_EXPORT_JOBS         7
#define TFI_EXPORT_LEAF_CTAS    8
tfi_status tfi_plan_export(tfi_plan_t plan, int32_t what, int64_t *dst, int64_t cap, int64_t *len);

/* Stages of an apply, in launch order, for profiling and the roofline model:
 *   LEAF    dense leaf calls f(D_S) x_S
 *   BUCKET  segmented bin sums of field rows (A_r[t] and b_alpha[r])
 *   FFT     cross tables / corrections by shared-memory FFT correlation
 *   DIRECT  cross tables / corrections by direct summation over occupied bins
 *   GATHER  per-vertex sum over calls of G - E, plus the leaf term, one write per row
 *   SWEEP   per call, G_0 by forward and backward backbone sweeps and E_alpha[0] per
 *           component, for each exponential term (TFI_PLAN_SWEEP plans)
 *   HANKEL  cross tables / corrections by the Hankel-matrix product and antidiagonal
 *           prefix sums (TFI_PLAN_HANKEL plans) */
#define TFI_STAGE_LEAF   0
#define TFI_STAGE_BUCKET 1
#define TFI_STAGE_FFT    2
#define TFI_STAGE_DIRECT 3
#define TFI_STAGE_GATHER 4
#define TFI_STAGE_SWEEP  5   /* exponential-sum sweeps (TFI_PLAN_SWEEP plans) */
#define TFI_STAGE_HANKEL 6   /* Hankel-matrix products on tensor cores (TFI_PLAN_HANKEL plans) */
#define TFI_N_STAGES     7

/* Per-stage timing with CUDA events recorded on the stream each stage runs on.
 * enable = 1 starts recording (and clears previous totals); 2 does the same and
 * also serialises the stages of every apply on the caller's stream (no side
 * streams), so that each stage's time is its time alone on the GPU (a
 * measurement mode: results are unchanged, the apply is slower); 0 stops and
 * restores the concurrent schedule. Adds two event records per stage per apply. */
tfi_status tfi_profile_enable(tfi_plan_t plan, int32_t enable);

/* Synchronise the recorded events and return, per stage, the summed device time
 * in milliseconds and the number of kernel launches since profiling was
 * enabled. ms and launches each hold TFI_N_STAGES values. */
tfi_status tfi_profile_read(tfi_plan_t plan, double *ms, int64_t *launches);

/* Algorithmic DRAM bytes and floating-point operations of one apply, per stage,
 * for d channels of the given dtype, from the plan's exact counts (bins, records,
 * leaf pairs, FFT sizes). bytes and flops each hold TFI_N_STAGES values. */
tfi_status tfi_stage_model(tfi_plan_t plan, int32_t d, int32_t dtype, double *bytes, double *flops);

/* Message describing the last error returned on the calling thread ("" if none). */
const char *tfi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TFI_H */
