/*
 * onmf.h - C ABI of libonmf: online and batch Itakura-Saito NMF on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Lefevre, Bach, Fevotte, "Online algorithms for Nonnegative Matrix
 * Factorization with the Itakura-Saito divergence" (arXiv:1106.4198).
 *
 * Matrix conventions (all entry points):
 *   - column-major; a frame is a column. V is F x n with leading dimension
 *     ldv >= F (frame j starts at V + j*ldv). W is F x K (ld = F).
 *     A, B are F x K (ld = F). H is K x n with leading dimension ldh >= K.
 *   - V, W, H are float32. A, B and the loss sums are float64.
 *   - V must be finite and >= 0. eps (default 1e-12, Section 3) smooths the
 *     divergence: d_IS(eps + v, eps + W h) (Section 2.3).
 *
 * Pointers marked "host or device" may point to either; the library asks the
 * CUDA runtime which it is and copies host data through its own buffers.
 * The caller always owns the memory it passes in; the library owns
 * everything it allocates (state, staging, scratch) until onmf_destroy.
 *
 * Errors are returned as values; no call aborts the process. Work is
 * asynchronous on the stream given at onmf_init: an error found by a kernel
 * (invalid input, non-finite result, a device wait that ran out) is recorded
 * in a per-state error word and returned by the next call that can see it
 * (at the latest by the next call that synchronizes). Such an error is
 * sticky: the state then refuses work until onmf_set_state restores it.
 * Calls on one state are not thread-safe; distinct states are independent.
 */
#ifndef ONMF_H
#define ONMF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ONMF_ABI_VERSION 6

typedef struct onmf_state onmf_state;

typedef enum {
    ONMF_OK = 0,
    ONMF_EINVAL = 1,   /* bad argument (null pointer, size, layout, config)    */
    ONMF_ENOMEM = 2,   /* device or pinned host allocation failed               */
    ONMF_EBUDGET = 3,  /* request exceeds the memory budget (serving)           */
    ONMF_ECUDA = 4,    /* a CUDA runtime call failed                            */
    ONMF_ENUMERIC = 5, /* a kernel saw negative/NaN/Inf input or a non-finite W */
    ONMF_ETIMEOUT = 6, /* a bounded device-side wait ran out                    */
    ONMF_ESTATE = 7,   /* the state holds a sticky error or is in the wrong mode */
    ONMF_EAGAIN = 8    /* nothing ready yet / queue full (serving)              */
} onmf_status;

typedef enum {
    ONMF_FP32 = 0,  /* FP32 everywhere on the GPU; A and B in the
                       onmf_accumulate arithmetic (FP64 by default)          */
    ONMF_MIXED = 1  /* BF16 tensor-core products with FP32 accumulation, FP32
                       ratios y/x^2 and 1/x, A and B as above; K <= 256,
                       F <= 1024 (K > 128: the cluster h-solve; serving:
                       K <= 128, FP64 A and B) */
} onmf_precision;

/* Kernel of the mixed-precision h-solve (no counterpart in the paper; the
 * arithmetic is the same, the order of the sums differs):
 *   AUTO     mma for K <= 128, cluster for K > 128 (the environment variable
 *            ONMF_HSOLVE=mma|tc|cluster overrides AUTO where the shape allows);
 *   MMA      one CTA per 8-frame tile, W^T in shared memory, mma.sync (K <= 128);
 *   TC       tcgen05 with W in tensor memory, 16-frame tiles (K <= 128, F >= 128
 *            with at most 32 rows past the last 128-row tile);
 *   CLUSTER  a cluster of CTAs per 32-frame tile, W split by rows (K <= 256).
 * A choice the shape does not allow is rejected with EINVAL. onmf_autotune
 * picks one by measurement. Ignored on the FP32 path. */
typedef enum {
    ONMF_HSOLVE_AUTO = 0,
    ONMF_HSOLVE_MMA = 1,
    ONMF_HSOLVE_TC = 2,
    ONMF_HSOLVE_CLUSTER = 3
} onmf_hsolve;

/* Arithmetic of the running statistics A and B (onmf_config.accumulate).
 * Each entry takes 8 bytes on the device in every mode:
 *   FP64       a double (default);
 *   FP32       a float;
 *   FP32_COMP  a pair of floats (hi, lo) with hi = fl(hi + lo): the sum is
 *              carried to about twice float precision by error-free
 *              transformations (compensated summation).
 * onmf_get_stats and onmf_set_state convert to and from doubles. */
typedef enum {
    ONMF_ACC_FP64 = 0,
    ONMF_ACC_FP32 = 1,
    ONMF_ACC_FP32_COMP = 2
} onmf_accumulate;

/* Parameters of Algorithm 1 (Section 2.3). */
typedef struct {
    int32_t F;          /* frequency bins (rows of V and W), >= 1              */
    int32_t K;          /* dictionary size, 1..256                              */
    int32_t beta;       /* minibatch size: W is updated every beta frames       */
    int32_t n_inner;    /* multiplicative h updates per frame (fresh restart)   */
    double eps;         /* smoothing eps >= 0 (Section 2.3), default 1e-12      */
    double r;           /* forgetting base in [0, 1] ("Scaling past data")     */
    int64_t n_ref;      /* rho = r^(beta'/n_ref); n_ref <= 0 gives rho = 1      */
    double h_exponent;  /* gamma of the h update, default 0.5 (MM); 1.0 = MU    */
    int32_t normalize;  /* 1: rescale W columns to unit L1 norm (Algorithm 1)   */
    int32_t rho_on_new; /* 0: A <- rho*A + sum a (past scaled, default);
                           1: A <- A + rho*sum a (literal Algorithm 1)          */
    int32_t precision;  /* onmf_precision                                       */
    int32_t hsolve;     /* onmf_hsolve: h-solve kernel of the mixed path (0 = auto) */
    int32_t accumulate; /* onmf_accumulate: arithmetic of A and B (0 = FP64)    */
    int32_t stats_ranges; /* mma h-solve path: frame ranges per frequency tile of
                             the tcgen05 statistics (each range one partial sum
                             per entry), 0..256; 0 = automatic (frequency tiles
                             x ranges about half the CTAs); onmf_autotune
                             searches it. Ignored elsewhere.                 */
    /* Penalties (Section 2.2, "Extensions"; FP32 path and the mma h-solve of
     * the mixed path, EINVAL with the others; 0 = none):
     * h_penalty lambda >= 0 on each frame's h, lambda * log(a + sum_k h_k)
     * with a = h_penalty_a > 0 (a concave increasing psi of the column sum);
     * the h update becomes h_k <- h_k ((W^T p)_k / ((W^T q)_k +
     * lambda / (a + sum_j h_j)))^gamma (tangent majorization of psi).
     * w_penalty mu >= 0: mu * sum W, the dictionary step W = sqrt(A/(B + mu)). */
    double h_penalty;
    double h_penalty_a;
    double w_penalty;
} onmf_config;

/* Fill *cfg with the defaults for an F x K problem: beta = 1000,
 * n_inner = 10, eps = 1e-12, r = 1, n_ref = 0, h_exponent = 0.5,
 * normalize = 1, rho_on_new = 0, precision = ONMF_FP32, hsolve = AUTO,
 * accumulate = FP64, no penalties (h_penalty = 0, h_penalty_a = 1,
 * w_penalty = 0). */
void onmf_config_default(onmf_config *cfg, int32_t F, int32_t K);

/* Create an online state (Algorithm 1, "Input": W^(0), A^(0) = B^(0) = 0).
 *   W0: F x K initial dictionary, host or device (W0_on_device is ignored
 *       and kept for ABI stability; the pointer kind is detected). It is
 *       copied; W0 entries must be finite and >= 0.
 *   stream: a cudaStream_t (NULL = the legacy default stream) on which every
 *       later call of this state runs.
 * Allocates the device state (W, A, B, the running loss), a beta-frame
 * staging buffer and the scratch of the step kernels.
 * Errors: EINVAL (config out of range, W0 NULL), ENOMEM, ECUDA. */
onmf_status onmf_init(const onmf_config *cfg, const float *W0,
                      int32_t W0_on_device, void *stream, onmf_state **out);

/* Append n frames and run one step of Algorithm 1 for every minibatch of
 * beta frames that becomes complete (draw v_t, solve h_t with W fixed,
 * accumulate a^(t), b^(t), then A, B and W = sqrt(A/B) with the L1 rescale;
 * Algorithm 1, Section 2.3 "Mini-batch", "Scaling past data").
 *   V: F x n, leading dimension ldv >= F, host or device.
 *   H_out: NULL, or K x n with ldh >= K (host or device) that receives h_t of
 *       every frame. Frames that stay in the staging buffer get their h
 *       written when their minibatch runs (a later push or onmf_flush), so
 *       H_out must stay valid until then.
 * Asynchronous on the state's stream; V (if on the device) must stay valid
 * until the stream reaches this call. Host V goes through a two-slot device
 * ring filled on a private copy stream, so the transfer of one slot overlaps
 * the steps on the other (page-locked V is read by a small copy kernel
 * through its mapped address, pageable V goes through the copy engine):
 * pageable host V may be reused as soon as the call returns, page-locked
 * host V must stay unchanged until the state's stream reaches this call
 * (onmf_synchronize). n = 0 is a no-op.
 * Errors: EINVAL, ESTATE (sticky error), ECUDA; kernel-detected input errors
 * surface later as ENUMERIC. */
onmf_status onmf_push_frames(onmf_state *s, const float *V, int64_t ldv,
                             int64_t n, float *H_out, int64_t ldh);

/* Warm restarts over a finite data set (Section 2.3, "Fresh or warm
 * restarts" and "Finite data sets"): one pass of Algorithm 1 over the frames
 * V[order[0]], V[order[1]], ..., V[order[n-1]] in that order, where each
 * frame's h-solve starts from its kept activation H[order[i]] (instead of
 * the fresh-restart point) and the final h is written back there; the
 * config's n_inner applies (the paper takes a single update per visit). A
 * caller that permutes the frames anew for every pass passes a new order.
 *   V: device, frame rows of F floats, ld ldv >= F (the whole data set).
 *   order: device int64 array of n row indices, or NULL for rows 0..n-1.
 *   H: device, frame rows of K floats, ld ldh >= K, read and written.
 * Frames are grouped into minibatches in pass order; a trailing partial
 * minibatch waits in the staging buffer for the next warm push with the
 * same H, or for onmf_flush. The kept activations are not rescaled with W.
 * Errors: EINVAL (host pointers, sizes), ESTATE (frames of a fresh push are
 * staged, or staged warm frames belong to another H), ECUDA. */
onmf_status onmf_push_frames_warm(onmf_state *s, const float *V, int64_t ldv, int64_t n,
                                  const int64_t *order, float *H, int64_t ldh);

/* Run the partial minibatch left in the staging buffer (beta' < beta frames,
 * rho = r^(beta'/n_ref)). No-op when the buffer is empty. */
onmf_status onmf_flush(onmf_state *s);

/* Wait for all queued work of the state and return its error status. */
onmf_status onmf_synchronize(onmf_state *s);

/* Copy the current dictionary W (F x K, normalized as Algorithm 1 leaves
 * it) to W_out (host or device). Synchronizes the state's stream. */
onmf_status onmf_get_W(onmf_state *s, float *W_out, int32_t on_device);

/* Copy the sufficient statistics and counters to host memory. Any pointer
 * may be NULL. A, B: F x K float64 (Eq. aux_fun, accumulated as in
 * Algorithm 1 in the state's onmf_accumulate arithmetic and converted to
 * double; device pointers are taken only with ONMF_ACC_FP64, else EINVAL).
 * t: frames processed by completed minibatches. loss_sum:
 * running sum of d_IS(eps + v_t, eps + W h_t) over those frames (the online
 * loss of Eq. online_loss times t). Synchronizes. */
onmf_status onmf_get_stats(onmf_state *s, double *A, double *B, int64_t *t,
                           double *loss_sum);

/* Restore a state (checkpoint/resume). W: F x K float32, A, B: F x K
 * float64, all host memory (device pointers: EINVAL); t and loss_sum as
 * returned by onmf_get_stats. A and B are rounded to the state's
 * onmf_accumulate arithmetic (a float pair holds a double to about 2^-48).
 * Clears the staging buffer and any sticky error. Synchronizes. */
onmf_status onmf_set_state(onmf_state *s, const float *W, const double *A,
                           const double *B, int64_t t, double loss_sum);

/* Project n frames on the current W without changing the state: the h-solve
 * of Algorithm 1 (fresh restart, n_inner multiplicative steps; n_inner < 0
 * uses the config's value). Used for held-out evaluation (Section 3).
 *   V: F x n (ldv), host or device.  H_out: K x n (ldh), host or device.
 *   obj_sum: NULL, or a host double that receives
 *       sum_n d_IS(eps + v_n, eps + W h_n) (synchronizes when non-NULL). */
onmf_status onmf_project(onmf_state *s, const float *V, int64_t ldv, int64_t n,
                         float *H_out, int64_t ldh, int32_t n_inner,
                         double *obj_sum);

/* Batch IS-NMF (Section 2.1): n_iter cycles, each updating all of H with W
 * fixed (the h update of the online solver, applied once to every column),
 * then W <- W o sqrt((P H^T)/(Q H^T)) (= sqrt(A/B) of Eq. aux_fun, with
 * P = Y/X^2, Q = 1/X, X = eps + W H), then, if normalize, W_:k /= s_k and
 * H_k: *= s_k with s_k = sum_f W_fk.
 *   V: F x N (ldv) on the device. W: F x K (ld F) and H: K x N (ld K) on the
 *   device, updated in place. obj_out: NULL or n_iter host doubles that
 *   receive the objective (1/N) sum_n d_IS(eps+v_n, eps+W h_n) after each
 *   cycle (synchronizes when non-NULL).
 *   stream: cudaStream_t (NULL = legacy default stream).
 * Takes its scratch from the stream's memory pool for the call and returns
 * it in stream order (cudaMallocAsync / cudaFreeAsync); to run cycles with
 * no allocation at all, make a plan once (nmf_batch_plan_create) and call
 * nmf_batch_plan_step. */
onmf_status nmf_batch_step(const float *V, int64_t ldv, float *W, float *H,
                           int32_t F, int32_t K, int64_t N, double eps,
                           double h_exponent, int32_t n_iter, int32_t normalize,
                           int32_t precision, double *obj_out, void *stream);

/* Scratch of batch IS-NMF cycles (Section 2.1) for one shape, allocated once
 * on the current device: the derived images of W, the P, Q, H operands of
 * the W step for up to N_max frames, the split statistics, the loss slots.
 * About (2 or 4 bytes) x N_max x (2 F + K) plus O(F K). Synchronizes.
 * Destroy with nmf_batch_plan_destroy (synchronizes the device first). */
typedef struct nmf_batch_plan nmf_batch_plan;
onmf_status nmf_batch_plan_create(int32_t F, int32_t K, int64_t N_max,
                                  int32_t precision, nmf_batch_plan **out);

/* nmf_batch_step on a plan: the same cycles, kernels and results, for N <=
 * N_max frames on the plan's device, with no allocation or free (the per-call
 * objective buffer of nmf_batch_step lives in the plan). Asynchronous unless
 * obj_out is given. Calls on one plan must not overlap on the GPU. */
onmf_status nmf_batch_plan_step(nmf_batch_plan *plan, const float *V,
                                int64_t ldv, float *W, float *H, int64_t N,
                                double eps, double h_exponent, int32_t n_iter,
                                int32_t normalize, double *obj_out,
                                void *stream);

void nmf_batch_plan_destroy(nmf_batch_plan *plan);

/* Batch start point for H: every column gets the fresh-restart value
 * sum_f (eps + V_fn) / sum_{f,k} W_fk. V, W, H on the device. */
onmf_status nmf_batch_init_H(const float *V, int64_t ldv, const float *W,
                             float *H, int32_t F, int32_t K, int64_t N,
                             double eps, void *stream);

/* Size of the fixed device scratch array used by onmf_project_static. */
#define ONMF_STATIC_SCRATCH_BYTES (4u << 20)

/* Bits a kernel ORs into a device error word (onmf_project_static's err_out):
 * INPUT    a frame value was negative, NaN or Inf (the h of that tile is
 *          meaningless);
 * NUMERIC  a result was not finite;
 * TIMEOUT  a bounded device-side wait ran out (2 s) and the kernel left early,
 *          so outputs may be unwritten;
 * CONFIG   a kernel was launched with a shape it cannot run (cluster size) and
 *          returned at entry without writing its outputs. */
#define ONMF_DEVERR_INPUT 1
#define ONMF_DEVERR_NUMERIC 2
#define ONMF_DEVERR_TIMEOUT 4
#define ONMF_DEVERR_CONFIG 8

/* Projection (the h-solve of onmf_project, same kernels and results) for
 * callers that cannot allocate device memory: code running in a real-time
 * audio callback, where cudaMalloc may stall on a device-wide
 * synchronization, or inside a host that gives the library a fixed memory
 * arena. The paper has no counterpart; this is a deployment variant.
 *   W: F x K dictionary (device, ld F). V: F x n frames (device, ldv >= F).
 *   H_out: K x n (device, ldh >= K) or NULL. obj_sum: NULL or a device double
 *   that receives sum_n d_IS(eps + v_n, eps + W h_n). precision: onmf_precision.
 *   err_out: NULL or a device int32 that the call clears and the kernels OR
 *   their ONMF_DEVERR_* bits into; read it after the stream reaches the end
 *   of the call (0: every output was written from valid input). With NULL
 *   the bits go to the scratch array and are lost.
 *   stream: cudaStream_t (NULL = legacy default stream).
 * Allocates nothing: its scratch lives in one static device array of
 * ONMF_STATIC_SCRATCH_BYTES (4 MiB) that every GPU loading the library keeps
 * until the process exits. A call whose scratch would not fit returns
 * ONMF_EINVAL. With a(x) = x rounded up to a multiple of 256, Kp = K rounded
 * up to 16 and Fp = F rounded up to 16, the need in bytes is
 *   FP32 (any K):         a(4 F K) + a(4 K) + 8 ceil(n / 8);
 *   mixed, K <= 128:      a(2 Kp (Fp + 8)) + a(4 K) + 8 ceil(n / 8)
 *                         (with ONMF_HSOLVE=tc in the environment:
 *                         a(2 Kp (Fp + 8)) + a(2 F Kp) + a(4 K) + 8 ceil(n / 16));
 *   mixed, K > 128:       a(2 F Kp) + a(4 K) + 8 C ceil(n / 32), C the
 *                         cluster size (1, 2, 4 or 8; at most 8);
 * and it must not exceed ONMF_STATIC_SCRATCH_BYTES - 256 (F = 513, K = 100
 * leaves room for about 4 million frames per call in FP32). All calls share
 * the array: calls that run at the same time on the GPU (different streams or
 * threads) race and must be serialized by the caller. The first call on each
 * device looks up the array's device address (and sets kernel attributes);
 * make that first call before any stream capture. Asynchronous. */
onmf_status onmf_project_static(const float *W, int32_t F, int32_t K,
                                const float *V, int64_t ldv, int64_t n,
                                float *H_out, int64_t ldh, double eps,
                                double h_exponent, int32_t n_inner,
                                int32_t precision, double *obj_sum,
                                int32_t *err_out, void *stream);

/* Release the state and everything the library allocated for it. */
void onmf_destroy(onmf_state *s);

/* ------------------------------------------------------------------ serving
 * Many concurrent streams, each its own run of Algorithm 1 (own W, A, B),
 * fed chunk by chunk. Every chunk is one minibatch of that stream (beta' =
 * chunk length, rho = r^(beta'/n_ref)): h-solve with the stream's W, then
 * the statistics and the dictionary step. A worker thread batches the
 * queued chunks of all admitted streams that have no chunk on the GPU
 * (continuous batching: chunks that arrive while a batch runs join the next
 * one, and up to `slots` batches are in flight on separate CUDA streams).
 * A batch runs as three phases over all its (chunk, work unit) pairs: the
 * h-solve of every 8-frame tile (one launch for every dictionary size in
 * the batch; the environment variable ONMF_SERVE_FORK=1 selects one launch
 * per size on forked streams instead), the statistics of every output tile,
 * the rescale of every column. By default the phases of a batch are one
 * CUDA graph launch: the graph is captured once per slot and reads the
 * batch's layout from device memory, so a batch needs no capture or update
 * whatever dictionary sizes it mixes. Every
 * work unit is computed in a fixed order of operations, so a chunk's result
 * does not depend on what it is batched with. Streams are admitted by a
 * device-memory budget: a stream whose state does not fit waits (its chunks
 * queue) until closed streams free memory. */

/* How a serving batch is launched (onmf_server_config.launch). */
typedef enum {
    ONMF_SERVE_GRAPH = 0,  /* replay a captured CUDA graph (default)        */
    ONMF_SERVE_DIRECT = 1  /* launch the phase kernels one by one           */
} onmf_serve_launch;

typedef struct onmf_server onmf_server;

typedef struct {
    int32_t F;              /* frequency bins shared by all streams          */
    int32_t max_chunk;      /* largest chunk in frames (<= 4096)             */
    int32_t max_batch;      /* chunks per launch                             */
    int32_t slots;          /* batches in flight (1..4)                      */
    int64_t budget_bytes;   /* device memory for stream states               */
    int32_t precision;      /* onmf_precision for all streams                */
    int32_t launch;         /* onmf_serve_launch                             */
} onmf_server_config;

typedef struct {
    int64_t stream_id;
    int64_t tag;            /* the caller's tag from onmf_server_submit      */
    int64_t frames;
    double loss;            /* sum of d_IS(eps+v, eps+W h) over the chunk    */
    double t_submit;        /* seconds, CLOCK_MONOTONIC, at submit           */
    double t_done;          /* seconds, when the worker saw the result ready */
    int32_t status;         /* onmf_status of this chunk                     */
    int32_t reserved;
} onmf_completion;

typedef struct {
    int64_t launches, chunks, frames, batches_overlapped;
    int64_t streams_admitted, streams_pending, bytes_in_use;
    int64_t host_batch_ns;  /* worker time forming batches (items, offsets)    */
    int64_t device_ns;      /* sum over batches of device time from the first
                               copy to the last (slots overlap, so this can
                               exceed the wall time)                          */
} onmf_server_stats;

/* Create a server (allocates the per-slot device buffers; the budget covers
 * only stream states). Errors: EINVAL, ENOMEM, ECUDA. */
onmf_status onmf_server_create(const onmf_server_config *cfg, onmf_server **out);

/* Open a stream with its own parameters (cfg->F must equal the server's F;
 * K <= 128; hsolve AUTO or MMA; accumulate FP64; no penalties; cfg->beta is ignored:
 * chunks are the minibatches) and initial
 * dictionary W0 (F x K, host). Returns its id; the stream is admitted now if
 * its state fits the budget, else it waits in FIFO order. */
onmf_status onmf_server_open_stream(onmf_server *srv, const onmf_config *cfg,
                                    const float *W0, int64_t *stream_id);

/* Queue a chunk of n frames (F x n host memory, leading dimension ldv) for
 * a stream; the frames are copied before the call returns. H_out: NULL or
 * host memory K x n (ld K) that receives the chunk's h when it completes.
 * Errors: EINVAL (n < 1, n > max_chunk, unknown or closing stream),
 * ESTATE (an earlier chunk of the stream failed), ENOMEM (host memory). */
onmf_status onmf_server_submit(onmf_server *srv, int64_t stream_id,
                               const float *V, int64_t ldv, int64_t n,
                               float *H_out, int64_t tag);

/* Queue several chunks in one call, each under the rules of
 * onmf_server_submit: chunk i is stream_ids[i], V[i] (F x n[i] host memory,
 * leading dimension ldv[i]), H_out[i] (NULL, or host K x n[i]; H_out itself
 * may be NULL: no h for any chunk) and tags[i]. Chunks of one stream run in
 * the order given. Stops at the first chunk that is refused and returns its
 * status; *queued (may be NULL) receives how many were queued. */
onmf_status onmf_server_submit_many(onmf_server *srv, int32_t count, const int64_t *stream_ids,
                                    const float *const *V, const int64_t *ldv, const int64_t *n,
                                    float *const *H_out, const int64_t *tags, int32_t *queued);

/* Take up to max completions (oldest first), waiting up to wait_ms for the
 * first one. *count receives how many were written (0 on timeout). */
onmf_status onmf_server_poll(onmf_server *srv, onmf_completion *out,
                             int32_t max, int32_t *count, int32_t wait_ms);

/* Copy a stream's current W (F x K, host) once its queued chunks are done. */
onmf_status onmf_server_get_W(onmf_server *srv, int64_t stream_id, float *W_out);

/* Close a stream after its queued chunks complete; frees its device memory
 * and admits waiting streams. */
onmf_status onmf_server_close_stream(onmf_server *srv, int64_t stream_id);

onmf_status onmf_server_get_stats(onmf_server *srv, onmf_server_stats *out);

/* Stop the worker (after the work already queued) and free everything. */
void onmf_server_destroy(onmf_server *srv);

/* Static string naming a status. */
const char *onmf_status_string(onmf_status st);

/* Text of the last CUDA failure seen by this thread ("" if none). */
const char *onmf_last_error_message(void);

/* Number of kernel launches this process has issued through the library
 * (all states), for launch accounting in benchmarks. */
int64_t onmf_kernel_launches(void);

/* Fault-path self-test (no counterpart in the paper). Runs one of the
 * library's bounded device waits on a condition that never holds, on a
 * two-CTA launch on `stream` (a cudaStream_t, NULL = legacy default):
 *   which 0: the grid barrier of the persistent step kernel, told to expect
 *            one CTA more than the grid has;
 *   which 1: an mbarrier phase that nothing arrives on;
 *   which 2: as 1, while the CTA holds tensor memory, freed before it returns.
 * Each wait gives up after its limit (2 s), flags a timeout and leaves the
 * kernel; the CUDA context stays usable. Blocks until the stream drains.
 * elapsed_ns (may be NULL) receives the device time from kernel start to the
 * first CTA's exit.
 * Returns ETIMEOUT when the wait ran out as designed, OK if it did not,
 * EINVAL (which out of range), ENOMEM, ECUDA. */
onmf_status onmf_selftest_wait(int32_t which, void *stream, int64_t *elapsed_ns);

/* Autotuner (no counterpart in the paper): time every schedule of the
 * mixed-precision online step that the shape in *cfg allows (cfg->hsolve and
 * cfg->stats_ranges are ignored) on a synthetic stream of 23 minibatches on
 * `stream` (3 warm-up, 20 timed with CUDA events) and return the fastest.
 * The candidates are the h-solve kernels, which fix the frames per tile
 * (mma 8, tcgen05 16, cluster 32), and with the mma kernel the frame ranges
 * of the tcgen05 statistics, stats_ranges in {0 (automatic), 2, 4, 8, 16}.
 *   hsolve_out: the kernel (ONMF_HSOLVE_*); stats_ranges_out: NULL or its
 *       statistics schedule (for onmf_config.stats_ranges).
 *   cache_path: NULL, or a file of JSON lines keyed by the device name, F,
 *       K, beta and n_inner (each line also records tile_frames); a hit
 *       returns the stored choice without timing (*from_cache = 1), a miss
 *       appends the new result.
 *   us_out: NULL or 4 doubles, the best microseconds per minibatch of each
 *       kernel, indexed by ONMF_HSOLVE_* (-1 for kernels not timed).
 *   ranges_us_out: NULL or 5 doubles, the mma kernel's time for each
 *       stats_ranges candidate in the order above (-1 if not timed).
 * On the FP32 path it returns AUTO without timing. Blocks until done.
 * A kernel whose run ends with an error that leaves the CUDA context usable
 * (a device wait that timed out, a launch its entry check refused) is left
 * out of the choice, its time -1; a context error ends the call.
 * Errors: EINVAL (no kernel fits the shape), ENOMEM, ECUDA, ETIMEOUT (every
 * kernel that fits failed: the status of the last one). */
onmf_status onmf_autotune(const onmf_config *cfg, void *stream, const char *cache_path,
                          int32_t *hsolve_out, int32_t *stats_ranges_out, double *us_out,
                          double *ranges_us_out, int32_t *from_cache);

/* ABI version (ONMF_ABI_VERSION). */
int32_t onmf_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ONMF_H */
