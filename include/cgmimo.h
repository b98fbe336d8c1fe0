/*
 * cgmimo.h - C ABI of libcgmimo: conjugate-gradient (CG) soft-output MMSE
 * detection and CG precoding for massive MIMO on one NVIDIA GB300 (sm_103a).
 *
 * The method is Algorithm 1 of Yin, Wu, Cavallaro and Studer, "Conjugate
 * Gradient-based Soft-Output Detection and Precoding in Massive MIMO Systems"
 * (arXiv 1404.0424), run in bulk: one CG solve per (instance, right-hand
 * side). An instance is one subcarrier: a channel H shared by R right-hand
 * sides (OFDM symbols). The paper's comparison methods are offered beside
 * it: CG least squares (Sec. III-E, amul_mode CG_AMUL_CGLS) and the
 * truncated Neumann series (Sec. III-F, cg_neumann_detect/cg_neumann_precode).
 *
 * Data layout (row-major, no padding, little-endian):
 *   complex values are complex64: interleaved (re, im) float32 pairs;
 *   H      [n][B][U]  uplink channel H_u of Eq. 1 (the downlink uses H_d = H_u^H);
 *   Y      [n][R][B]  receive vectors y of Eq. 1;
 *   T      [n][R][U]  precoder input symbols t of Eq. 5;
 *   xhat   [n][R][U]  x_hat_K = v_K (Algorithm 1, detection output);
 *   mu,rho [n][R][U]  float32 mu_{i|K}, rho_{i|K} (Sec. III-C);
 *   llr    [n][R][U][qam_bits] float32 max-log LLRs of Eq. 4, bit b_0 first;
 *   q      [n][R][B]  precoded vectors q_K = H_d^H v_K (Algorithm 1, precoding output);
 *   qnorm  [n][R]     float32 ||q_K||_2;
 *   status [n]        int32 bitwise OR of CG_STATUS_* over the instance's right-hand sides.
 *
 * Constellation: square Gray QAM with E|x|^2 = Es. Bits b_0..b_{q/2-1} pick
 * the in-phase level and b_{q/2}..b_{q-1} the quadrature level, each read
 * MSB-first as the Gray code j ^ (j >> 1) of the level index j; level j is
 * (2j - (L-1)) c sqrt(Es) with L = 2^(q/2) and c = sqrt(3 / (2 (M - 1))).
 * LLR sign follows Eq. 4 as printed: L > 0 favours bit 1.
 *
 * Memory and streams: every pointer argument of cg_detect / cg_precode is a
 * DEVICE pointer owned by the caller; the library keeps no reference after
 * the call returns. Work is enqueued asynchronously on `stream` (a
 * cudaStream_t; NULL is the legacy default stream) on the current device.
 * The *_host variants take HOST pointers (pinned memory gives the best
 * bandwidth), stage through a library-owned device workspace and return
 * after the results are back in host memory.
 *
 * Errors: functions return CG_OK (0) or a negative CG_E* code and enqueue no
 * work on error; cg_strerror() names the code. Argument checks happen on the
 * host before any CUDA call. Per-instance numerical conditions are reported
 * in `status`, never as a return code.
 */
#ifndef CGMIMO_H
#define CGMIMO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define CG_OK 0
#define CG_EINVAL (-1)     /* invalid argument (size, mode, pointer or alignment) */
#define CG_ECUDA (-2)      /* a CUDA runtime call or kernel launch failed */
#define CG_ENOMEM (-3)     /* device or pinned-host allocation failed */
#define CG_EAGAIN (-4)     /* resource temporarily full (serving queue) */
#define CG_ETIMEDOUT (-5)  /* a bounded wait expired */
#define CG_ENOTSUP (-6)    /* valid but unsupported combination of modes */
#define CG_ETOOBIG (-7)    /* request exceeds a fixed capacity (cg_batch_run_static,
                              or a served request larger than the HBM budget) */

/* Per-instance status bits. */
#define CG_STATUS_BREAKDOWN 1  /* CG stopped before K: ||r_{k-1}||^2 or Re(p^H A p) not > 0 */
#define CG_STATUS_MU_NONPOS 2  /* some mu_{i|K} <= 0: that user's LLRs are set to 0 */
#define CG_STATUS_TIMEOUT 4    /* an input copy did not complete in time (FP32 kernels
                                  and TMA-staged CG-D, cg_set_wait_limit); outputs not
                                  written */

/* SINR tracker (Sec. III-C). */
#define CG_SINR_APPROX 0  /* Eqs. 11-13: diagonal recursion, rho = G_ii / N0 */
#define CG_SINR_EXACT 1   /* Eq. 10 and the B = L_K G, C = B L_K^H expressions */

/* How e = A p is formed inside the CG iterations of Algorithm 1.
 * CG_AMUL_IMPLICIT forms no Gram: each product costs 2 B U complex
 * multiply-adds per right-hand side, done in FP32 on the CUDA cores whatever
 * the precision field says (there is no Gram, and the matched filter is an
 * FP32 sum). It does not combine with
 * CG_SINR_EXACT (CG_ENOTSUP), whose expressions need the Gram.
 * CG_AMUL_AUTO picks the implicit product on the FP32 path when it is the
 * cheaper one, 4 K R < U + 1 (the Hermitian Gram costs B U (U + 1) / 2 per
 * instance), and the explicit Gram otherwise and on the tensor-core paths.
 * The batched and serving entry points always form the Gram. */
#define CG_AMUL_AUTO 0      /* library choice (above) */
#define CG_AMUL_EXPLICIT 1  /* form A = H^H H + (N0/Es) I once per instance */
#define CG_AMUL_IMPLICIT 2  /* e = H^H (H p) + (N0/Es) p, two matrix-vector products */
/* CG least squares (Sec. III-E) in place of Algorithm 1: detection solves
 * min || [y; 0] - [H; sqrt(N0/Es) I] x ||, precoding min || t - [H^H, sqrt(N0/Es) I] x ||
 * with q = the first B entries of x, both by K CGLS iterations from x = 0,
 * in FP32 on the CUDA cores whatever the precision field says, with no Gram.
 * Detection keeps the approximate tracker (Eqs. 11-13) on CGLS's step sizes,
 * which equal CG's in exact arithmetic; in precoding CGLS minimises the
 * residual, so its iterates differ from CG-P's before K = U. Not with
 * CG_SINR_EXACT (CG_ENOTSUP). For cg_detect, cg_precode and their host
 * variants; the batched and serving entry points always form the Gram. */
#define CG_AMUL_CGLS 3

/* Arithmetic of the Gram H^H H and matched filter H^H y; on the tensor-core
 * paths the products A p and q = H v use the same operands (the CG vectors,
 * step sizes and sums are FP32 in every mode). */
#define CG_PREC_FP32 0
#define CG_PREC_BF16 1    /* one BF16 tensor-core pass, FP32 accumulate */
#define CG_PREC_FP16 2    /* one FP16 tensor-core pass, FP32 accumulate */
#define CG_PREC_BF16X3 3  /* hi+lo split BF16, three tensor-core passes */
#define CG_PREC_FP16X3 4  /* hi+lo split FP16, three tensor-core passes */

/* Size limits of one call. */
#define CG_U_MAX 32
#define CG_B_MAX 256
#define CG_R_MAX 16
#define CG_K_MAX 32

/* Problem description shared by every instance of one call.
 *   B         base-station antennas, U <= B <= CG_B_MAX (Sec. II)
 *   U         users, 1 <= U <= CG_U_MAX
 *   qam_bits  bits per symbol q, one of 2, 4, 6, 8 (QPSK..256-QAM)
 *   K         CG iterations, 1 <= K <= U (CG is exact at K = U, Sec. III-B)
 *   R         right-hand sides per instance, 1 <= R <= CG_R_MAX
 *   N0, Es    noise variance and symbol energy, finite and > 0; the
 *             regulariser is N0/Es (rho_u^-1 of Eq. 2, rho_d^-1 of Eq. 6)
 *   sinr_mode CG_SINR_*; amul_mode CG_AMUL_*; precision CG_PREC_*          */
typedef struct cg_params {
  int32_t B, U, qam_bits, K, R;
  float N0, Es;
  int32_t sinr_mode;
  int32_t amul_mode;
  int32_t precision;
} cg_params;

/* CG-D soft-output detection (Sec. III-B, Algorithm 1 with the SINR tracker):
 * b = H^H y, A = H^H H + (N0/Es) I, K CG iterations, the chosen SINR tracker,
 * then x_hat, mu, rho and max-log LLRs (Eq. 4). H and Y must be 8-byte
 * aligned; any of xhat, mu, rho, llr, status may be NULL (not written).
 * n_inst = 0 is a no-op. */
int cg_detect(const cg_params* p, int64_t n_inst, const void* H, const void* Y,
              void* xhat, float* mu, float* rho, float* llr, int32_t* status,
              void* stream);

/* CG-P precoding (Sec. III-D): b = t, A = H_d H_d^H + (N0/Es) I with
 * H_d = H_u^H, K CG iterations, q = H_d^H v_K (Sec. III-D).
 * With normalize != 0 the power-normalised s = q / ||q||_2 (Sec. II-B) is
 * written to q instead. qnorm and status may be NULL. The sinr_mode and
 * qam_bits fields are ignored. */
int cg_precode(const cg_params* p, int64_t n_inst, const void* H, const void* T,
               void* q, float* qnorm, int32_t normalize, int32_t* status,
               void* stream);

/* Host-memory variants of the two calls above: same arguments and layouts,
 * but every array is in HOST memory. Inputs are copied in chunks to a
 * device workspace owned by the library (allocated on first use, grown as
 * needed, freed by cg_release_workspace), processed, and copied back;
 * copies of one chunk overlap the compute of the next. Blocking: returns
 * once all outputs are in host memory. `stream` orders the work after
 * earlier work on that stream. */
int cg_detect_host(const cg_params* p, int64_t n_inst, const void* H, const void* Y,
                   void* xhat, float* mu, float* rho, float* llr, int32_t* status,
                   void* stream);
int cg_precode_host(const cg_params* p, int64_t n_inst, const void* H, const void* T,
                    void* q, float* qnorm, int32_t normalize, int32_t* status,
                    void* stream);

/* ------------------------------------------------------------------------
 * Neumann-series detection and precoding (Sec. III-F), a comparator
 * ------------------------------------------------------------------------ */

/* Largest number of Neumann terms. */
#define CG_NEUMANN_K_MAX 16

/* The truncated K-term Neumann series of Sec. III-F,
 *   A^-1 ~ sum_{k=0}^{K-1} (-D^-1 E)^k D^-1,  A = D + E,  D = diag(A),
 * applied to b = H^H y (detection: x_hat) or to t (precoding: q = H v, with
 * ||q|| and the optional normalisation of cg_precode), on the same Gram and
 * tensor-core staging as CG. The series converges when A is strongly
 * diagonally dominant (B >> U); K terms cost K - 1 products A v.
 * Arguments, layouts, ownership and errors follow cg_detect / cg_precode,
 * except:
 *   K         number of terms, 1 <= K <= CG_NEUMANN_K_MAX (not bounded by U);
 *   precision CG_PREC_BF16, CG_PREC_FP16, CG_PREC_BF16X3 or CG_PREC_FP16X3;
 *             CG_PREC_FP32 returns CG_ENOTSUP;
 *   sinr_mode and amul_mode are ignored; qam_bits must be valid but is unused;
 *   detection writes x_hat only (required): the paper's soft outputs are
 *   those of CG; status is written as 0. */
int cg_neumann_detect(const cg_params* p, int64_t n_inst, const void* H, const void* Y,
                      void* xhat, int32_t* status, void* stream);
int cg_neumann_precode(const cg_params* p, int64_t n_inst, const void* H, const void* T,
                       void* q, float* qnorm, int32_t normalize, int32_t* status,
                       void* stream);

/* ------------------------------------------------------------------------
 * Batched uneven problems (one plan, one CUDA-graph launch per run)
 * ------------------------------------------------------------------------ */

#define CG_OP_DETECT 0
#define CG_OP_PRECODE 1

/* One problem of a batch: n_inst instances of one shape, with its own
 * parameters and its own DEVICE buffers in the layouts above.
 *   op = CG_OP_DETECT:  in = Y, out = xhat, mu, rho, aux = llr  (NULL = not written)
 *   op = CG_OP_PRECODE: in = T, out = q (required), aux = qnorm; mu, rho unused;
 *                       normalize selects s = q / ||q||.
 * B, U, R, K, qam_bits, N0, Es and sinr_mode follow cg_params. */
typedef struct cg_desc {
  int32_t op, B, U, R, K, qam_bits, sinr_mode, normalize;
  float N0, Es;
  int64_t n_inst;
  const void* H;
  const void* in;
  void* out;
  float* mu;
  float* rho;
  float* aux;
  int32_t* status;
} cg_desc;

/* Precision value for plans: let the autotuner pick the schedule and the
 * split precision (CG_PREC_FP16X3 or CG_PREC_BF16X3, both FP32-accurate). */
#define CG_PREC_AUTO (-1)

typedef struct cg_plan cg_plan;

/* Builds a plan for n problems (descs is a HOST array; the library keeps a
 * device copy, so the descriptor memory may be reused after the call).
 * Problems are grouped into bins by operation, padded user count and
 * tracker; each bin runs one persistent fused kernel whose warps claim
 * (problem, instance) work units from a device counter, so uneven problems
 * balance across SMs. All bins are captured once into a CUDA graph and
 * replayed by cg_plan_run; creation is ordered after earlier work on
 * `stream`. precision is a CG_PREC_* tensor-core value (the default
 * schedule: longest units first, bins side by side, full grids) or
 * CG_PREC_AUTO, for which the schedule autotuner times its candidates on
 * the batch itself (claim order, bins side by side or one after another,
 * grid share, split precision; these runs write the outputs) and keeps the
 * fastest per device and shape class for later plans (cg_tune_cache_*).
 * The plan owns its device memory until cg_plan_destroy. The buffers named
 * by the descriptors must stay valid while the plan is used. Returns
 * CG_EINVAL for an invalid descriptor (the first bad index is reported in
 * *bad_index if non-NULL). */
int cg_plan_create(const cg_desc* descs, int64_t n, int32_t precision, void* stream,
                   cg_plan** plan, int64_t* bad_index);

/* Enqueues one run of the plan on `stream` (a single graph launch). */
int cg_plan_run(cg_plan* plan, void* stream);

/* Precision chosen for the plan (after autotuning) and the number of bins. */
int cg_plan_info(const cg_plan* plan, int32_t* precision, int32_t* n_bins);

/* How a plan runs its bins (cg_plan_schedule). */
#define CG_TUNE_FIXED 0   /* precision given: the default schedule */
#define CG_TUNE_TIMED 1   /* CG_PREC_AUTO: timed on this batch now */
#define CG_TUNE_CACHED 2  /* CG_PREC_AUTO: taken from the autotuner's cache */
typedef struct cg_schedule {
  int32_t precision;   /* CG_PREC_* the plan runs */
  int32_t order;       /* 0: work units claimed in descriptor order; 1: longest first */
  int32_t concurrent;  /* 1: bins side by side on forked streams; 0: one after another */
  int32_t grid_pct;    /* grid of each bin, in percent of its resident CTAs */
  int32_t source;      /* CG_TUNE_* */
  float ms;            /* one run as the autotuner timed it (0 if not timed) */
} cg_schedule;

/* The schedule the plan runs. */
int cg_plan_schedule(const cg_plan* plan, cg_schedule* out);

/* Releases the plan (waits for its outstanding runs first). */
int cg_plan_destroy(cg_plan* plan);

/* The autotuner's cache of schedules, keyed by device name and shape class.
 * It lives in host memory; cg_tune_cache_save writes it to a JSON file (an
 * array with one object per entry, one entry per line: key, precision,
 * order, concurrent, grid_pct, ms) and cg_tune_cache_load merges a file
 * written that way (so a schedule tuned on one machine can be shipped to
 * others with the same device). If the environment variable
 * CGMIMO_TUNE_CACHE names a file, the first plan that needs the cache loads
 * it and every new entry rewrites it. load returns the number of entries
 * read, save the number written, or CG_EINVAL (unreadable or malformed
 * file: nothing merged). Host-only: no CUDA call. */
int cg_tune_cache_load(const char* path);
int cg_tune_cache_save(const char* path);
int cg_tune_cache_size(void);

/* ------------------------------------------------------------------------
 * Serving: a device-resident request loop with continuous batching
 * ------------------------------------------------------------------------ */

/* Server configuration.
 *   capacity          requests in flight at most (ring slots), 1 to 16384
 *   precision         CG_PREC_BF16, CG_PREC_FP16, CG_PREC_BF16X3 or CG_PREC_FP16X3
 *   hbm_budget_bytes  admission limit: input + output bytes of admitted,
 *                     unfinished requests (a request larger than it is CG_ETOOBIG)
 *   max_B, max_R      largest B and R a request may have (they size the kernels)
 *   ctas_per_class    upper limit on the CTAs of each serving kernel; 0 = no
 *                     limit. Every serving CTA fills one SM: the kernel for the
 *                     approximate tracker holds all SMs but 1/16, which the
 *                     exact-tracker kernel holds, so either one always finds
 *                     room when it is relaunched
 *   idle_timeout_ms   a class kernel exits after this long without work and is
 *                     relaunched by the next submit or poll that needs it          */
typedef struct cg_serve_cfg {
  int32_t capacity;
  int32_t precision;
  int64_t hbm_budget_bytes;
  int32_t max_B, max_R;
  int32_t ctas_per_class;
  int32_t idle_timeout_ms;
} cg_serve_cfg;

/* Timing of one request. Host times are CLOCK_MONOTONIC nanoseconds; device
 * times are the GPU global timer (nanoseconds, its own epoch). */
typedef struct cg_req_stats {
  int32_t status;           /* OR of the instances' CG_STATUS_* bits */
  int32_t pad;
  int64_t submit_ns;        /* host, cg_serve_submit accepted the request */
  int64_t complete_ns;      /* host, first cg_serve_poll that saw it complete */
  int64_t device_first_ns;  /* device, its first instance was claimed */
  int64_t device_done_ns;   /* device, its last instance was finished */
} cg_req_stats;

typedef struct cg_server cg_server;

/* Creates a server on the current device and starts nothing yet. Requests
 * fall into classes by operation and padded user count (8, 16, 32), and for
 * exact-tracker detection by padded user count too; each class publishes in
 * order through its own ring in pinned, mapped host memory. One persistent
 * kernel serves every class up to 16 users with the exact tracker and every
 * approximate-tracker class: each of its warps takes instances of the oldest
 * request of its home class while there are any, and otherwise of another
 * class that has work, so a request alone on the device is spread over every
 * SM, and requests that arrive while others run are admitted as warps free
 * up. A second kernel serves exact-tracker detection with 32 padded users.
 * Each kernel launches on the first request that needs it, on its own
 * stream, and exits after idle_timeout_ms without work. A served request
 * gives the same bits as the single call of the same precision. Every device
 * wait is bounded. */
int cg_serve_create(const cg_serve_cfg* cfg, cg_server** out);

/* Non-blocking submit of one request (a cg_desc with 1 <= n_inst < 2^24
 * whose DEVICE buffers stay valid until it completes). Returns CG_EAGAIN when
 * all ring slots are in use or admitting it would exceed the HBM budget (poll
 * and retry), CG_EINVAL for an invalid request, CG_ETOOBIG when it alone
 * exceeds the budget or has 2^24 instances or more; on success *ticket
 * identifies it. A request's bytes count against the budget until it
 * completes; its slot stays in use until a cg_serve_poll has reported it
 * done, so poll every ticket until done. Submitting makes no CUDA call: the
 * request is published through pinned, mapped host memory.
 * The server's kernels run on streams of their own and may start on the
 * request at once: its inputs must already hold their values, and no other
 * work may touch its outputs, when submit is called (synchronise the stream
 * that produced them first). */
int cg_serve_submit(cg_server* s, const cg_desc* req, uint64_t* ticket);

/* *done = 1 once every instance of the request is finished and its outputs
 * are visible to the host; stats (may be NULL) are filled when done. The
 * first poll that reports done releases the ticket's slot; later polls of
 * the same ticket report done again until the slot is reused by a newer
 * request, after which they return CG_EINVAL. Polling makes no CUDA call
 * unless the request's class kernel has exited and must be relaunched. */
int cg_serve_poll(cg_server* s, uint64_t ticket, int32_t* done, cg_req_stats* stats);

/* Stops the class kernels (bounded wait) and frees the server. Requests still
 * in flight may not complete. Returns CG_ETIMEDOUT, leaving the server's
 * memory allocated, if a kernel did not stop in time. */
int cg_serve_destroy(cg_server* s);

/* ------------------------------------------------------------------------
 * Batched problems without any allocation
 * ------------------------------------------------------------------------ */

/* Capacity of cg_batch_run_static per call. */
#define CG_STATIC_MAX_PROBLEMS 4096
#define CG_STATIC_MAX_INSTANCES 65536

/* The paper has no counterpart to this entry point; it serves callers that
 * are not allowed to allocate. A real-time receiver that runs detection
 * once per slot under a sub-millisecond deadline cannot call cudaMalloc or
 * cudaFree in that loop: both may synchronise the device and take unbounded
 * time, so such code allocates everything at start-up. Code that works
 * inside a device-memory budget owned by another allocator is in the same
 * position. cg_plan_create keeps its work tables in memory it allocates;
 * this call runs the same batched kernels with those tables in a static
 * device array of the library instead (about 1 MiB, held by every GPU that
 * loads the library until the process exits), and it calls no allocating
 * routine.
 *
 * Arguments: descs is a HOST array of n problems with the meaning of
 * cg_desc; all buffers they name are caller-provided DEVICE memory.
 * precision is CG_PREC_BF16, CG_PREC_FP16, CG_PREC_BF16X3 or
 * CG_PREC_FP16X3 (no autotuning). Work is enqueued on `stream`; the call
 * returns once the descriptor copy is queued, and the host array may be
 * reused at once.
 *
 * Limits: more than CG_STATIC_MAX_PROBLEMS problems or more than
 * CG_STATIC_MAX_INSTANCES instances in total returns CG_ETOOBIG with no
 * work enqueued; invalid descriptors return CG_EINVAL, also with no work
 * enqueued (every bin's launch shape is checked before the first copy).
 * CG_ECUDA from a copy or a launch may leave the work of earlier bins
 * enqueued. Descriptors with n_inst = 0 are validated and then skipped.
 * Exact-tracker detection runs in bins of its own, as in cg_plan_create.
 *
 * Each call looks up the device address of the static array on the
 * current device (make the device current first); the first call on a
 * device may load the library's device code, so make one call ahead of
 * deadline-bound use. Every call reuses the same array, which keeps the previous
 * call's contents; the call resets the parts that must start at zero.
 * Calls whose work overlaps on the GPU (different streams, or other
 * threads) race on the array: order them on one stream. */
int cg_batch_run_static(const cg_desc* descs, int64_t n, int32_t precision, void* stream);

/* Limit on the device-side waits for an instance's inputs: those of the
 * FP32 kernels (CG_PREC_FP32, and the implicit and CGLS modes), which fetch
 * them with bulk copies into shared memory, and those of CG-D single calls
 * in the tensor-core precisions, which stage H and Y with tensor-map copies
 * (TMA). After timeout_ns nanoseconds of GPU time without the copies
 * landing, the instance's status gets CG_STATUS_TIMEOUT, its CTA (FP32) or
 * warp (TMA) issues nothing more, waits (at most 2 s) for the copies still
 * in flight and stops, and the call completes without a fault; the
 * remaining instances of that CTA or warp are left unwritten. 0 restores
 * the default of 2 s; the limit applies to calls made after it is set, in
 * every thread. The paper has no counterpart: it exists so that the timeout
 * path can be exercised. Returns CG_EINVAL outside [0, 60 s]. The other
 * tensor-core paths stage their inputs with copies that always complete and
 * have no such wait. */
int cg_set_wait_limit(int64_t timeout_ns);

/* Frees the workspace of the *_host calls on the current device. */
int cg_release_workspace(void);

/* Human-readable name of a CG_* return code (static string, never NULL). */
const char* cg_strerror(int code);

/* Library version as major * 10000 + minor * 100 + patch. */
int cg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CGMIMO_H */
