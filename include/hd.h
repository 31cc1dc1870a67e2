/*
 * hd.h -- C ABI of the GB300 hybrid-dealiased convolution library (libhd.so).
 *
 * Method: Murasko & Bowman, "Hybrid Dealiasing of Complex Convolutions",
 * arXiv 2303.17510.  A general convolution maps A inputs of length L,
 * zero padded to at least the dealiasing length M, to B outputs whose DFT is
 * a pointwise function `mult` of the inputs' DFTs (Section 2, problem
 * statement).  The library pads each input explicitly to p*m, implicitly to
 * q*m, and computes the result one residue contribution at a time
 * (Section 2.2, Alg. convolve / convolveX): per residue, A forward
 * transforms, `mult`, B backward transforms accumulated into the output;
 * the sum is divided by q*m.
 *
 * Conventions shared by every entry point
 *   - All data are complex, interleaved (re, im): HD_F32 = two floats,
 *     HD_F64 = two doubles.
 *   - zeta_N = exp(2 pi i / N); forward transforms use zeta^{+}, backward
 *     transforms zeta^{-} (Section 2).
 *   - Stored layout of one 1D array (per axis for N-D arrays):
 *       HD_COMPLEX    f_0 .. f_{L-1}                       (L values)
 *       HD_CENTERED   f_c at stored index c + floor(L/2),   (L values)
 *                     c = -floor(L/2) .. L-floor(L/2)-1     (Section 3)
 *       HD_HERMITIAN  f_0 .. f_{ceil(L/2)-1} of an array with
 *                     f_{-c} = conj(f_c); Im f_0 is ignored (Section 4).
 *     Outputs use the same stored layout as the inputs: the first L values
 *     of the linear convolution (complex), the centered range (centered) or
 *     the non-negative half (Hermitian).  Results are already divided by q*m.
 *   - Device pointers are raw CUDA device addresses on the plan's device;
 *     `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous with respect to the host and stream ordered.
 *   - The caller owns every input and output buffer.  A plan owns its
 *     twiddle tables and its scratch memory; it is not re-entrant across
 *     concurrent streams.
 *   - Errors: invalid arguments return HD_ERR_INVALID, unsupported shapes
 *     HD_ERR_UNSUPPORTED, M below the dealiasing bound HD_ERR_ALIASED, device
 *     allocation failures HD_ERR_NOMEM, CUDA errors HD_ERR_CUDA (and make the
 *     plan's status sticky: later calls on that plan return HD_ERR_CUDA).
 *     A failed call writes nothing to caller buffers except, for
 *     HD_ERR_CUDA, what kernels already launched may have written.
 */
#ifndef HD_H
#define HD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HD_OK = 0,
    HD_ERR_INVALID = 1,
    HD_ERR_UNSUPPORTED = 2,
    HD_ERR_NOMEM = 3,
    HD_ERR_CUDA = 4,
    HD_ERR_TIMEOUT = 5,
    HD_ERR_ALIASED = 6,
    HD_ERR_SCRATCH_LIMIT = 7
} hd_status;

enum { HD_COMPLEX = 0, HD_CENTERED = 1, HD_HERMITIAN = 2 };
enum { HD_F32 = 0, HD_F64 = 1 };
/* The pointwise mult from the A transformed inputs to the B transformed
 * outputs (Section 2).
 * HD_MULT_PRODUCT: A = 2, B = 1, F1*F2 (the binary convolution of Section 2).
 * HD_MULT_SUM_PAIRS3: A = 3, B = 1, F1F2 + F2F3 + F3F1, a sum of binary
 * products; it dealiases at the binary bound.
 * HD_MULT_BASDEVANT2: A = 2, B = 2, (F1 F2, F1^2 - F2^2): from the velocity
 * components u, v of a 2D incompressible flow, the products u v and
 * u^2 - v^2 of its nonlinear term in Basdevant's form (Section 9 counts
 * A = B = 2).  Binary bound; 1D plans (fused kernel, S up to 4096 FP32 /
 * 2048 FP64; FP32 from S = 512 on unless a candidate of hd_enumerate_candidates
 * is given; larger transforms on the split path) and 2D/3D plans.
 * HD_MULT_BASDEVANT3: A = 3, B = 5, (F1 F2, F2 F3, F3 F1, F1^2 - F3^2,
 * F2^2 - F3^2): from the velocity components u, v, w of a 3D incompressible
 * flow, the products u v, v w, w u, u^2 - w^2 and v^2 - w^2 of its nonlinear
 * term in Basdevant's form (Section 9 counts A = 3, B = 5).  Binary bound; 1D
 * plans (fused kernel: the five residue sums live in shared memory, so FP32
 * transforms up to S = 1024 and FP64 up to 512 for short rows; larger ones on
 * the split path) and 2D/3D plans.
 * HD_MULT_MHD3: A = 6, B = 8: from the Elsasser components z+ = u + b
 * (inputs 0, 1, 2) and z- = u - b (inputs 3, 4, 5) of a 3D incompressible
 * magnetohydrodynamic flow, the eight entries of the traceless part of the
 * flux tensor T_ij = z-_i z+_j: T_01, T_02, T_10, T_12, T_20, T_21,
 * T_00 - T_22, T_11 - T_22 (Section 9 counts A = 6, B = 8 without giving the
 * form; the trace, like that of Basdevant's velocity tensor, goes into the
 * pressure).  Binary bound; 1D plans (fused kernel: the eight residue sums
 * live in shared memory, so FP32 transforms up to S = 1024 and FP64 up to 512
 * for short rows; larger ones on the split path) and 2D/3D plans.  Ragged
 * batches take the single-output mults only. */
enum { HD_MULT_PRODUCT = 0, HD_MULT_SUM_PAIRS3 = 1, HD_MULT_BASDEVANT2 = 2, HD_MULT_BASDEVANT3 = 3, HD_MULT_MHD3 = 4 };

typedef struct hd_plan hd_plan;

/* Full plan description.  Axis 0 is the outermost axis; for ndim = 1 only
 * index 0 is used.  For N-D plans the innermost axis is contiguous and
 * axis i has stride row_pitch[i] elements (0 = packed).  kind applies to the
 * innermost axis; outer axes are HD_COMPLEX when kind is HD_COMPLEX and
 * HD_CENTERED otherwise (Section 5, Hermitian data: centered outer axes,
 * Hermitian innermost axis).  m[i] = 0 selects parameters automatically;
 * p[i], q[i] = 0 derive them from m (Eq. pqdef1, Alg. convolve/convolveX,
 * Section 6.1-6.2).  D[i], residues per pass (Section 6.5): 0 selects the
 * grouping automatically.  On the outer axes of N-D plans all residues of an
 * axis run in one block by default; fewer residues per block (D[i] < n) are
 * allowed on the outermost axis only (a middle axis of a 3D plan writes its
 * outputs over its inputs, so it reads all of them first).  On a 1D axis
 * whose residue transforms fit one CTA (complex or centered data), D > 1 runs
 * D residues at once on a thread-block cluster of D * A CTAs (for few
 * convolutions; D <= n, D * A <= 8).  On a 1D axis on the split path (larger
 * transforms), 1 < D < n processes the residues in blocks of D, whose
 * contributions are added into the output, so the work buffer holds A * D * S
 * values per instance instead of A * n * S; such plans cannot write over
 * their inputs (HD_ERR_INVALID at the call).  HD_ERR_UNSUPPORTED for a D the
 * axis cannot take.  flags: 0, or HD_PLAN_NO_WORK_BUFFER (below);
 * unknown bits are HD_ERR_INVALID.  Zero-initialize the struct (memset or
 * = {0}) so that fields added at its end later read as 0. */
typedef struct {
    int ndim;
    int64_t L[3];
    int64_t M[3];
    int A;
    int B;
    int kind;
    int dtype;
    int mult;
    int64_t m[3];
    int64_t p[3];
    int64_t q[3];
    int D[3];
    int64_t row_pitch[3];
    int flags;
} hd_desc;

/* Plan flag, 1D plans only (N-D plans return HD_ERR_UNSUPPORTED): a plan whose
 * residue transforms take the split path allocates no work buffer of its own.
 * Only hd_convolve_batched_noalloc runs such a plan (hd_convolve and
 * hd_convolve_batched return HD_ERR_UNSUPPORTED on it); on the fused path the
 * flag changes nothing, since no work buffer is needed there. */
enum { HD_PLAN_NO_WORK_BUFFER = 1 };

/* Derive (p, q, n) from (kind, L, M, m): Eq. pqdef1 with Alg. convolve
 * (complex: p = ceil(L/m); p <= 2: q = n = ceil(M/m); p > 2: n =
 * ceil(M/(p m)), q = n p) or Alg. convolveX with Section 6.2 (centered and
 * Hermitian: p = 2 ceil(L/(2m)), n = ceil(2M/(p m)), q = n p / 2).  n is the
 * number of residue contributions.  Host only; no device is needed.
 * Returns HD_ERR_INVALID for non-positive L, M, m or an unknown kind. */
hd_status hd_derive_params(int kind, int64_t L, int64_t M, int64_t m, int64_t* p, int64_t* q, int64_t* n);

/* Smallest dealiasing length for L stored-layout outputs (host only):
 * complex 2L-1 (Section 2, M = sum L_i - (A-1)); centered L + floor(L/2);
 * Hermitian the centered bound of the odd expanded length 2 ceil(L/2) - 1.
 * The sum-of-pairs and Basdevant mults have the binary bounds.  Returns -1 on
 * bad input. */
int64_t hd_dealias_bound(int kind, int mult, int64_t L);

/* 1D complex FP32 plan.  (A, B) = (2, 1) selects HD_MULT_PRODUCT, (3, 1)
 * HD_MULT_SUM_PAIRS3, (2, 2) HD_MULT_BASDEVANT2, (3, 5) HD_MULT_BASDEVANT3, (6, 8) HD_MULT_MHD3; other (A, B) are
 * HD_ERR_INVALID.  m = 0 selects parameters automatically
 * (tuned cache, learned selector, else a cost model); nonzero m, p, q are
 * validated: p m >= L, q m >= M, and p > 2 requires q % p == 0 (complex).
 * An explicit plan (p = q = 1, m >= M) is always legal.  D as in hd_desc.
 * *out receives the plan or NULL on error. */
hd_status hd_plan_create(hd_plan** out, int64_t L, int64_t M, int A, int B, int64_t m, int64_t p, int64_t q,
                         int D);

/* General plan (kind, dtype, mult, 1-3 dimensions).  Same validation as
 * hd_plan_create per axis; centered/Hermitian axes need p even (or the
 * explicit p = q = 1) and q % (p/2) == 0. */
hd_status hd_plan_create_ex(hd_plan** out, const hd_desc* d);

/* One convolution: f[a] (a < A) are device pointers to the A stored
 * inputs, h[b] (b < B) to the B outputs.  h[b] may equal f[b] for every
 * b < B (in place, allowed because A >= B: the inputs are read before any
 * output is written); other overlaps are not allowed. */
hd_status hd_convolve(const hd_plan* plan, const void* const* f, void* const* h, void* stream);

/* `count` independent convolutions of one plan: instance i of input a
 * starts at f[a] + i*batch_stride elements (likewise h[b]).  batch_stride
 * >= the stored length of one instance (all stored values for N-D plans).
 * count = 0 is a no-op. */
hd_status hd_convolve_batched(const hd_plan* plan, int64_t count, const void* const* f, void* const* h,
                              int64_t batch_stride, void* stream);

/* Partial convolution over a range of residues (Section 2.2: the transformed
 * residues are independent and each one's backward transform is added into the
 * output, so the output is the sum of the n residue contributions).  Writes to
 * h[b] the sum of the contributions of residues r_begin <= r < r_end of the
 * plan's outermost axis (for N-D plans, the residues of axis 0; every residue
 * of the inner axes), divided by q m like the whole result.  Summing the
 * outputs of calls whose ranges partition [0, n) gives hd_convolve_batched's
 * result up to rounding: this is how a convolution is split across GPUs, each
 * taking a residue range and the partial outputs summed by one reduction.
 * n is hd_plan_get_axis_params(plan, 0, ...)'s n.  Hermitian 1D plans transform
 * residues in pairs (r, r + 1) starting at r_begin.
 *   - 0 <= r_begin <= r_end <= n, else HD_ERR_INVALID; r_begin = r_end writes
 *     zeros to the outputs.
 *   - Outputs must not overlap the inputs when the range is a proper part of
 *     [0, n) (HD_ERR_INVALID where the library can tell); ragged plans are
 *     HD_ERR_INVALID.
 * Other arguments and results are those of hd_convolve_batched. */
hd_status hd_convolve_residues(const hd_plan* plan, int64_t r_begin, int64_t r_end, int64_t count,
                               const void* const* f, void* const* h, int64_t batch_stride, void* stream);

/* Parameters actually used (per axis 0): m, p, q, D and the plan's device
 * scratch bytes.  Any output pointer may be NULL. */
hd_status hd_plan_get_params(const hd_plan* plan, int64_t* m, int64_t* p, int64_t* q, int* D,
                             size_t* scratch_bytes);

/* Parameters of one axis (0 = outermost) of a plan: (m, p, q, D) as in the
 * paper, the residue transform size S and the residue count n. */
hd_status hd_plan_get_axis_params(const hd_plan* plan, int axis, int64_t* m, int64_t* p, int64_t* q, int* D,
                                  int64_t* S, int64_t* n);

/* Residue contribution r of one stored 1D input (the forward residue
 * transform alone, without mult or the backward transform).  Writes the values of residue r in the order the
 * paper's transforms return them (Section 2.2 forward1/forward2: F_{q l + r},
 * l < m; Section 6.1-6.2 inner: F[u m + l] = F_{q l + u n + v}), i.e. m
 * values for complex p <= 2 and centered/Hermitian p = 2, p m values for
 * complex p > 2, p m / 2 for centered/Hermitian p > 2.  For Hermitian
 * plans the values are real and stored with zero imaginary part.  r < n.
 * 1D plans only. */
hd_status hd_forward_residue(const hd_plan* plan, const void* f, int64_t r, void* out, void* stream);

/* ---------------------------------------------------------------------------
 * Parameter selection (the paper's optimizer, Section 7: scan m, D and the
 * transform variant, time each candidate, keep the fastest).
 * ------------------------------------------------------------------------- */

/* One legal, supported parameter choice for a 1D plan and its kernel
 * variant: (m, p, q, D) as in the paper; S the size-S FFT each residue uses
 * (m, p m or p m / 2), n the residue count, E values per thread, minb the
 * register variant (1 or 2 CTAs per SM), comp compensated residue sums.
 * ms: measured time of one batched call in milliseconds (0 if untimed). */
typedef struct {
    int64_t m, p, q;
    int D;
    int64_t S, n;
    int E, minb, comp;
    double ms;
} hd_candidate;

/* Lists the legal, supported candidates of a 1D description (host only; no
 * device needed).  Writes up to cap entries to out (may be NULL with cap 0)
 * and the total count to *count. */
hd_status hd_enumerate_candidates(const hd_desc* d, hd_candidate* out, int cap, int* count);

/* Times every candidate on the current device for a batch of `count`
 * instances (inputs allocated and freed by the call; `reps` timed launches
 * each, median kept), fills out[0..*n) with ms set, and records the fastest
 * in the process-wide tuning cache used by plans with m = 0.  Ties within
 * 1% prefer the smaller q m, then the smaller m.  best may be NULL. */
hd_status hd_autotune(const hd_desc* d, int64_t count, int reps, hd_candidate* out, int cap, int* n,
                      hd_candidate* best);

/* Plan for an explicit candidate (as returned by the two calls above). */
hd_status hd_plan_create_candidate(hd_plan** out, const hd_desc* d, const hd_candidate* c);

/* Process-wide tuning cache: entries are keyed by (dtype, kind, mult, L, M).
 * hd_tune_cache_put stores c for the description; hd_tune_cache_get returns
 * HD_OK and fills c when an entry exists, HD_ERR_INVALID otherwise;
 * hd_tune_cache_clear empties it. */
hd_status hd_tune_cache_put(const hd_desc* d, const hd_candidate* c);
hd_status hd_tune_cache_get(const hd_desc* d, hd_candidate* c);
hd_status hd_tune_cache_clear(void);

/* ---------------------------------------------------------------------------
 * Learned parameter selector (not in the paper; it stands in for the timed
 * search of Section 7).  A small MLP predicts the log time of one convolution
 * for a (problem, candidate) pair; an installed ensemble picks the candidate
 * with the lowest mean prediction.  Training runs on the GPU with the
 * library's own kernels: tanh hidden layers, a linear output, mean squared
 * error, Adam (beta1 0.9, beta2 0.999, eps 1e-8).  FP32.
 * ------------------------------------------------------------------------- */

typedef struct hd_mlp hd_mlp;
#define HD_SELECTOR_FEATURES 13

/* Network with nlayers dense layers of sizes dims[0] -> dims[1] -> ... ->
 * dims[nlayers] (the last must be 1); parameters start at zero. */
hd_status hd_mlp_create(hd_mlp** out, int nlayers, const int* dims);
/* Parameter count: for each layer W (dims[l+1] x dims[l], row-major) then b. */
int64_t hd_mlp_num_params(const hd_mlp* m);
/* Host <-> device copies of the parameter vector (set also resets Adam). */
hd_status hd_mlp_set_params(hd_mlp* m, const float* host);
hd_status hd_mlp_get_params(const hd_mlp* m, float* host);
/* Predictions for N rows of X (device, N x dims[0] row-major) into Y (device, N). */
hd_status hd_mlp_forward(hd_mlp* m, const float* X, int64_t N, float* Y, void* stream);
/* Mean squared error against targets t (device, N) and its gradient (kept on
 * the device; copied to grads_host, when non-NULL, in the parameter order).
 * Synchronizes the stream; loss may be NULL. */
hd_status hd_mlp_gradients(hd_mlp* m, const float* X, const float* t, int64_t N, float* loss, float* grads_host,
                           void* stream);
/* One Adam step with learning rate lr on the batch (X, t); loss (if non-NULL)
 * receives the loss before the step (synchronizes the stream). */
hd_status hd_mlp_train_step(hd_mlp* m, const float* X, const float* t, int64_t N, float lr, float* loss,
                            void* stream);
hd_status hd_mlp_destroy(hd_mlp* m);

/* The HD_SELECTOR_FEATURES inputs of a (1D description, candidate) pair:
 * log2 L/16, log2 M/16, L/M, A-2, centered, Hermitian, FP64, log2 S/16,
 * log2 n/8, (n S - M)/M, split path, E/16, minb-1. */
hd_status hd_selector_features(const hd_desc* d, const hd_candidate* c, float* out);

/* Installs k trained networks (owned by the caller, kept alive while
 * installed) as the process-wide selector used by plans with m = 0 after the
 * tuning cache.  The ensemble is unsure about a problem when the spread (std.
 * dev.) of its predictions for the chosen candidate exceeds sigma, or when its
 * members disagree on the best candidate and the predicted log-time margin to
 * the second best is below tau.  fallback = 1: an unsure choice is replaced by
 * the timed search (hd_autotune); 0: the ensemble's choice is used anyway. */
hd_status hd_selector_install(hd_mlp* const* models, int k, float tau, float sigma, int fallback);
hd_status hd_selector_clear(void);
/* The installed selector's choice for a 1D description (HD_ERR_INVALID when
 * none is installed); *confident = 1 when the ensemble is sure. */
hd_status hd_selector_choose(const hd_desc* d, hd_candidate* out, int* confident);

/* ---------------------------------------------------------------------------
 * Ragged batches: many 1D convolutions of different L, M, A and kind in one
 * persistent kernel launch, replayed from a CUDA graph.  (The paper computes
 * C copies of one transform with multithreading, Section 7; a ragged batch
 * generalizes the copies to different sizes.)  FP32, complex and centered
 * kinds, A = 2 (product) or 3 (sum of pairwise products), B = 1.
 * ------------------------------------------------------------------------- */

/* One ragged plan for n 1D descriptions (ndim = 1 each).  Per instance,
 * m = 0 picks parameters from the tuning cache if it holds the instance's
 * (dtype, kind, mult, L, M), else from the learned selector if one is loaded
 * and confident, else from the cost model.  Allocates the queue of tiles, the
 * graph and the work buffers of the instances whose residue transforms exceed
 * one CTA: those instances are packed into groups that take turns in a ring of
 * four buffers of at most 16 MiB each (larger when one instance needs more),
 * so the work buffers stay in L2 whatever the batch size.  HD_ERR_INVALID on bad descriptions, HD_ERR_ALIASED below a
 * dealiasing bound, HD_ERR_UNSUPPORTED when no parameters fit. */
hd_status hd_ragged_create(hd_plan** out, int64_t n, const hd_desc* descs);

/* As hd_ragged_create with the candidate of every instance given (c[i]
 * from hd_enumerate_candidates or hd_autotune for descs[i]). */
hd_status hd_ragged_create_candidates(hd_plan** out, int64_t n, const hd_desc* descs, const hd_candidate* c);

/* Binds device buffers: f holds 3 n host-side entries, f[3 i + a] the device
 * address of input a of instance i (entries a >= A ignored); h holds n output
 * addresses.  Uploads the instance table (synchronously); rebinding is
 * allowed between runs.  h[i] may equal f[3 i]. */
hd_status hd_ragged_bind(hd_plan* plan, const void* const* f, void* const* h);

/* Runs the whole ragged batch: one graph launch (a counter reset and the
 * persistent kernel) on `stream`.  Asynchronous. */
hd_status hd_ragged_run(const hd_plan* plan, void* stream);

/* Synchronizes the stream of the last run and reports its outcome:
 * HD_ERR_TIMEOUT if a dependency wait of the persistent kernel ran past the
 * plan's limit (the affected tiles were skipped), HD_OK otherwise. */
hd_status hd_ragged_status(const hd_plan* plan);

/* Parameters used for instance i. */
hd_status hd_ragged_get_params(const hd_plan* plan, int64_t i, hd_candidate* c);

/* Limit of every dependency wait in the persistent kernel, in nanoseconds
 * (default 2e9).  Re-captures the graph. */
hd_status hd_ragged_set_wait_limit(hd_plan* plan, int64_t ns);

/* Test hook: makes the row tiles of split-path instance i wait for one more
 * column tile than exists, so that the wait runs out (HD_ERR_INVALID for an
 * instance on the fused path). */
hd_status hd_ragged_inject_stall(hd_plan* plan, int64_t i);

/* ---------------------------------------------------------------------------
 * Allocation-free batched convolution (no counterpart in the paper).
 *
 * Some callers cannot allocate device memory when they convolve: a service
 * that reserves all of its GPU memory at start-up and must not grow it while
 * serving, code that runs inside another runtime's memory manager, or a hot
 * loop where a device allocation would synchronize the device and stall other
 * streams.  For plans whose residue transforms are too large for one CTA (the
 * split path, which needs a work buffer of A * n * S values per instance),
 * this entry point uses a fixed work buffer that is part of the library image
 * on each GPU instead of the plan's own buffer, and itself calls no device
 * allocation or free.  The plan is still created beforehand (plan creation
 * allocates its twiddle tables).
 *
 *   - The fixed buffer holds HD_NOALLOC_SCRATCH_BYTES bytes on every GPU that
 *     loads the library, until the process exits.  Batches are processed in
 *     chunks that fit it; a plan whose single instance needs more returns
 *     HD_ERR_SCRATCH_LIMIT before launching anything.
 *   - The first call on a device looks up the buffer's device address on that
 *     device (the device current at the call); make that first call before any
 *     stream capture begins.
 *   - All calls share the buffer and it keeps the last call's contents.  The
 *     kernels write every work-buffer entry before they read it, so nothing
 *     needs clearing, but calls whose kernels overlap on the GPU (different
 *     streams, or several host threads) race on the buffer: order them on one
 *     stream or synchronize between them.
 *   - Plans that use no work buffer (the fused path) return HD_ERR_UNSUPPORTED;
 *     ragged and N-D plans return HD_ERR_INVALID.
 *   - A plan created with the flag HD_PLAN_NO_WORK_BUFFER skips the plan's own
 *     work buffer, so nothing but its twiddle tables is allocated for it.
 *   - Like hd_convolve_batched, the call makes the plan's device current for
 *     its duration (and restores the caller's device).
 * Arguments and results are otherwise those of hd_convolve_batched. */
#define HD_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
hd_status hd_convolve_batched_noalloc(const hd_plan* plan, int64_t count, const void* const* f, void* const* h,
                                      int64_t batch_stride, void* stream);

/* Synchronizes the current device and reports whether any persistent
 * batched kernel launched on it since the last call had a bounded wait on its
 * staging copies run out (HD_ERR_TIMEOUT), HD_ERR_CUDA on a device error,
 * HD_OK otherwise.  Clears the report.  After HD_ERR_TIMEOUT the outputs of
 * every batched call since the last report are undefined (a CTA that gave up
 * leaves its remaining batch elements uncomputed, and waits once more, with the
 * same limit, for its copies in flight before it exits).  (No counterpart in the paper: the persistent kernels stage their
 * inputs with asynchronous bulk copies whose completion they wait for with a
 * time limit.) */
hd_status hd_device_status(void);

/* Arithmetic peak of the current device (no counterpart in the paper; the
 * roofline of the FFT kernels, which run on the CUDA cores): FMA throughput in
 * TFLOP/s (2 flops per FMA lane) measured by the library's own kernels, many
 * CTAs per SM each running independent chains of dependent FMAs, timed with
 * CUDA events over 5 launches after one warm-up launch.  kind: HD_PEAK_F32
 * (scalar FP32 FMA), HD_PEAK_F64 (FP64 FMA) or HD_PEAK_F32X2 (the packed
 * two-lane FP32 FMA of sm_100 and later).  Synchronizes the device; allocates
 * and frees a small output buffer. */
enum { HD_PEAK_F32 = 0, HD_PEAK_F64 = 1, HD_PEAK_F32X2 = 2 };
hd_status hd_alu_peak(int kind, double* tflops);

/* Releases the plan's device memory (after synchronizing its device). NULL ok. */
hd_status hd_plan_destroy(hd_plan* plan);

/* Static string for a status code. */
const char* hd_status_string(hd_status s);

#ifdef __cplusplus
}
#endif

#endif /* HD_H */
