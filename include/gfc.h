/*
 * gfc.h -- C ABI of the GB300 Green Function Convolution (GFC) Poisson solver.
 *
 * GFC (Beaini et al., arXiv 1902.00176) recovers an image from a gradient
 * field (possibly non-conservative) or from a Laplacian by one convolution
 * with a numerical Green's function, done in the Fourier domain:
 *
 *   L      = div E                               (Eq. 3)
 *   G      = F(delta) / F(K_laplace)             (Eq. 19-22, Algorithm A)
 *   I_c    = Re(F^-1(F(L) o G)) + c              (Eq. 23, Algorithm B)
 *
 * Conventions used by every entry point below:
 *  - Fields are contiguous [batch, C, H, W] arrays (row-major, W fastest) in
 *    the plan's storage dtype; each (batch, channel) slice is one independent
 *    solve. Arithmetic is FP32 for every storage dtype.
 *  - gx is the forward difference along W, gy along H:
 *      gx[i,j] ~ I[i,j+1] - I[i,j],  gy[i,j] ~ I[i+1,j] - I[i,j].
 *    The solver accepts any values (non-conservative edits are the point).
 *  - The field is zero-extended into an M x N padded domain (Algorithm A;
 *    pad p, default 4) with the image block at offset (p, p). The DFT makes
 *    that domain a torus; gradients are zero in the pad (zero flux, Sec. 2.2).
 *  - L[p+i, p+j] = gx[i,j] - gx[i,j-1] + gy[i,j] - gy[i-1,j], out-of-range
 *    terms are 0 (so L is supported on (H+1) x (W+1) cells).
 *  - Algorithm A's kernel sign is used (positive Laplacian, -4 centre; Eq. 15
 *    prints the negated kernel). G[0,0] (0/0 in Algorithm A) is set to 0.
 *  - The constant of Eq. 23 is Algorithm B's: the solution at the pad's corner
 *    u[0,0] is subtracted, then the image block is cropped:
 *      out[i,j] = u[p+i, p+j] - u[0,0].
 *  - Size policy GFC_SIZE_SMOOTH (default): M, N are the smallest even 7-smooth
 *    integers >= H + 2p and >= W + 2p; the image stays at (p, p) and the extra
 *    zero rows/columns go to the bottom/right. This is the same least-squares
 *    problem (Sec. 2.2) on a slightly larger torus.
 *
 * Memory: every tensor pointer is caller-owned DEVICE memory on the plan's
 * device, 16-byte aligned, not aliasing any other argument of the same call.
 * The plan owns its tables and its scratch. All solve calls are asynchronous
 * on the plan's stream; a device-side failure is reported by a later call or
 * by gfc_plan_sync. A plan is not thread-safe: one plan serves one stream at
 * a time. Every function returns a gfc_status; on failure gfc_last_error()
 * returns a thread-local message.
 */
#ifndef GFC_H
#define GFC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gfc_plan gfc_plan;

typedef enum { GFC_F32 = 0, GFC_F16 = 1, GFC_BF16 = 2 } gfc_dtype;

typedef enum {
  GFC_OK = 0,
  GFC_ERR_INVALID_ARG = 1, /* bad size, null or misaligned pointer, bad enum */
  GFC_ERR_UNSUPPORTED = 2, /* size or feature the library does not support */
  GFC_ERR_ALLOC = 3,       /* device or host allocation failed */
  GFC_ERR_CUDA = 4,        /* a CUDA runtime call or a launch failed */
  GFC_ERR_TIMEOUT = 5      /* a bounded device-side wait ran out */
} gfc_status;

/* GFC_SIZE_SMOOTH: M = the smallest even 7-smooth size >= H + 2p; N = the
 * smallest row length >= W + 2p that has register-resident row passes
 * (gfc_row_lengths) when W + 2p lies in (136, 2058], else the smallest even
 * 7-smooth size >= W + 2p. Either way the torus is at least Algorithm A's
 * padded size and the extra zero rows and columns go to the bottom and right:
 * the same least-squares problem on a slightly larger torus. GFC_SIZE_EXACT: Algorithm A's own size,
 * M = H + 2p, N = W + 2p, whatever their prime factors: row DFTs by
 * Bluestein's chirp-z for lengths that are not 7-smooth, the column direction
 * by the recursive column solve (any M); H + 2p and W + 2p <= 2048, uniform
 * plans; solves, edited solves and the adjoint (gfc_backward) on that torus. */
typedef enum { GFC_SIZE_SMOOTH = 0, GFC_SIZE_EXACT = 1 } gfc_size_policy;

/* How the column direction of Eq. 23's Green multiply is applied on the
 * register-resident sizes (the row direction is always the real FFT).
 * GFC_COLUMN_RECURSIVE: after the row transforms, column l of the Green
 * spectrum 1/lambda(k, l) is the inverse of the cyclic tridiagonal operator
 * S + S^-1 - b_l along the torus rows (b_l = 4 - 2 cos(2 pi l / N)); it is
 * applied as convolution with that column's Green's function, a two-sided
 * geometric sequence, by one causal and one anticausal first-order recursion
 * (bands of rows with carries swept around the cycle; column l = 0, where the
 * operator is singular, is solved exactly with its mean removed, the reading
 * G[0,0] = 0). Same operator as the column FFTs, O(M) per column instead of
 * two length-M transforms, no spectrum transpose. Used by solves, edited
 * solves and gfc_backward (which sweeps half-bands of rows so its inverse row
 * pass can produce one band of output rows per item; the -(sum grad_out) e_00
 * term enters the sweep and column 0 at torus row 0). Where the adjoint's
 * grad_out rows cannot be bulk-copied (W x element size not a multiple of 16
 * bytes) it runs the column transforms instead.
 * GFC_COLUMN_FFT: column FFT, multiply by G, inverse column FFT. */
typedef enum { GFC_COLUMN_RECURSIVE = 0, GFC_COLUMN_FFT = 1 } gfc_column_solver;

typedef struct {
  int H, W;          /* image height and width, each >= 2 */
  int C, batch;      /* channels and batch size, each >= 1 */
  gfc_dtype dtype;   /* storage dtype of inputs and outputs */
  int pad;           /* p >= 1; 0 selects Algorithm A's pad of 4 */
  int size_policy;   /* gfc_size_policy */
  int chunk;         /* fields per pipeline chunk; 0 lets the plan choose */
  void* stream;      /* cudaStream_t to run on; NULL = the legacy default stream */
  int streams;       /* chunks in flight at once (1..4), each on an internal stream
                        forked from and joined back into the plan's stream; 0 = auto */
  int column_solver; /* gfc_column_solver (register-resident sizes only) */
  int block_items;   /* register-resident passes: 0 = persistent grids (as many blocks as fit,
                        each looping over items), 1 = one block per item (blocks of passes
                        on other streams interleave as soon as blocks retire) */
} gfc_plan_opts;

/* One item of a ragged batch: C fields of H x W, stored contiguously
 * ([C, H, W], W fastest) starting `offset` elements into the caller's arrays. */
typedef struct {
  int H, W, C;
  long long offset;
} gfc_item;

/* Padded-domain size for an H x W image (Algorithm A: size = image + 2 pad,
 * rounded up by the size policy). Host-only, needs no GPU. pad <= 0 selects 4.
 * Writes M, N; returns GFC_ERR_INVALID_ARG for H or W < 2 or null outputs,
 * GFC_ERR_UNSUPPORTED when M or N would exceed the largest supported length. */
gfc_status gfc_padded_size(int H, int W, int pad, int size_policy, int* M, int* N);

/* The row lengths N with register-resident row passes, ascending. Writes up to
 * `capacity` of them to `lengths` (may be NULL when capacity is 0) and returns
 * how many there are. Host-only. */
int gfc_row_lengths(int* lengths, int capacity);

/* Create a plan for batch x C fields of H x W in `dtype` on the current CUDA
 * device (Algorithm A: the Green spectrum is built once per size, in FP64 on
 * the GPU, and stored rounded to FP32; Sec. 3.1.3 keeps it out of the solve
 * time). Synchronous. On success *plan owns device memory until gfc_destroy. */
gfc_status gfc_plan_create(gfc_plan** plan, int H, int W, int C, int batch, gfc_dtype dtype);

/* As gfc_plan_create, with the options above.
 *
 * Two environment variables select equivalent paths, for comparisons (both
 * give results within FP32 rounding of the default; nothing is skipped):
 *   GFC_FORCE_GENERIC (read at plan creation): the shared-memory Stockham
 *     passes instead of the register-resident ones for every size;
 *   GFC_UNFUSED_DIV (read at each call): the divergence of the gradient, or the
 *     adjoint's packing of grad_out, as its own pass before the row transforms
 *     instead of inside them (bit-identical for the forward solve). */
gfc_status gfc_plan_create_ex(gfc_plan** plan, const gfc_plan_opts* opts);

/* Create a plan for a ragged batch of n items of different sizes (each field
 * solved exactly as by a uniform plan of its own size: Eq. 3, Eq. 23,
 * Algorithm B, pad 4, SMOOTH sizes). Items may share or differ in size; one
 * Green spectrum and one pair of twiddle tables is built per distinct padded
 * size. Fields are processed in chunks that keep the spectrum scratch within
 * 1 GB; every pass of a chunk is one launch over all its fields. The solve,
 * Laplacian and backward entry points take the packed arrays (each item at
 * its offset). gfc_plan_padded_size reports the largest M and N.
 * gfc_solve_from_gradient_host is not supported on ragged plans. Synchronous. */
gfc_status gfc_plan_create_ragged(gfc_plan** plan, int n, const gfc_item* items, gfc_dtype dtype);

/* Run later calls of this plan on `stream` (a cudaStream_t of the plan's device). */
gfc_status gfc_plan_set_stream(gfc_plan* plan, void* stream);

/* Report the plan's padded size M x N and pad p (any pointer may be NULL). */
gfc_status gfc_plan_padded_size(const gfc_plan* plan, int* M, int* N, int* pad);

/* Copy the plan's Green spectrum to host memory `host_out` as M x (N/2+1)
 * FP32 values, row-major: G[k,l] = 1 / (M N lambda(k,l)) with
 * lambda = 2cos(2 pi k/M) + 2cos(2 pi l/N) - 4 and G[0,0] = 0 (Eq. 22 with the
 * 1/(MN) of the inverse transform folded in). Synchronous. */
gfc_status gfc_plan_copy_green(const gfc_plan* plan, float* host_out);

/* Solve every field from its gradient (Eq. 3 then Eq. 23 and Algorithm B).
 * gx, gy: [batch, C, H, W] inputs; out: [batch, C, H, W] output, all in the
 * plan's dtype. out may not alias gx or gy. Asynchronous. */
gfc_status gfc_solve_from_gradient(gfc_plan* plan, const void* gx, const void* gy, void* out);

/* Solve every field from a given Laplacian (Eq. 23, Algorithm B): lap is
 * [batch, C, H, W], zero-extended into the padded domain ("padded_L"); its
 * mean is projected out by G[0,0] = 0. out may not alias lap. Asynchronous. */
gfc_status gfc_solve_from_laplacian(gfc_plan* plan, const void* lap, void* out);

/* Adjoint (vector-Jacobian product) of gfc_solve_from_gradient, used to make
 * GFC a network layer (Sec. 4). With y = solve(gx, gy) linear, returns
 * grad_gx = dy/dgx^T grad_out and grad_gy likewise:
 *   z = Crop^T(grad_out) - (sum grad_out) e_00,  w = Re(F^-1(F(z) o G)),
 *   grad_gx[i,j] = w[p+i,p+j] - w[p+i,p+j+1],  grad_gy[i,j] = w[p+i,p+j] - w[p+i+1,p+j].
 * All three arrays are [batch, C, H, W] in the plan's dtype, pairwise
 * non-aliasing. Asynchronous. */
gfc_status gfc_backward(gfc_plan* plan, const void* grad_out, void* grad_gx, void* grad_gy);

/* Batched complex FFT with the library's own mixed-radix engine: `count`
 * contiguous rows of n complex FP32 values (interleaved re, im) from `in` to
 * `out` (which may be the same buffer). dir = -1 forward
 * X[k] = sum x[m] exp(-2 pi i k m / n), dir = +1 unnormalised inverse. n must
 * be 7-smooth and at most 4096. Device pointers; runs on `stream`
 * (cudaStream_t). Asynchronous. Exposed to test the transform on its own
 * (Eq. 17's F). */
gfc_status gfc_fft_c2c(int n, int count, int dir, const void* in, void* out, void* stream);

/* Solve from gradients held in HOST memory (Eq. 3, Eq. 23, Algorithm B), the
 * same computation as gfc_solve_from_gradient with the transfers included:
 * the batch is cut into about 32 steps; per step gx and gy are copied
 * host-to-device, solved, and the result copied device-to-host, with the
 * copies of each step overlapping the solves and copies of the others (three
 * rotating staging buffers and two copy streams owned by the plan, allocated
 * on the first call). gx, gy, out: [batch, C, H, W] host arrays in
 * the plan's dtype; page-locked memory gives asynchronous, overlapped copies.
 * Asynchronous on the plan's stream: `out` is complete once the plan's stream
 * (or gfc_plan_sync) has completed. */
gfc_status gfc_solve_from_gradient_host(gfc_plan* plan, const void* gx, const void* gy, void* out);

/* Per-pass device time and launch counts, for tracing. pass index 0 = row
 * pass (divergence + row transforms; a one-launch solve of a small torus
 * counts here alone), 1 = column direction (the carry sweep of the recursive
 * column solve, or the column transforms and Green multiply), 2 = inverse row
 * pass (offset, crop, cast), 3 = other. */
typedef struct {
  double pass_ms[4];  /* device time summed over launches (only while profiling is on) */
  long launches[4];   /* kernel launches issued (always counted) */
  long calls;         /* solve / backward calls */
  long dropped;       /* launches not timed because the event pool was full */
} gfc_profile;

/* Turn per-launch CUDA-event timing on (enable != 0) or off. Events are
 * recorded on the plan's stream around every kernel launch, from a pool of
 * 65536 event pairs created here. Synchronous when turning on. */
gfc_status gfc_plan_set_profiling(gfc_plan* plan, int enable);

/* Synchronize the plan's stream and return the accumulated profile; reset != 0
 * clears it afterwards. */
gfc_status gfc_plan_get_profile(gfc_plan* plan, gfc_profile* out, int reset);

/* ---- Autotuning ----
 * A plan's results do not depend on how its work is split, only its speed
 * does. gfc_plan_autotune times the plan's candidate splits on synthetic
 * inputs (CUDA events on the plan's stream, after warm-up runs) and keeps the
 * fastest: for uniform plans the column solver (gfc_column_solver, where both
 * exist) and the pipeline split (one chunk of all fields, or on two streams
 * chunks whose hand-off scratch fits 32 or 64 MB of L2, halves or quarters of
 * the batch, thirds on three streams, quarters on four) x the grids
 * (persistent, or one block per item, gfc_plan_opts.block_items); for ragged
 * plans the number of internal
 * streams (1, 2, 4, 8) the per-item sub-plans are spread over. The plan handle
 * stays valid (a uniform plan's internals are replaced by the winner's). With
 * a cache_path (may be NULL) the choice is looked up first under the plan's
 * key (gfc_plan_tune_key: the problem, the device and the library build) and
 * stored after timing, in a text file of "key<TAB>value" lines rewritten
 * atomically (a temporary file renamed). Synchronous; allocates temporary
 * device buffers of the plan's input and output size while timing. */
typedef struct {
  int column_solver;  /* uniform plans: the chosen gfc_column_solver */
  int block_items;    /* uniform plans: the chosen gfc_plan_opts.block_items */
  int chunk;          /* uniform plans: fields per pipeline chunk */
  int streams;        /* uniform plans: chunks in flight */
  int rag_streams;    /* ragged plans: streams of the per-item sub-plans */
  double ms;          /* the winner's time per solve (0 when read from the cache) */
  int candidates;     /* candidates timed (0 when read from the cache) */
  int from_cache;     /* 1 when the choice came from the cache */
  int l2_resident;    /* uniform plans: the winner keeps its spectrum hand-off in L2 (gfc_plan_l2_resident) */
} gfc_tune_result;
gfc_status gfc_plan_autotune(gfc_plan* plan, const char* cache_path, gfc_tune_result* result);

/* 1 when the plan keeps the spectrum that its row pass hands to its inverse
 * row pass in L2, else 0 (-1 for a null plan). That holds for plans with the
 * recursive column solve whose chunk x streams x hand-off bytes per field (the
 * row-major spectrum, the bands' sums and carries) fit 80 MB: the row pass
 * reads the gradients with an evict-first L2 policy and writes the spectrum
 * with an evict-last one, and the inverse row pass drops the spectrum's L2
 * lines after reading them for the last time, so they are never written back.
 * Results do not depend on it (a pure data-placement choice, like the chunk
 * size; the paper has no counterpart). GFC_NO_L2RES=1 at plan creation turns
 * it off. */
int gfc_plan_l2_resident(const gfc_plan* plan);

/* The tuning-cache key of a plan, NUL-terminated in key[capacity]. */
gfc_status gfc_plan_tune_key(const gfc_plan* plan, char* key, int capacity);

/* The tuning cache itself (host-only): gfc_tune_cache_get copies the value of
 * the last entry for `key` into value[capacity] and returns 1, returns 0 when
 * the file or the key is absent, -1 on bad arguments. gfc_tune_cache_put
 * replaces the entry for `key` (keys and values may hold no tab or newline). */
int gfc_tune_cache_get(const char* path, const char* key, char* value, int capacity);
gfc_status gfc_tune_cache_put(const char* path, const char* key, const char* value);

/* Allocation-free solve from gradients, for callers that cannot allocate
 * device memory: plug-ins whose host application owns all device memory,
 * fixed-budget real-time or embedded pipelines, and latency-bound loops where
 * cudaMalloc/cudaFree would synchronise the device. The paper has no
 * counterpart. It solves the problem gfc_solve_from_gradient solves for FP32
 * storage, pad 4 and the SMOOTH size policy, without a plan, on the generic
 * shared-memory passes only (never the register-resident ones a plan uses for
 * some sizes), so the two agree to FP32 rounding (the tests hold them to 1e-5
 * relative L2 and 1e-4 max-abs), not bit for bit.
 * gx, gy, out: `fields` contiguous H x W FP32 fields in device memory of the
 * current device (the caller still owns inputs and outputs), 16-byte aligned;
 * runs on `stream` (cudaStream_t of the current device), asynchronously, one
 * field at a time.
 * Working memory is one library-owned static device array of about 24 MiB that
 * every GPU loading this library holds until the process exits. It limits the
 * padded size to M x ldS <= 2^21 complex elements, where ldS is N/2 + 1
 * rounded up to a multiple of 4 (square images up to 2008 x 2008, which pad
 * to 2016 x 2016); larger sizes return GFC_ERR_UNSUPPORTED before anything is
 * launched. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, which may
 * load the module; the lookup is guarded by a mutex, so first calls from
 * several host threads are safe), so make that first call before any stream
 * capture. Every call rebuilds the Green spectrum and twiddle tables in the
 * array and clears its error word; all calls share the array, so calls that
 * overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller. Calls no cudaMalloc, cudaFree or allocating
 * library routine. */
gfc_status gfc_solve_from_gradient_noalloc(int H, int W, int fields, const void* gx, const void* gy, void* out,
                                           void* stream);

/* ---- Gradient-domain editing around the solve (Sec. 2.3.2, Sec. 3.2) ----
 * These act on [batch, C, H, W] arrays of a uniform plan, in the plan's dtype,
 * on the plan's stream; per-field statistics are FP32 device arrays of
 * batch * C values. Reductions accumulate in FP64 in a fixed order
 * (deterministic). Ragged plans return GFC_ERR_UNSUPPORTED. */

/* Mean and population standard deviation of every field of `fields`
 * (mean, std: device arrays of batch * C floats). */
gfc_status gfc_field_stats(gfc_plan* plan, const void* fields, float* mean, float* std);

/* Colour correction of Eq. 25 (Sec. 3.2.2), in place on a solved `out`:
 * out = (out - mean(out)) * ref_std / std(out) + ref_mean per field, where
 * ref_mean / ref_std are the statistics of the original image (for example
 * from gfc_field_stats). A field with std(out) = 0 becomes ref_mean. */
gfc_status gfc_color_correct(gfc_plan* plan, void* out, const float* ref_mean, const float* ref_std);

/* Gradient thresholding (Sec. 3.1.4, Sec. 3.2.3): pixels whose gradient
 * magnitude |E| = sqrt(gx^2 + gy^2) is below frac * r get gx = gy = 0; other
 * pixels are copied bit for bit. r is `ref` when ref > 0 (the highest
 * possible gradient of an image of known range), else the field's largest
 * magnitude. The decision is taken in FP32 without contraction:
 * m2 = fl(fl(gx*gx) + fl(gy*gy)), r = fl(sqrt(max m2)), t = fl(frac*r), and
 * the pixel is dropped when m2 < fl(t*t). frac >= 0. Writes gx_out, gy_out
 * (which may be gx, gy). */
gfc_status gfc_gradient_threshold(gfc_plan* plan, const void* gx, const void* gy, float frac, float ref,
                                  void* gx_out, void* gy_out);

/* Gradient-domain merging of Eq. 26 (Sec. 3.2.4): |E_p| = |E|^(1-alpha) C^alpha
 * with the orientation of E kept, i.e. E_p = E |E|^(-alpha) C^alpha per pixel
 * (E_p = 0 where |E| = 0). `edges` holds the edge intensity C >= 0 in the
 * plan's layout and dtype; 0 <= alpha <= 1. Writes gx_out, gy_out (which may
 * be gx, gy). */
gfc_status gfc_gradient_merge(gfc_plan* plan, const void* gx, const void* gy, const void* edges, float alpha,
                              void* gx_out, void* gy_out);

/* A gradient edit applied inside a solve (gfc_solve_edited). */
typedef enum { GFC_EDIT_NONE = 0, GFC_EDIT_THRESHOLD = 1, GFC_EDIT_MERGE = 2 } gfc_edit_kind;
typedef struct {
  int kind;          /* gfc_edit_kind */
  float frac, ref;   /* GFC_EDIT_THRESHOLD: as in gfc_gradient_threshold */
  float alpha;       /* GFC_EDIT_MERGE: as in gfc_gradient_merge */
  const void* edges; /* GFC_EDIT_MERGE: edge map [batch, C, H, W] in the plan's dtype */
} gfc_edit;

/* Solve (Eq. 23) from a gradient edited as it is loaded: the same output, bit
 * for bit, as gfc_gradient_threshold or gfc_gradient_merge into temporaries
 * followed by gfc_solve_from_gradient, without the edited gradient ever being
 * written or read back. A threshold with ref <= 0 first reads gx and gy once
 * for the per-field largest magnitudes. Uniform plans only; `edit` is read
 * during the call. */
gfc_status gfc_solve_edited(gfc_plan* plan, const void* gx, const void* gy, const gfc_edit* edit, void* out);

/* The gradient-domain editing flow of Sec. 3.1.1 (Fig. 1) in one call: edit
 * (optional), solve (Eq. 23), colour-correct (Eq. 25, Sec. 3.2.2):
 * out = (I_c - mean(I_c)) * ref_std / std(I_c) + ref_mean per field, I_c the
 * solved field, ref_mean / ref_std the original image's statistics (device
 * arrays of batch * C floats, e.g. from gfc_field_stats); a field with
 * std(I_c) = 0 becomes ref_mean. `edit` may be NULL (no edit) or as for
 * gfc_solve_edited. On plans with the recursive column solve the statistics of
 * I_c are taken while the last pass stores it (per-item FP64 partials, reduced
 * in a fixed order), and one more pass applies the correction in place: out is
 * written once by the solve and read and written once more. Other plans run the
 * solve and then gfc_color_correct. The result matches those two calls to FP32
 * rounding of the statistics. Layout and errors as gfc_solve_edited; ragged
 * plans return GFC_ERR_UNSUPPORTED. */
gfc_status gfc_solve_corrected(gfc_plan* plan, const void* gx, const void* gy, const gfc_edit* edit,
                               const float* ref_mean, const float* ref_std, void* out);

/* Boundary-preserving offset (Sec. 2.3.2): for fields solved from an image
 * that was padded by `ring` pixels on every side, subtract the mean of the
 * solution over that ring (the least-squares constant that makes the padded
 * region zero) and write the inner (H - 2 ring) x (W - 2 ring) block of every
 * field to `inner`, contiguous [batch, C, H - 2 ring, W - 2 ring]. */
gfc_status gfc_boundary_offset(gfc_plan* plan, const void* out, int ring, void* inner);

/* A solve call captured once as a CUDA graph and replayed with one launch.
 * The graph is bound to the plan, the operation and the pointers given at
 * capture; replaying it recomputes the same operation on whatever those
 * buffers hold at replay time. op: 0 = solve from gradient (in0 = gx,
 * in1 = gy, out0 = out), 1 = solve from Laplacian (in0 = lap, out0 = out),
 * 2 = backward (in0 = grad_out, out0 = grad_gx, out1 = grad_gy). Capture runs
 * one ordinary call first (to finish lazy set-up), then records a second one on
 * an internal stream; both run synchronously inside gfc_graph_create. The
 * plan must outlive the graph. */
typedef struct gfc_graph gfc_graph;
gfc_status gfc_graph_create(gfc_plan* plan, int op, const void* in0, const void* in1, void* out0, void* out1,
                            gfc_graph** graph);
/* Launch the captured graph on `stream` (cudaStream_t). Asynchronous. */
gfc_status gfc_graph_launch(gfc_graph* graph, void* stream);
/* Free the graph. NULL is accepted. */
gfc_status gfc_graph_destroy(gfc_graph* graph);

/* Self-test of the failure path of the bounded device-side waits (not from the
 * paper): queues one block on the plan's stream that waits on an mbarrier
 * nothing ever arrives at, with a limit of timeout_ms (1..2000). The wait runs
 * out and records its error code in the plan's device error word, exactly as
 * a bulk copy that never completed would, so the next gfc_plan_sync returns
 * GFC_ERR_TIMEOUT (and clears the word). No GPU fault or hang is involved and
 * the context stays usable. */
gfc_status gfc_plan_selftest_wait(gfc_plan* plan, int timeout_ms);

/* Wait for the plan's stream and report any device-side error since the last
 * sync (GFC_ERR_TIMEOUT for a bounded wait that ran out, GFC_ERR_CUDA otherwise). */
gfc_status gfc_plan_sync(gfc_plan* plan);

/* Free the plan and everything it owns. NULL is accepted. */
gfc_status gfc_destroy(gfc_plan* plan);

/* Thread-local text of the last failure in this thread ("" if none). */
const char* gfc_last_error(void);

/* Static name of a status code. */
const char* gfc_status_string(gfc_status s);

#ifdef __cplusplus
}
#endif

#endif /* GFC_H */
