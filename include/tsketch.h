/*
 * tsketch.h - C ABI of the GB300 sketched discord miner.
 *
 * Implements, on one GPU, the data-parallel path of Yeh et al., "Sketching
 * Multidimensional Time Series for Fast Discord Mining" (arXiv 2311.03393):
 * the random-projection sketch S = R^T T_bar of d z-normalised streams into k
 * sketch streams (Sec. III-A, Alg. 1), the self-join matrix profile of every
 * stream (Def. 6), aggregation over streams (Def. 5), the ranked discords
 * (Alg. 2), dimension addition/deletion by linearity (Sec. III-C) and the
 * adjoint of the discord scores.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All array arguments are DEVICE pointers owned by the caller unless the
 *    parameter name ends in _host.  The library never frees caller memory.
 *  - Every call is asynchronous on the context's CUDA stream and returns a
 *    tsk_status; nothing throws across the ABI.  On failure the reason is in
 *    tsk_last_error(ctx).  Argument errors are detected on the host before
 *    any launch and leave the outputs untouched.
 *  - Batch layout: a batch holds n_series independent multivariate series.
 *    Series s has d streams of series_len_host[s] samples each, stored
 *    stream-major and packed back to back: element (s, j, t) of T lives at
 *        T[d * cum[s] + j * len[s] + t],  cum[s] = sum_{s' < s} len[s'].
 *    A sketch uses the same packing with k streams in place of d.
 *    All streams of one series have the same length (Sec. III-C advises that
 *    only streams starting at the same time be combined).
 *  - Stream layout (matrix profile calls): n_streams streams of
 *    stream_len_host[q] samples packed back to back, X[cum[q] + t].  Per
 *    stream the profile has l = len - m + 1 entries; P and I use the same
 *    packing as X (entry i of stream q at cum[q] + i) and the entries
 *    i >= l of each stream are set to NaN / -1.
 *  - Workspace: the context owns a grow-only device workspace.  A call that
 *    needs more than it holds allocates (cudaMalloc) first; call
 *    tsk_reserve() beforehand when the calls will be captured in a CUDA graph
 *    (growing during capture fails with TSK_ERR_OOM).
 *  - Device-side problems (non-finite input) set an error word that
 *    tsk_sync() reports as TSK_ERR_NONFINITE.  No kernel traps or spins.
 */
#ifndef TSKETCH_H
#define TSKETCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSK_API __attribute__((visibility("default")))

typedef int32_t tsk_status;
enum {
  TSK_OK = 0,
  TSK_ERR_INVALID_ARG = 1,  /* bad shape, size, pointer or enum; nothing launched      */
  TSK_ERR_CUDA = 2,         /* a CUDA runtime call failed (message has the CUDA error) */
  TSK_ERR_OOM = 3,          /* workspace could not grow                                */
  TSK_ERR_UNSUPPORTED = 4,  /* valid request outside what this build implements        */
  TSK_ERR_TIMEOUT = 5,      /* tsk_sync deadline passed, or a device-side wait gave up */
  TSK_ERR_NONFINITE = 6     /* a kernel met NaN/Inf in its input                        */
};

/* element types of input series */
enum { TSK_F32 = 0, TSK_F64 = 1 };

/* arithmetic of the sketch S = R^T T_bar */
enum {
  TSK_SKETCH_BF16 = 0, /* T_bar and R rounded to bfloat16 (nearest even, from the
                          float64 value), products summed in float32 on tensor cores;
                          S is float32                                             */
  TSK_SKETCH_FP32 = 1, /* float32 products and sums; S is float32                   */
  TSK_SKETCH_FP64 = 2  /* float64 throughout; S is float64                          */
};

/* arithmetic of the matrix profile */
enum {
  TSK_MP_FP32 = 0, /* float32 diagonal recurrence from periodic anchors (float32
                      from centred values for float32 input, float64 for float64
                      input, at most 8192 rows apart), then an exact re-evaluation
                      of every row's chosen neighbour (compensated float32 sums
                      for float32 input); P is float32                          */
  TSK_MP_FP64 = 1  /* float64 throughout; P is float64                            */
};

typedef struct tsk_ctx tsk_ctx;

/* Create a context on `device`, issuing work on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  *ctx receives the handle. */
TSK_API tsk_status tsk_create(tsk_ctx** ctx, int32_t device, void* cuda_stream);
/* Switch the stream later calls are issued on. */
TSK_API tsk_status tsk_set_stream(tsk_ctx* ctx, void* cuda_stream);
/* Free the context and its workspace (waits for the stream first). */
TSK_API void tsk_destroy(tsk_ctx* ctx);
/* Text of the last error on this context ("" if none).  Valid until the next call. */
TSK_API const char* tsk_last_error(const tsk_ctx* ctx);
/* Grow the workspace to at least `bytes` now (use before graph capture). */
TSK_API tsk_status tsk_reserve(tsk_ctx* ctx, size_t bytes);
/* Bytes of workspace mp_selfjoin needs for this stream layout. */
TSK_API tsk_status tsk_mp_workspace_bytes(tsk_ctx* ctx, int32_t n_streams, const int32_t* stream_len_host,
                                          int32_t m, size_t* bytes_out);
/* Wait until the stream drains, at most timeout_s seconds (<= 0: no limit),
 * then read and clear the device error word.  TSK_ERR_TIMEOUT if the deadline
 * passed (the work keeps running; call again), or if a kernel's bounded wait
 * for its own asynchronous copies ran out (about a second; the results of the
 * calls since the last sync are then invalid). */
TSK_API tsk_status tsk_sync(tsk_ctx* ctx, double timeout_s);
/* Failure-path self-test: issues, on the context's stream, one block whose
 * bounded device-side wait (the kind the sketch kernel uses for its own
 * copies) waits on a barrier nothing completes.  It gives up after about a
 * second and sets the device error word, so the next tsk_sync returns
 * TSK_ERR_TIMEOUT; the context stays usable.  No fault, trap or unbounded
 * wait is involved.  (Not a step of the paper's method.) */
TSK_API tsk_status tsk_selftest_timeout(tsk_ctx* ctx);
/* Rows per matrix-profile work unit (a band of 512 diagonals x `rows` rows):
 * 0 = automatic (about 64 units per resident warp, 2048..8192), else a
 * multiple of 32 in [32, 1 << 20].  Smaller units balance short streams,
 * larger ones amortise the anchors. */
TSK_API tsk_status tsk_set_tile_rows(tsk_ctx* ctx, int32_t rows);
/* Number of kernels this context has launched since creation. */
TSK_API int64_t tsk_launch_count(const tsk_ctx* ctx);

/* Kernel timing: when enabled, CUDA events are recorded on the context
 * stream around every launch of the named kernels (not during graph capture).
 * tsk_profile_read waits for them, returns the summed device time and the
 * launch count since the last read, and clears them. */
enum { TSK_PROF_MP_DIAG = 0, TSK_PROF_SKETCH = 1, TSK_PROF_DIMS = 2, TSK_PROF_COUNT = 3 };
TSK_API tsk_status tsk_profile_enable(tsk_ctx* ctx, int32_t enable);
TSK_API tsk_status tsk_profile_read(tsk_ctx* ctx, int32_t kernel, double* total_ms, int64_t* launches);

/*
 * ts_sketch_build - global z-normalisation and the sketch (Sec. III-A, Alg. 1).
 *
 *   mu[s][j], sigma[s][j] = mean and population std of stream j of series s
 *   T_bar[s][j][t]        = (T[s][j][t] - mu) / sigma   (0 for a constant stream)
 *   S[s][g][t]            = sum_j R[j][g] * T_bar[s][j][t]
 *
 * Alg. 1 is the special case of a count-sketch R (one +-1 per row, at column
 * h(j)); any dense R (e.g. Gaussian) is accepted.
 *   T      : input series, batch layout with d streams, element type t_dtype.
 *   R      : float32, d x k row-major, shared by all series.
 *   S      : output sketch, batch layout with k streams; float32, or float64
 *            when precision == TSK_SKETCH_FP64.
 *   stats  : output float64 [n_series][d][2] = {mu, sigma}; may be NULL.
 * Requires n_series >= 1, d >= 1, 1 <= k <= 4096, every len >= 1.
 */
TSK_API tsk_status ts_sketch_build(tsk_ctx* ctx, const void* T, int32_t t_dtype, int32_t n_series,
                                   const int32_t* series_len_host, int32_t d, const float* R, int32_t k,
                                   int32_t precision, void* S, double* stats);

/*
 * ts_sketch_update_dims - add or delete dimensions by linearity (Sec. III-C).
 *
 * For each listed dimension q (raw streams T_dims, batch layout with nd
 * streams per series): z-normalise it over its whole length and apply
 *   S[s][g][t] += op[q] * R_rows[q][g] * T_bar_dims[s][q][t],  op = +1 add, -1 delete.
 * Deleting a dimension with the same raw stream and R row it was built with
 * restores the sketch without it (up to float32 rounding of S).
 *   R_rows_host : float32 nd x k, HOST memory (copied to the device once per
 *                 distinct content and cached, so a repeated update can be
 *                 captured in a CUDA graph).
 *   op_host     : int8 [nd], each +1 or -1, HOST memory.
 *   S           : sketch from ts_sketch_build (same k, precision), updated in place.
 *   stats       : output float64 [n_series][nd][2] for the listed dims; may be NULL.
 *   dirty_host  : output uint8 [k] HOST memory, 1 for every sketch stream g that
 *                 some row R_rows[q][g] != 0 touched (a count sketch touches one
 *                 stream per dimension, a Gaussian R all k).  Re-profile those.
 */
TSK_API tsk_status ts_sketch_update_dims(tsk_ctx* ctx, void* S, const void* T_dims, int32_t t_dtype,
                                         int32_t n_series, const int32_t* series_len_host, int32_t nd,
                                         const float* R_rows_host, const int8_t* op_host, int32_t k,
                                         int32_t precision, double* stats, uint8_t* dirty_host);

/*
 * ts_sketch_point_update - point updates (Sec. III-C): sample t of dimension
 * j of series s changes by delta, and the sketch follows by linearity,
 * S_g[t] += R[j][g] * delta / sigma_j for every g (Alg. 1's s(j) delta for a
 * count sketch), with the build's normalisation (mean, sigma in stats) held
 * fixed.
 *   S, stats, R : the ts_sketch_build outputs/inputs (S of `precision`'s type).
 *   T           : optional (NULL to skip) device batch layout of the series;
 *                 when given it is updated in place and S moves by R[j][g]
 *                 times the change of the stored sample's normalised value (in
 *                 TSK_SKETCH_BF16 mode: of its bfloat16 rounding), so S stays
 *                 the sketch of the updated T.  Required for TSK_SKETCH_BF16.
 *   upd_*_host  : n_upd host arrays (series, dimension, time, delta); repeated
 *                 points are merged (deltas summed).  The arrays are read
 *                 before the call returns.
 * The changed sketch streams need a new profile (mp_selfjoin or mp_abjoin).
 * Errors: TSK_ERR_INVALID_ARG for NULL arrays, a bad dtype or precision, an
 * update out of range or a non-finite delta; nothing is changed then.
 */
TSK_API tsk_status ts_sketch_point_update(tsk_ctx* ctx, void* S, void* T, int32_t t_dtype, int32_t n_series,
                                          const int32_t* series_len_host, int32_t d, const float* R, int32_t k,
                                          int32_t precision, const double* stats, int32_t n_upd,
                                          const int32_t* upd_series_host, const int32_t* upd_dim_host,
                                          const int32_t* upd_time_host, const double* upd_delta_host);

/*
 * mp_selfjoin - self-join matrix profile of every stream (Def. 6 with
 * T_test = T_train; Def. 3 z-normalised Euclidean distance).
 *
 *   P[q][i] = min over j with |i - j| >= excl of dist(X_q[i:i+m], X_q[j:j+m])
 *   I[q][i] = that j (-1, with P = +inf, when no j is admissible)
 * dist(a, b) = || z(a) - z(b) ||, z with the population std; a constant window
 * (variance <= 1e-12 * max(1, mean^2)) z-normalises to zeros, so two constant
 * windows are at 0 and a constant and a non-constant one at sqrt(m).  Equal
 * distances may resolve to any of the tied j.
 *   X              : streams, stream layout, element type x_dtype.
 *   stream_mask_host: uint8 [n_streams] HOST, 0 = skip the stream (outputs
 *                     untouched); NULL = all.
 *   excl           : exclusion half-width, 1 <= excl (ceil(m/4) is customary).
 *   precision      : TSK_MP_FP32 (P float32) or TSK_MP_FP64 (P float64).
 *   P, I           : outputs, stream layout (I int32).
 * Requires 2 <= m <= 4096 and m <= len for every stream.
 */
TSK_API tsk_status mp_selfjoin(tsk_ctx* ctx, const void* X, int32_t x_dtype, int32_t n_streams,
                               const int32_t* stream_len_host, const uint8_t* stream_mask_host, int32_t m,
                               int32_t excl, int32_t precision, void* P, int32_t* I);

/*
 * mp_selfjoin_update - the self-join profile of float32 streams after point
 * updates: Sec. III-C's point update moves a sketch stream at single times
 * (ts_sketch_point_update), and the profile follows incrementally, the
 * streaming use Sec. III-B names.  A changed sample t moves windows
 * t-m+1 .. t (set A).  Windows of A get their whole row anew; a window whose
 * old nearest neighbour was in A is re-scanned whole; every other window
 * keeps its old value unless a window of A is now nearer.  The result is the
 * profile mp_selfjoin would compute for the updated streams (Def. 6), at a
 * cost of about (2|A| + 512) l + |R| l m operations per stream instead of l^2.
 *   X               : device float32 streams, already updated, stream layout.
 *   stream_len_host : int32 [n_streams] HOST.
 *   m, excl         : as given to the mp_selfjoin call that produced P, I.
 *   P, I            : device float32 / int32, stream layout: on entry the
 *                     profile of the streams before the updates (as
 *                     mp_selfjoin, TSK_MP_FP32, wrote it), on return the
 *                     profile after them.  Streams with no point are untouched.
 *   pt_stream_host, pt_time_host : n_pts HOST (stream, time) pairs, the
 *                     samples that changed (repeats allowed); read before the
 *                     call returns.
 * Errors: TSK_ERR_INVALID_ARG for NULL arrays, bad m / excl, or a point out of
 * range (nothing issued).
 */
TSK_API tsk_status mp_selfjoin_update(tsk_ctx* ctx, const float* X, int32_t n_streams, const int32_t* stream_len_host,
                                      int32_t m, int32_t excl, float* P, int32_t* I, int32_t n_pts,
                                      const int32_t* pt_stream_host, const int32_t* pt_time_host);

/*
 * mp_abjoin - AB-join matrix profile (Def. 6 with T_test != T_train), the
 * form Alg. 2 runs on: for every window i of test stream A_q,
 *   P_a[i] = min over EVERY window j of training stream B_q of dist(A_q[i:i+m], B_q[j:j+m]),
 *   I_a[i] = that j (a tie may return any j at the same distance),
 * and, optionally, the training side's profile against the test stream
 * (P_b, I_b: for every window of B_q its nearest window of A_q).  No
 * exclusion zone; the constant-window rules of mp_selfjoin apply.
 *   A, B        : device streams, packed like mp_selfjoin's X (A: n_pairs
 *                 streams of len_a_host[q] samples; B: n_pairs streams of
 *                 len_b_host[q]); both float32 or both float64 (x_dtype).
 *   P_a, I_a    : device float32 (float64 for TSK_MP_FP64) / int32, packed like
 *                 A (entries past the last window are NaN / -1).
 *   P_b, I_b    : optional (both NULL to skip), packed like B, same types.
 *   precision   : TSK_MP_FP32 (the float32 recurrence with periodic anchors and
 *                 an exact re-evaluation of each chosen neighbour) or
 *                 TSK_MP_FP64 (float64 throughout, lowest index on ties).
 * Errors: TSK_ERR_INVALID_ARG for NULL required arrays, only one of P_b / I_b,
 * a bad dtype or precision, m outside [2, 4096] or a stream shorter than m.
 */
TSK_API tsk_status mp_abjoin(tsk_ctx* ctx, const void* A, const void* B, int32_t x_dtype, int32_t n_pairs,
                             const int32_t* len_a_host, const int32_t* len_b_host, int32_t m, int32_t precision,
                             void* P_a, int32_t* I_a, void* P_b, int32_t* I_b);

/*
 * discord_topk - aggregate over the streams of each series and rank the
 * discords (Def. 5, Alg. 2 extended to a ranked list of K).
 *
 * Series s owns streams s*group .. s*group+group-1 of P/I (stream layout, all
 * of length series_len_host[s], l = len - m + 1 profile entries):
 *   A[i] = max_g P_g[i],  G[i] = the lowest g attaining it.
 * Then K times: i* = argmax A (lowest i on ties), report
 *   idx = i*, grp = G[i*], score = A[i*], nn = I_G[i*][i*]
 * and exclude every i with |i - i*| < topk_excl.  When fewer than K indices
 * remain the rest of the row is idx = grp = nn = -1, score = NaN.
 *   P     : float32 (p_dtype TSK_F32) or float64 (TSK_F64).
 *   outputs: device arrays [n_series][K]; score has P's element type.
 */
TSK_API tsk_status discord_topk(tsk_ctx* ctx, const void* P, int32_t p_dtype, const int32_t* I, int32_t n_series,
                                const int32_t* series_len_host, int32_t group, int32_t m, int32_t K,
                                int32_t topk_excl, int32_t* idx, int32_t* grp, void* score, int32_t* nn);

/*
 * mp_backward - adjoint of the ranked discord scores (not in the paper: the
 * derivative of the definitions above, for attributing a discord to input
 * dimensions).
 *
 * With the selections (idx, grp, nn) of discord_topk held fixed, the loss
 *   L = sum_{s,r} dscore[s][r] * dist(S_s,g[i:i+m], S_s,g[j:j+m])
 * is differentiated through the sketch and the global z-normalisation
 * (bfloat16 rounding is treated as the identity):
 *   d dist/dx = (rho x_hat - y_hat)/(sigma_x dist), d dist/dy = (rho y_hat - x_hat)/(sigma_y dist),
 *   dT_bar = R dS, dR = sum_s T_bar dS^T,
 *   dT_j = (dT_bar_j - mean(dT_bar_j) - T_bar_j mean(dT_bar_j T_bar_j)) / sigma_j.
 * Entries with idx < 0, a constant window or dist = 0 contribute nothing.
 *   dscore, idx, grp, nn : [n_series][K] (float32 / int32).
 *   T, stats, R, S       : the forward's inputs and outputs (S float32).
 *   dT                   : output float32, batch layout with d streams.
 *   dR                   : output float32 d x k (summed over series).
 */
TSK_API tsk_status mp_backward(tsk_ctx* ctx, const float* dscore, const int32_t* idx, const int32_t* grp,
                               const int32_t* nn, int32_t K, const void* T, int32_t t_dtype, const double* stats,
                               const float* R, const float* S, int32_t n_series, const int32_t* series_len_host,
                               int32_t d, int32_t k, int32_t m, float* dT, float* dR);

/*
 * dimension_detection - Alg. 3 (Sec. III-C, "Detection", second phase): the
 * raw dimension behind each discord found on the sketch.
 *
 * For discord r of series s (window i* = idx[s][r] in sketch stream
 * g* = grp[s][r], as returned by discord_topk on the sketch profiles), the
 * group is J_g* = {j : R[j][g*] != 0} (the dimensions a count sketch hashes to
 * g*; every dimension for a dense R).  Each j in J_g* is scored by the 1NN
 * distance of its own window i*:
 *   s_j = min over |t - i*| >= excl of dist(T_j[i*:i*+m], T_j[t:t+m])
 * (Def. 6 at one row, z-normalised distance, the constant-window and
 * no-neighbour rules of mp_selfjoin), and
 *   j* = the first j (ascending) with s_j above every earlier score, from 0;
 *        the lowest j of J_g* when no score exceeds 0; -1 for an empty group.
 * Each s_j is the exact distance of the window the scan chose (re-evaluated
 * with compensated sums); the scan picks it in float32.
 *   T          : device, batch layout of ts_sketch_build (d streams per series,
 *                float32 or float64 per t_dtype).
 *   R          : device float32 d x k (row-major), the sketch matrix.
 *   idx, grp   : device int32 [n_series][K]; idx < 0 marks an empty slot.
 *   dim, dim_nn: device int32 [n_series][K] outputs: j*, and s_j*'s neighbour.
 *   dim_score  : device float64 [n_series][K] output: s_j* (NaN when j* = -1,
 *                +inf when window i* has no admissible neighbour).
 *   dim_scores : optional (NULL to skip) device float64 [n_series][K][d]:
 *                every s_j, NaN for j outside J_g*.
 *   T_sel      : optional (NULL to skip) device buffer of T's element type:
 *                per series s, K streams of series_len_host[s] samples (the
 *                layout ts_sketch_build gives S for k = K), stream r a copy of
 *                T_j* for discord r (zeros when j* = -1), for the optional
 *                refinement (mp_selfjoin over T_sel, then discord_topk with
 *                group 1).
 *   T_train, train_len_host : optional (NULL for the self-join form): the
 *                training series in the same batch layout (d streams per
 *                series, lengths train_len_host[s]).  Then T holds the test
 *                series, s_j = min over EVERY window t of training stream j of
 *                dist(T_j[i*:i*+m], T_train_j[t:t+m]) (Def. 6 AB form, Alg. 3
 *                as printed), excl is ignored, and dim_nn indexes the
 *                training stream.
 *   T_sel_train: optional (needs T_train): the chosen training streams, laid
 *                out like T_sel with the training lengths, for the AB-join
 *                refinement (mp_abjoin of T_sel against T_sel_train).
 * Errors: TSK_ERR_INVALID_ARG for NULL required arrays, a bad dtype,
 * m outside [2, 4096], excl < 1 (self-join form), K < 1, k < 1, d < 1, a series
 * shorter than m, T_train without train_len_host, or T_sel_train without
 * T_train; nothing is issued then.  Out-of-range idx/grp entries are treated
 * as empty slots.
 */
TSK_API tsk_status dimension_detection(tsk_ctx* ctx, const void* T, int32_t t_dtype, int32_t n_series,
                                       const int32_t* series_len_host, int32_t d, const float* R, int32_t k,
                                       int32_t m, int32_t excl, int32_t K, const int32_t* idx, const int32_t* grp,
                                       int32_t* dim, double* dim_score, int32_t* dim_nn, double* dim_scores,
                                       void* T_sel, const void* T_train, const int32_t* train_len_host,
                                       void* T_sel_train);

/*
 * mp_selfjoin_static - the matrix profile of ONE float32 stream, like
 * mp_selfjoin with precision TSK_MP_FP32, but without allocating any device
 * memory and without a context.  The paper has no counterpart; this entry
 * point exists for callers that cannot call cudaMalloc: code that runs after
 * start-up in a real-time monitor that must not allocate, code whose device
 * memory is owned by another framework's pool, or code called back from
 * inside an allocator, where allocating again would deadlock or fail.
 *
 * All scratch (window statistics, the per-window maxima and near-tie
 * candidates, the work list and counters) lives in one 6 MiB array in the
 * library's global device memory; every GPU that loads the library holds that
 * array until the process exits.
 *   X      : device float32 [n] input stream (caller-owned).
 *   P, I   : device float32 / int32 [n] outputs, as mp_selfjoin (entries
 *            i >= l = n - m + 1 are NaN / -1).
 *   cuda_stream : the cudaStream_t the work is issued on (NULL = default).
 * Limits: 2 <= m <= 4096, m <= n, excl >= 1 and l <= 65536 windows; larger
 * inputs are rejected with TSK_ERR_INVALID_ARG before anything is issued.
 * The first call on a device looks up the array's device address and sets the
 * kernels' shared-memory limits for that device (the device current at the
 * call); make that first call before any CUDA-graph stream capture.  Every
 * call uses the same array and leaves its contents behind (the call clears
 * what must start at zero), so calls whose work may overlap on the GPU - on
 * different streams, or from several host threads - race and must be
 * serialised by the caller.  Non-finite input is not reported (no error word
 * is read back); the outputs are then unspecified.
 */
TSK_API tsk_status mp_selfjoin_static(const float* X, int32_t n, int32_t m, int32_t excl, float* P, int32_t* I,
                                      void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TSKETCH_H */
